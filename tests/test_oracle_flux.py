"""Pins of the oracle's gas-kinetic fluxes (Sec. 2 Eq. flux; Sec. 3 Remark 1 Eq. flux-2; Eq. expansion-1).

* time-integral weights against numerical quadrature of Eq. (flux)'s
  coefficients, and the factored differences against sympy;
* tau = 0 at a continuous state: Euler flux in closed form and its time
  derivative dF/dQ . (-sum_e dF_e/dQ dQ/dx_e) by complex-step Jacobians;
* tau > 0 at a continuous linear state: Navier-Stokes flux with mu = tau p,
  bulk viscosity from K internal degrees of freedom, heat flux
  -(mu/Pr) (K+5)/2 grad(p/rho) (Chapman-Enskog limit of the BGK model);
* symmetry: mirror and tangential-swap equivariance of the interface flux;
* dual-number derivatives against central differences.
"""
import math

import numpy as np
import pytest
import sympy as sp
from scipy.integrate import quad

GAM = 1.4
KDOF = (5 - 3 * GAM) / (GAM - 1)


def cons(rho, u, p):
    u = np.asarray(u, dtype=complex if np.iscomplexobj(u) else float)
    return np.array([rho, rho * u[0], rho * u[1], rho * u[2], p / (GAM - 1) + 0.5 * rho * np.dot(u, u)])


def euler_flux(Q, d):
    rho = Q[0]
    u = Q[1:4] / rho
    p = (GAM - 1) * (Q[4] - 0.5 * rho * np.sum(u * u))
    F = rho * u[d] * np.concatenate([[1.0], u, [0.0]])
    F = F.astype(Q.dtype)
    F[1 + d] += p
    F[4] = u[d] * (Q[4] + p)
    return F


def jac(Q, d):
    """dF_d/dQ by complex step (exact to rounding)."""
    J = np.zeros((5, 5))
    h = 1e-30
    for m in range(5):
        Qc = Q.astype(complex)
        Qc[m] += 1j * h
        J[:, m] = euler_flux(Qc, d).imag / h
    return J


def linear_state(seed):
    rng = np.random.default_rng(seed)
    rho, p = rng.uniform(0.6, 1.8), rng.uniform(0.5, 2.5)
    u = rng.uniform(-1, 1, 3)
    Q = cons(rho, u, p)
    dQ = 0.3 * rng.standard_normal((3, 5)) * np.abs(Q)
    return Q, dQ


def ns_flux(Q, dQ, d, mu, Pr):
    """Euler + Navier-Stokes flux along e_d for the BGK gas (mu = tau p)."""
    rho = Q[0]
    u = Q[1:4] / rho
    p = (GAM - 1) * (Q[4] - 0.5 * rho * u @ u)
    # velocity gradients du_j/dx_e and grad(p/rho) from the conservative gradients
    du = np.zeros((3, 3))
    dpr = np.zeros(3)
    for e in range(3):
        drho = dQ[e, 0]
        dm = dQ[e, 1:4]
        du[:, e] = (dm - u * drho) / rho
        dp = (GAM - 1) * (dQ[e, 4] - 0.5 * drho * u @ u - rho * u @ du[:, e])
        dpr[e] = dp / rho - p * drho / rho ** 2
    div = np.trace(du)
    sigma = mu * (du + du.T) - mu * 2.0 / (KDOF + 3) * div * np.eye(3)
    F = euler_flux(Q, d)
    F[1:4] -= sigma[:, d]
    F[4] -= u @ sigma[:, d]
    F[4] -= (mu / Pr) * (KDOF + 5) / 2 * dpr[d]
    return F


def euler_dt_flux(Q, dQ, d):
    dQdt = -sum(jac(Q, e) @ dQ[e] for e in range(3))
    return jac(Q, d) @ dQdt


def coeffs(t, tau):
    E = math.exp(-t / tau)
    return [1 - E, (t + tau) * E - tau, t - tau + tau * E, E, -(tau + t) * E, -tau * E]


@pytest.mark.parametrize("tau,dt", [(1e-5, 1.3e-3), (0.01 * 8e-3, 8e-3), (2e-3, 1e-3), (0.5, 1e-3)])
def test_time_weights_match_quadrature(orc, tau, dt):
    wF, wFt = orc.fit_weights(tau, dt)
    I1 = [quad(lambda t: coeffs(t, tau)[j], 0, dt, epsabs=0, epsrel=1e-13, limit=200)[0] for j in range(6)]
    Ih = [quad(lambda t: coeffs(t, tau)[j], 0, dt / 2, epsabs=0, epsrel=1e-13, limit=200)[0] for j in range(6)]
    for j in range(6):
        # F dt + F_t dt^2/2 = I(dt); F dt/2 + F_t dt^2/8 = I(dt/2)
        A = np.array([[dt, dt * dt / 2], [dt / 2, dt * dt / 8]])
        F, Ft = np.linalg.solve(A, [I1[j], Ih[j]])
        scale = max(abs(F), abs(Ft) * dt, 1e-300)
        assert abs(wF[j] - F) <= 1e-9 * scale + 1e-13
        assert abs(wFt[j] - Ft) * dt <= 1e-8 * scale + 1e-13


def test_time_weight_factored_differences_symbolic():
    t, tau, d = sp.symbols("t tau delta", positive=True)
    c = [1 - sp.exp(-t / tau), (t + tau) * sp.exp(-t / tau) - tau, t - tau + tau * sp.exp(-t / tau),
         sp.exp(-t / tau), -(tau + t) * sp.exp(-t / tau), -tau * sp.exp(-t / tau)]
    Eh = sp.exp(-d / (2 * tau))
    s = 1 - Eh
    factored = [tau * s ** 2, -2 * tau ** 2 * s ** 2 + tau * d * Eh * s, d ** 2 / 4 - tau ** 2 * s ** 2,
                -tau * s ** 2, 2 * tau ** 2 * s ** 2 - tau * d * Eh * s, tau ** 2 * s ** 2]
    for j in range(6):
        I = sp.integrate(c[j], (t, 0, d))
        Ih = sp.integrate(c[j], (t, 0, d / 2))
        diff = sp.simplify(sp.expand(I - 2 * Ih - factored[j]).rewrite(sp.exp))
        assert diff == 0, (j, diff)


def test_tau_zero_weights(orc):
    wF, wFt = orc.fit_weights(0.0, 1e-3)
    np.testing.assert_array_equal(wF, [1, 0, 0, 0, 0, 0])
    np.testing.assert_array_equal(wFt, [0, 0, 1, 0, 0, 0])


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("d", [0, 1, 2])
def test_euler_limit_continuous_state(orc, seed, d):
    Q, dQ = linear_state(seed)
    F, Ft = orc.face_flux(d, Q, dQ, Q, dQ, mu=0.0, tau_eps=0.0, dt=1e-3)
    np.testing.assert_allclose(F, euler_flux(Q, d), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(Ft, euler_dt_flux(Q, dQ, d), rtol=1e-11, atol=1e-12)
    Fc, Ftc = orc.cell_flux(Q, dQ, mu=0.0, dt=1e-3)
    np.testing.assert_allclose(Fc[d], euler_flux(Q, d), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(Ftc[d], euler_dt_flux(Q, dQ, d), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("Pr", [1.0, 0.72])
@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("d", [0, 1, 2])
def test_navier_stokes_limit_continuous_state(orc, seed, d, Pr):
    Q, dQ = linear_state(10 + seed)
    mu = 3e-3
    p = (GAM - 1) * (Q[4] - 0.5 * (Q[1:4] @ Q[1:4]) / Q[0])
    dt = 1e-3
    F, Ft = orc.face_flux(d, Q, dQ, Q, dQ, mu=mu, Pr=Pr, dt=dt)
    ref = ns_flux(Q, dQ, d, mu, Pr)  # tau = mu/p exactly reproduces viscosity mu
    np.testing.assert_allclose(F, ref, rtol=1e-12, atol=1e-12)
    Fc, Ftc = orc.cell_flux(Q, dQ, mu=mu, Pr=Pr, dt=dt)
    np.testing.assert_allclose(Fc[d], ref, rtol=1e-12, atol=1e-12)
    # at a continuous state Eq. (flux) collapses to Eq. (flux-2): same F_t
    np.testing.assert_allclose(Ft, Ftc[d], rtol=1e-11, atol=1e-11)
    if Pr == 1.0:
        np.testing.assert_allclose(Ftc[d], euler_dt_flux(Q, dQ, d), rtol=1e-11, atol=1e-12)


def _two_states(seed):
    QL, dQL = linear_state(100 + seed)
    QR, dQR = linear_state(200 + seed)
    return QL, dQL, QR, dQR


@pytest.mark.parametrize("mu,Pr", [(0.0, 1.0), (2e-3, 1.0), (2e-3, 0.72)])
@pytest.mark.parametrize("seed", range(3))
def test_mirror_equivariance(orc, seed, mu, Pr):
    QL, dQL, QR, dQR = _two_states(seed)
    M = np.diag([1.0, -1.0, 1.0, 1.0, 1.0])
    kw = dict(mu=mu, Pr=Pr, tau_eps=0.02, dt=1e-3)
    F, Ft = orc.face_flux(0, QL, dQL, QR, dQR, **kw)
    # mirror x -> -x: left and right swap, normal momentum and normal derivative flip
    S = np.diag([-1.0, 1.0, 1.0])
    mQL, mQR = M @ QR, M @ QL
    mdQL = S @ dQR @ M.T
    mdQR = S @ dQL @ M.T
    Fm, Ftm = orc.face_flux(0, mQL, mdQL, mQR, mdQR, **kw)
    np.testing.assert_allclose(Fm, -M @ F, rtol=1e-12, atol=1e-12 * np.abs(F).max())
    np.testing.assert_allclose(Ftm, -M @ Ft, rtol=1e-10, atol=1e-10 * np.abs(Ft).max())


@pytest.mark.parametrize("seed", range(3))
def test_tangential_swap_equivariance(orc, seed):
    QL, dQL, QR, dQR = _two_states(seed)
    P = np.eye(5)[[0, 1, 3, 2, 4]]  # swap y and z momentum
    Pd = np.eye(3)[[0, 2, 1]]
    kw = dict(mu=1e-3, Pr=0.72, tau_eps=0.0, dt=1e-3)
    F, Ft = orc.face_flux(0, QL, dQL, QR, dQR, **kw)
    Fs, Fts = orc.face_flux(0, P @ QL, Pd @ dQL @ P.T, P @ QR, Pd @ dQR @ P.T, **kw)
    np.testing.assert_allclose(Fs, P @ F, rtol=1e-13, atol=1e-13 * np.abs(F).max())
    np.testing.assert_allclose(Fts, P @ Ft, rtol=1e-11, atol=1e-11 * np.abs(Ft).max())


def test_flux_of_uniform_state_is_euler(orc):
    Q = cons(1.3, [0.4, -0.7, 0.2], 0.9)
    z = np.zeros((3, 5))
    for d in range(3):
        F, Ft = orc.face_flux(d, Q, z, Q, z, mu=1e-2, tau_eps=0.1, dt=1e-2)
        np.testing.assert_allclose(F, euler_flux(Q, d), rtol=1e-13, atol=1e-14)
        assert np.abs(Ft).max() < 1e-11


def test_dual_numbers_match_central_differences(orc):
    pb = orc.Problem(order=1, nq=2, n=(3, 3, 3), mu=2e-2, tau_eps=0.0)
    from paper_2202_13821_b300 import inputs

    Q = inputs.random_state(pb.n, 1, seed=3, vel=0.5)
    rng = np.random.default_rng(9)
    dQ = rng.standard_normal(Q.shape) * np.abs(Q).max(axis=(1, 2, 3, 4), keepdims=True) * 1e-1
    dmu = 1e-2
    dt = 1e-2
    L, Lt, dL, dLt = orc.residual_jvp(pb, Q, dQ, dmu, dt)
    L0, Lt0 = orc.residual(pb, Q, dt)
    np.testing.assert_array_equal(L, L0)
    h = 1e-6
    pbp = orc.Problem(**{**pb.__dict__, "mu": pb.mu + h * dmu})
    pbm = orc.Problem(**{**pb.__dict__, "mu": pb.mu - h * dmu})
    Lp, Ltp = orc.residual(pbp, Q + h * dQ, dt)
    Lm, Ltm = orc.residual(pbm, Q - h * dQ, dt)
    fd = (Lp - Lm) / (2 * h)
    fdt = (Ltp - Ltm) / (2 * h)
    assert np.abs(dL - fd).max() <= 1e-6 * np.abs(fd).max()
    assert np.abs(dLt - fdt).max() <= 1e-6 * np.abs(fdt).max()
