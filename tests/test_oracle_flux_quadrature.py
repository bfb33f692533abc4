"""Brute-force pin of the interface flux at discontinuous states (Sec. 2, Eq. flux).

The oracle evaluates Eq. (flux) through closed-form Maxwellian moments (recurrences,
erfc), Gaussian elimination and closed-form time weights.  Here the same flux is
computed with none of that machinery: every velocity integral is a quadrature
sum over particle velocities and internal energies, and the time integrals are
quadrature sums over t, so that the distribution function f(t, u, v, w, xi) of
Eq. (flux) is evaluated explicitly at every node.

* Velocity space, for a Maxwellian of density rho, velocity U and lambda =
  rho/(2p): Gauss-Hermite in each full-line velocity component (exact for a
  polynomial times that Gaussian), Gauss-Legendre on a half line u > 0 or
  u < 0 truncated 16/sqrt(lambda) beyond the mean (the Heaviside H(u) of
  Eq. flux), and Gauss-Laguerre in s = xi^2 (the K internal degrees of freedom
  make s Gamma(K/2)-distributed).
* Slopes: <a psi> = dQ/dn / rho and the compatibility condition
  <(a.u) psi + A psi> = 0, with the 5x5 matrix <psi psi^T> summed from the
  same nodes and solved by numpy.
* Q_0 and dQ_0/dn_i from half-space sums of g_l (u > 0) and g_r (u < 0),
  then g_0, abar_i and Abar (the relations below Eq. flux).
* tau = mu/p_0 + tau_eps dt.
* F(t) = sum over nodes of u psi f(t, node) for t at Gauss-Legendre nodes of
  [0, dt] and [0, dt/2]; the linear fit of Eq. (expansion-1) then gives F and
  F_t.  With Pr != 1 the heat flux q(t) = 1/2 <(u - U_0)(|u - U_0|^2 + xi^2) f>
  of the same f, fitted alike, adds (1/Pr - 1) q(t_n) to the energy flux F
  and nothing to F_t (the reading of the Prandtl correction that the oracle
  takes: the fitted slope of q about the fixed U_0 would be a frame shift).

At discontinuous states with tau > 0 the side terms of Eq. (flux), which
carry the side slopes a^l_i, A^l, a^r_i, A^r, differ from their equilibrium
counterparts, so a mistake there (such as using abar, Abar on the sides)
fails these comparisons while it passes every continuous-state limit.
"""
import math

import numpy as np
import pytest
from scipy.special import erfc, gamma as gamma_fn, roots_genlaguerre, roots_hermite, roots_legendre

GAM = 1.4
KDOF = (5 - 3 * GAM) / (GAM - 1)

_XH, _WH = roots_hermite(10)          # exact for degree <= 19 in each full-line component
_XL, _WL = roots_legendre(120)        # half line: 16 standard widths, smooth integrand
_XS, _WS = roots_genlaguerre(8, KDOF / 2 - 1)  # s = xi^2, Gamma(K/2) weight
_XT, _WT = roots_legendre(64)         # time nodes


def primitives(Q):
    rho = Q[0]
    U = Q[1:4] / rho
    p = (GAM - 1) * (Q[4] - 0.5 * rho * U @ U)
    return rho, U, rho / (2 * p)


def nodes(U, lam, half=0):
    """Quadrature nodes (u, v, w, s) and weights of g/rho for a Maxwellian (U, lam).

    half = 0: all velocities; +1: u > 0 only; -1: u < 0 only.  The weights of the
    full space sum to 1."""
    sig = 1.0 / math.sqrt(lam)
    if half == 0:
        u1 = U[0] + _XH * sig
        w1 = _WH / math.sqrt(math.pi)
    else:
        # Gaussian density of u on the half line, Gauss-Legendre on [0, U+16 sig] or [U-16 sig, 0]
        if half > 0:
            a, b = 0.0, max(U[0] + 16 * sig, 16 * sig)
        else:
            a, b = min(U[0] - 16 * sig, -16 * sig), 0.0
        u1 = 0.5 * (b - a) * _XL + 0.5 * (b + a)
        w1 = 0.5 * (b - a) * _WL * math.sqrt(lam / math.pi) * np.exp(-lam * (u1 - U[0]) ** 2)
    v1 = U[1] + _XH * sig
    w1v = _WH / math.sqrt(math.pi)
    x1 = U[2] + _XH * sig
    s1 = _XS / lam
    ws = _WS / gamma_fn(KDOF / 2)
    u, v, w, s = np.meshgrid(u1, v1, x1, s1, indexing="ij")
    W = np.einsum("i,j,k,l->ijkl", w1, w1v, w1v, ws)
    return dict(u=u.ravel(), v=v.ravel(), w=w.ravel(), s=s.ravel(), W=W.ravel())


def psi(nd):
    u, v, w, s = nd["u"], nd["v"], nd["w"], nd["s"]
    return np.stack([np.ones_like(u), u, v, w, 0.5 * (u * u + v * v + w * w + s)])


def lin(a, nd):
    """a . psi at the nodes (a = 5 coefficients)."""
    return a @ psi(nd)


def adotu(a3, nd):
    """a_1 u + a_2 v + a_3 w with a_i = a_i . psi (Eq. flux)."""
    return lin(a3[0], nd) * nd["u"] + lin(a3[1], nd) * nd["v"] + lin(a3[2], nd) * nd["w"]


def mom(nd, fvals):
    """5-vector sum of W psi f over the nodes."""
    return psi(nd) @ (nd["W"] * fvals)


def slopes(Q, dQ):
    """Side slopes a_i (3 x 5) and A (5) of Q with directional derivatives dQ (3 x 5)."""
    rho, U, lam = primitives(Q)
    nd = nodes(U, lam)
    P = psi(nd)
    M = (P * nd["W"]) @ P.T
    a = np.array([np.linalg.solve(M, dQ[i] / rho) for i in range(3)])
    A = np.linalg.solve(M, -mom(nd, adotu(a, nd)))
    return a, A


def face_flux_quadrature(QL, dQL, QR, dQR, mu, Pr, tau_eps, dt):
    """F, F_t of Eq. (flux) in the local frame (u = normal), by quadrature alone."""
    rl, Ul, laml = primitives(QL)
    rr, Ur, lamr = primitives(QR)
    al, Al = slopes(QL, dQL)
    ar, Ar = slopes(QR, dQR)
    ndl = nodes(Ul, laml, +1)
    ndr = nodes(Ur, lamr, -1)
    Q0 = rl * mom(ndl, 1.0) + rr * mom(ndr, 1.0)
    dQ0 = np.array([rl * mom(ndl, lin(al[i], ndl)) + rr * mom(ndr, lin(ar[i], ndr)) for i in range(3)])
    r0, U0, lam0 = primitives(Q0)
    ab, Ab = slopes(Q0, dQ0)
    nd0 = nodes(U0, lam0)
    p0 = r0 / (2 * lam0)
    tau = mu / p0 + tau_eps * dt

    # node-wise pieces of f (Eq. flux), split by their time coefficients
    g0_abu = adotu(ab, nd0)
    g0_Ab = lin(Ab, nd0)
    side = []
    for rk, nd, a, A in ((rl, ndl, al, Al), (rr, ndr, ar, Ar)):
        side.append((rk, nd, adotu(a, nd), lin(A, nd)))

    def weights(nd, rk):
        return rk * nd["W"]

    def integrand(t):
        """(flux 5-vector, heat flux) of f at time t."""
        if tau > 0:
            E = math.exp(-t / tau)
            c0, c1, c2 = 1 - E, (t + tau) * E - tau, t - tau + tau * E
        else:
            E, c0, c1, c2 = 0.0, 1.0, 0.0, t
        out = np.zeros(5)
        heat = 0.0
        f0 = c0 + c1 * g0_abu + c2 * g0_Ab
        parts = [(nd0, r0, f0)]
        for rk, nd, au, Ak in side:
            parts.append((nd, rk, E * (1 - (tau + t) * au - tau * Ak)))
        for nd, rk, f in parts:
            wf = weights(nd, rk) * f
            out += psi(nd) @ (nd["u"] * wf)
            cu, cv, cw = nd["u"] - U0[0], nd["v"] - U0[1], nd["w"] - U0[2]
            heat += np.sum(0.5 * cu * (cu * cu + cv * cv + cw * cw + nd["s"]) * wf)
        return out, heat

    def time_integral(delta):
        tt = 0.5 * delta * (_XT + 1)
        I, H = np.zeros(5), 0.0
        for t, wt in zip(tt, 0.5 * delta * _WT):
            f, h = integrand(t)
            I += wt * f
            H += wt * h
        return I, H

    I1, H1 = time_integral(dt)
    Ih, Hh = time_integral(0.5 * dt)
    # F dt + F_t dt^2/2 = I(dt), F dt/2 + F_t dt^2/8 = I(dt/2)  (Eq. expansion-1)
    S = np.array([[dt, dt * dt / 2], [dt / 2, dt * dt / 8]])
    sol = np.linalg.solve(S, np.stack([I1, Ih]))
    F, Ft = sol[0], sol[1]
    if Pr != 1.0:
        q, _ = np.linalg.solve(S, [H1, Hh])
        F[4] += (1 / Pr - 1) * q
    return F, Ft


def cons(rho, u, p):
    u = np.asarray(u, dtype=float)
    return np.array([rho, rho * u[0], rho * u[1], rho * u[2], p / (GAM - 1) + 0.5 * rho * u @ u])


def jump_states(seed, vel=1.0):
    """Independent left/right states with independent gradients (a discontinuity)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(2):
        rho, p = rng.uniform(0.6, 1.8), rng.uniform(0.5, 2.5)
        Q = cons(rho, rng.uniform(-vel, vel, 3), p)
        dQ = 0.3 * rng.standard_normal((3, 5)) * np.abs(Q)
        out += [Q, dQ]
    return out


def test_quadrature_reproduces_half_space_closed_form():
    # the half-line rule itself: <1>_+ = erfc(-sqrt(lam) U)/2, <u>_+ = U <1>_+ + e^{-lam U^2}/(2 sqrt(pi lam))
    for U, lam in ((0.3, 0.7), (-1.2, 2.0), (2.5, 0.4)):
        nd = nodes(np.array([U, 0.1, -0.2]), lam, +1)
        m0 = 0.5 * erfc(-math.sqrt(lam) * U)
        m1 = U * m0 + math.exp(-lam * U * U) / (2 * math.sqrt(math.pi * lam))
        assert abs(math.fsum(nd["W"]) - m0) < 1e-13
        assert abs(math.fsum(nd["W"] * nd["u"]) - m1) < 1e-13
        full = nodes(np.array([U, 0.1, -0.2]), lam)
        # <xi^2> = K/(2 lam), <(u-U)^2> = 1/(2 lam)
        assert abs(full["W"] @ full["s"] - KDOF / (2 * lam)) < 1e-13
        assert abs(full["W"] @ (full["u"] - U) ** 2 - 1 / (2 * lam)) < 1e-13


CASES = [
    # (mu, Pr, tau_eps, dt): tau ~ dt, tau << dt, tau = 0, tau from tau_eps only, Pr != 1
    (2e-3, 1.0, 0.0, 1e-3),
    (1e-4, 1.0, 0.0, 5e-3),
    (0.0, 1.0, 0.0, 1e-3),
    (0.0, 1.0, 0.5, 2e-3),
    (2e-3, 0.72, 0.0, 1e-3),
    (1e-3, 0.72, 0.3, 2e-3),
]


def _local(d, QL, dQL, QR, dQR):
    """Global inputs of a face normal to axis d in the oracle's local frame (d, d+1, d+2)."""
    ax = [d, (d + 1) % 3, (d + 2) % 3]
    P = np.eye(5)[[0, 1 + ax[0], 1 + ax[1], 1 + ax[2], 4]]
    return P, [P @ QL, (P @ dQL[ax].T).T, P @ QR, (P @ dQR[ax].T).T]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("seed", range(3))
def test_face_flux_matches_velocity_time_quadrature(orc, seed, case):
    mu, Pr, tau_eps, dt = CASES[case]
    QL, dQL, QR, dQR = jump_states(1000 + seed)
    d = seed % 3
    P, loc = _local(d, QL, dQL, QR, dQR)
    Fq, Ftq = face_flux_quadrature(*loc, mu, Pr, tau_eps, dt)
    F, Ft = orc.face_flux(d, QL, dQL, QR, dQR, mu=mu, Pr=Pr, tau_eps=tau_eps, dt=dt)
    F, Ft = P @ F, P @ Ft  # back to the local frame
    sF, sFt = np.abs(Fq).max(), np.abs(Ftq).max()
    assert np.all(np.abs(F - Fq) <= 1e-11 * sF), (F - Fq) / sF
    assert np.all(np.abs(Ft - Ftq) <= 1e-11 * sFt), (Ft - Ftq) / sFt


def test_side_slopes_matter_at_a_discontinuity(orc):
    """The pin is sensitive to the side terms: swapping the sides' slopes moves F well above tolerance."""
    QL, dQL, QR, dQR = jump_states(1000)
    mu, Pr, tau_eps, dt = CASES[0]
    F1, Ft1 = face_flux_quadrature(QL, dQL, QR, dQR, mu, Pr, tau_eps, dt)
    F2, Ft2 = face_flux_quadrature(QL, dQR, QR, dQL, mu, Pr, tau_eps, dt)
    assert np.abs(F1 - F2).max() > 1e-6 * np.abs(F1).max()
    assert np.abs(Ft1 - Ft2).max() > 1e-4 * np.abs(Ft1).max()
