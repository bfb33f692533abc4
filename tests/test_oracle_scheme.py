"""Scheme-level pins of the oracle (Sec. 3 Eqs. operator/two-stage, Sec. 5.1, Sec. 5.3).

* uniform flow is preserved: R = R_t = 0 to rounding;
* conservation: sum over cells of |K| L_(v, mode 0) = 0 on a periodic box;
* the S2O4 combination applied to dq/dt = lam q equals the degree-4 Taylor
  polynomial of exp(lam dt) (Eq. two-stage is fourth-order);
* optimal order k+1 on the 3D density advection against its exact solution,
  with rho = 1 + 0.2 sin(pi(x+y+z-3t)) (U = V = W = 1; the printed "-t" is
  inconsistent with the unit velocities, and the test shows the scheme does
  not approach it), from 8^3 to 16^3 cells; with the paper's Gauss rule
  (n_q = k) the measured L2 order matches the finest order the paper prints
  (Sec. 5.1, Tables tab-3d-1/2, held in tests/golden/advection_orders.txt);
* Taylor-Green vortex: E_k(0) = 1/8 for rho = 1 (closed form of the initial
  field), and dE_k/dt < 0.
"""
import math
import os

import numpy as np
import pytest

from paper_2202_13821_b300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def uniform_state(pb, rho=1.2, u=(0.3, -0.2, 0.5), p=1.1, gamma=1.4):
    Q = np.zeros(pb.shape)
    Q[0, 0] = rho
    for d in range(3):
        Q[1 + d, 0] = rho * u[d]
    Q[4, 0] = p / (gamma - 1) + 0.5 * rho * sum(x * x for x in u)
    return Q


@pytest.mark.parametrize("order,nq,mu", [(1, 2, 0.0), (2, 3, 1e-3), (2, 2, 0.0), (3, 4, 1e-3)])
def test_uniform_flow_preserved(orc, order, nq, mu):
    pb = orc.Problem(order=order, nq=nq, n=(3, 4, 5), mu=mu, Pr=0.72, tau_eps=0.01)
    L, Lt = orc.residual(pb, uniform_state(pb), 1e-2)
    assert np.abs(L).max() < 1e-12
    assert np.abs(Lt).max() < 1e-11


@pytest.mark.parametrize("order,nq,mu,Pr", [(1, 2, 0.0, 1.0), (2, 3, 5e-3, 0.72), (3, 3, 1e-3, 1.0)])
def test_conservation_periodic(orc, order, nq, mu, Pr):
    pb = orc.Problem(order=order, nq=nq, n=(4, 3, 5), mu=mu, Pr=Pr, tau_eps=0.01)
    Q = inputs.random_state(pb.n, order, seed=11)
    L, Lt = orc.residual(pb, Q, 1e-2)
    vol = np.prod([(pb.hi[d] - pb.lo[d]) / pb.n[d] for d in range(3)])
    for A in (L, Lt):
        tot = A[:, 0].sum(axis=(1, 2, 3)) * vol
        scale = np.abs(A[:, 0]).sum(axis=(1, 2, 3)) * vol
        assert np.all(np.abs(tot) <= 1e-13 * scale)
    # and through a full S2O4 step the totals are unchanged
    Q1 = orc.step(pb, Q, 1e-3)
    np.testing.assert_allclose(orc.totals(pb, Q1), orc.totals(pb, Q), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("lam", [-1.0, 0.7, -3.0])
@pytest.mark.parametrize("dt", [0.1, 0.03])
def test_s2o4_scalar_is_fourth_order_taylor(orc, lam, dt):
    z = lam * dt
    want = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    assert abs(orc.s2o4_scalar(lam, 1.0, dt) - want) < 1e-15


def _advection_state(orc, order, n, T=0.1, nq=None):
    h = 2.0 / n
    dt0 = 0.1 * h / (math.sqrt(3) + math.sqrt(1.4 / 0.8))  # CFL 0.1 with max(|U| + c)
    ns = math.ceil(T / dt0)
    pb = orc.Problem(order=order, nq=order + 1 if nq is None else nq, n=(n, n, n), tau_eps=0.01)
    Q = orc.project(pb, orc.IC_ADVECTION, (0.2, 0.0))
    return pb, orc.step(pb, Q, T / ns, ns)


def _advection_error(orc, order, n, T=0.1, nq=None):
    pb, Q = _advection_state(orc, order, n, T, nq)
    return orc.density_errors(pb, Q, orc.IC_ADVECTION, (0.2, T))


@pytest.mark.slow
@pytest.mark.parametrize("order,n0,min_order", [(1, 8, 1.9), (2, 8, 2.9)])
def test_advection_convergence_order(orc, order, n0, min_order):
    # measured (L1, L2) orders from 8^3 to 16^3: P1 2.06, 1.97; P2 (n_q = 3) 3.06, 2.98
    T = 0.1
    e0 = _advection_error(orc, order, n0, T)
    pb, Q1 = _advection_state(orc, order, 2 * n0, T)
    e1 = orc.density_errors(pb, Q1, orc.IC_ADVECTION, (0.2, T))
    orders = np.log2(e0 / e1)
    assert orders[0] > min_order and orders[1] > min_order, orders
    # the printed exact solution with "-t" is not approached
    bad = orc.density_errors(pb, Q1, orc.IC_ADVECTION, (0.2, T / 3))
    assert bad[1] > 20 * e1[1]


def golden_orders(name):
    """Rows (order k, expected order, finest L2 order the paper prints) of a golden fixture."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", name)) if l[0] != "#"]
    return [(int(k), int(e), float(f)) for k, e, f in rows]


@pytest.mark.slow
@pytest.mark.parametrize("row", golden_orders("advection_orders.txt"), ids=lambda r: f"P{r[0]}")
def test_advection_order_matches_paper_table(orc, row):
    """With the paper's Gauss rule (n_q = k, Sec. 3 Remark 2) the L2 order from 8^3 to 16^3 is the
    expected k+1 and agrees with the finest order of the paper's tables (measured: P2 3.04 against
    3.0821, P3 3.99 against 3.9962); the error values themselves depend on the unprinted final time
    and time step and are not compared."""
    k, expected, finest = row
    e0 = _advection_error(orc, k, 8, nq=k)
    e1 = _advection_error(orc, k, 16, nq=k)
    l2_order = math.log2(e0[1] / e1[1])
    assert l2_order > expected - 0.1, l2_order
    assert abs(l2_order - finest) < 0.15, (l2_order, finest)


def vortex_errors(orc, order, n, T=1.0, cfl=0.1):
    """Isotropic vortex of Sec. 5.1 as a 3-D problem with one cell along z; errors at time T.
    The vortex centre is the centre (5, 5) of the [0, 10]^2 domain (the paper's r is measured
    from it); the exact solution is the initial vortex moved by T (1, 1)."""
    h = 10.0 / n
    dt0 = cfl * h / (math.sqrt(2) + 1.0 + math.sqrt(1.4))
    ns = math.ceil(T / dt0)
    pb = orc.Problem(order=order, nq=order + 1, n=(n, n, 1), lo=(0.0, 0.0, 0.0), hi=(10.0, 10.0, h))
    Q = orc.project(pb, orc.IC_VORTEX, (5.0, 0.0, 5.0, 5.0, 10.0, 10.0))
    Q = orc.step(pb, Q, T / ns, ns)
    return orc.density_errors(pb, Q, orc.IC_VORTEX, (5.0, T, 5.0, 5.0, 10.0, 10.0))


@pytest.mark.slow
def test_isotropic_vortex_p1_order(orc):
    e0, e1 = vortex_errors(orc, 1, 20), vortex_errors(orc, 1, 40)
    orders = np.log2(e0 / e1)
    assert orders[1] > 1.7, orders  # L2 order ~ k+1 = 2


def test_tgv_initial_enstrophy_dissipation(orc):
    """omega of the initial field is (-cos x sin y sin z, -sin x cos y sin z, 2 sin x sin y cos z),
    whose mean square is 3/4, so eps(zeta) = 2 mu (1/2)(3/4) = 0.75 mu at rho = 1 (Sec. 5.3)."""
    mu = 1 / 1600
    errs = []
    for n in (8, 16):
        pb = orc.Problem(order=2, nq=3, n=(n,) * 3, lo=(-math.pi,) * 3, hi=(math.pi,) * 3, mu=mu)
        Q = orc.project(pb, orc.IC_TGV, (1.0, 1.0, 1.0 / (1.4 * 0.01), 0.0))
        errs.append(abs(orc.enstrophy_dissipation(pb, Q) - 0.75 * mu) / (0.75 * mu))
    # the gradient of the P2 projection converges at second order: 1.1e-2 at 8^3, 4.5e-3 at 16^3
    assert errs[1] < 6e-3 and errs[1] < errs[0] / 2


def test_tgv_initial_kinetic_energy(orc):
    pb = orc.Problem(order=2, nq=3, n=(8, 8, 8), lo=(-math.pi,) * 3, hi=(math.pi,) * 3, mu=1 / 1600, Pr=1.0)
    p0 = 1.0 / (1.4 * 0.01)
    Q = orc.project(pb, orc.IC_TGV, (1.0, 1.0, p0, 0.0))
    Ek = orc.kinetic_energy(pb, Q)
    assert abs(Ek - 0.125) < 2e-3  # closed form 1/8, up to the P2 projection / quadrature error at 8^3
    dt = inputs.tgv_dt(8, 2)
    Q1 = orc.step(pb, Q, dt, 2)
    assert orc.kinetic_energy(pb, Q1) < Ek
