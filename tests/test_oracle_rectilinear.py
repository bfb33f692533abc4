"""Pins of the oracle on rectilinear (non-uniform) meshes (Sec. 5.1, mapped grids).

A cell K_ijk = [x_{i-1/2}, x_{i+1/2}] x [y_{j-1/2}, y_{j+1/2}] x [z_{k-1/2}, z_{k+1/2}]
keeps the reference map of Sec. 3 with its own widths: gradients scale by
2/h_d of the cell whose polynomial is evaluated, faces by the product of the
two tangential widths, the mass matrix by the cell volume.

* nodes placed at the uniform positions reproduce the uniform residual;
* mirror symmetry: reflecting the mesh, the state and the x-momentum along an
  axis reflects the residual (fails if a face takes the gradient scale or the
  area of the wrong side);
* conservation: sum over cells of |K| L_(v, mode 0) = 0; uniform flow is kept;
* Navier-Stokes limit: on the mapped mesh x = xi + 0.05 sin(pi xi), the
  residual of a transverse shear wave u = eps sin(k y) converges to the
  viscous decay mu u'' (cell averages), at high order;
* slow: the k+1 convergence of the 3D density advection on the mapped mesh
  (Tables tab-3d-3 and tab-3d-4).
"""
import math
import os

import numpy as np
import pytest

from paper_2202_13821_b300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def _scale_close(a, b, rtol):
    s = max(np.abs(a).max(), np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() <= rtol * s


@pytest.mark.parametrize("order,nq", [(1, 2), (2, 3)])
def test_uniform_nodes_match_uniform_mesh(orc, order, nq):
    n = (5, 4, 3)
    Q = inputs.random_state(n, order, seed=5)
    u = orc.Problem(order=order, nq=nq, n=n, lo=(0.0, -1.0, 0.5), hi=(2.0, 1.0, 2.0), mu=3e-3, Pr=0.72,
                    tau_eps=0.01)
    nodes = tuple(np.linspace(u.lo[d], u.hi[d], n[d] + 1) for d in range(3))
    r = orc.Problem(order=order, nq=nq, n=n, mu=3e-3, Pr=0.72, tau_eps=0.01, nodes=nodes)
    Lu, Ltu = orc.residual(u, Q, 1e-2)
    Lr, Ltr = orc.residual(r, Q, 1e-2)
    assert _scale_close(Lu, Lr, 1e-13) and _scale_close(Ltu, Ltr, 1e-13)


def _mirror(Q, axis, nm_exps):
    """Reflect x_axis -> -x_axis: reverse the cells, flip odd modes along the axis and the momentum component."""
    ax = 4 - axis  # array axes: (var, mode, z, y, x)
    R = np.flip(Q, axis=ax).copy()
    for m, e in enumerate(nm_exps):
        if e[axis] % 2 == 1:
            R[:, m] *= -1.0
    R[1 + axis] *= -1.0
    return R


def _exps(orc, order):
    # mode exponents in the oracle's order, recovered from its basis at a point
    # where the monomials are distinguishable: B_m(r) = P_a(r0) P_b(r1) P_c(r2)
    from itertools import product

    k = order
    cands = [e for e in product(range(k + 1), repeat=3) if sum(e) <= k]
    r = np.array([0.31, -0.57, 0.73])
    vals, _ = orc.basis(order, r)
    leg = [np.polynomial.legendre.Legendre.basis(i) for i in range(k + 1)]
    out = []
    for v in vals:
        match = [e for e in cands if abs(leg[e[0]](r[0]) * leg[e[1]](r[1]) * leg[e[2]](r[2]) - v) < 1e-12]
        assert len(match) == 1
        out.append(match[0])
    return out


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry_on_random_nodes(orc, axis):
    order, n = 2, (5, 4, 6)
    nodes = [inputs.random_nodes(n[d], 0.0, 2.0, spread=0.4, seed=20 + d) for d in range(3)]
    pb = orc.Problem(order=order, nq=3, n=n, mu=5e-3, Pr=0.72, tau_eps=0.01, nodes=tuple(nodes))
    mn = list(nodes)
    mn[axis] = 2.0 - nodes[axis][::-1]
    pm = orc.Problem(order=order, nq=3, n=n, mu=5e-3, Pr=0.72, tau_eps=0.01, nodes=tuple(mn))
    ex = _exps(orc, order)
    Q = inputs.random_state(n, order, seed=9)
    L, Lt = orc.residual(pb, Q, 1e-2)
    Lm, Ltm = orc.residual(pm, _mirror(Q, axis, ex), 1e-2)
    assert _scale_close(Lm, _mirror(L, axis, ex), 1e-12)
    assert _scale_close(Ltm, _mirror(Lt, axis, ex), 1e-12)


def test_conservation_and_uniform_flow_on_random_nodes(orc):
    order, n = 2, (4, 5, 3)
    nodes = tuple(inputs.random_nodes(n[d], 0.0, 1.0, spread=0.4, seed=30 + d) for d in range(3))
    pb = orc.Problem(order=order, nq=3, n=n, mu=5e-3, Pr=0.72, tau_eps=0.01, nodes=nodes)
    Q = inputs.random_state(n, order, seed=12)
    L, Lt = orc.residual(pb, Q, 1e-2)
    w = [np.diff(x) for x in nodes]
    vol = w[2][:, None, None] * w[1][None, :, None] * w[0][None, None, :]
    for A in (L, Lt):
        tot = (A[:, 0] * vol).sum(axis=(1, 2, 3))
        scale = (np.abs(A[:, 0]) * vol).sum(axis=(1, 2, 3))
        assert np.all(np.abs(tot) <= 1e-13 * scale)
    Q1 = orc.step(pb, Q, 1e-3)
    np.testing.assert_allclose(orc.totals(pb, Q1), orc.totals(pb, Q), rtol=1e-14, atol=1e-14)
    # the totals are the volume-weighted cell means
    np.testing.assert_allclose(orc.totals(pb, Q), (Q[:, 0] * vol).sum(axis=(1, 2, 3)), rtol=1e-14)
    U = np.zeros(pb.shape)
    U[0, 0], U[1, 0], U[2, 0], U[3, 0], U[4, 0] = 1.2, 0.36, -0.24, 0.6, 1.1 / 0.4 + 0.5 * 1.2 * 0.7
    L, Lt = orc.residual(pb, U, 1e-2)
    assert np.abs(L).max() < 1e-12 and np.abs(Lt).max() < 1e-11


def _shear_error(orc, order, n, axis, mu=1e-2, eps=1e-2):
    nn = [3, 3, 3]
    nn[axis] = n
    nodes = [None, None, None]
    nodes[axis] = inputs.mapped_nodes(n)
    pb = orc.Problem(order=order, nq=order + 1, n=tuple(nn), lo=(0.0,) * 3, hi=(2.0,) * 3, mu=mu, Pr=1.0,
                     nodes=tuple(nodes))
    Q = orc.project(pb, orc.IC_SHEAR, (eps, axis, 0.0, 2.0, 1.0, 1.0))
    L, _ = orc.residual(pb, Q, 1e-4)
    x, k = nodes[axis], math.pi  # wavelength 2
    exact = -mu * eps * k * k * (np.cos(k * x[:-1]) - np.cos(k * x[1:])) / (k * np.diff(x))  # cell means of mu u''
    c = (axis + 1) % 3
    got = np.moveaxis(L[1 + c, 0], 2 - axis, -1).reshape(-1, n)
    err = np.abs(got - exact[None, :]).max() / np.abs(exact).max()
    return err, np.abs(L[0, 0]).max()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_shear_wave_viscous_decay_on_mapped_mesh(orc, axis):
    """mu u'' from the gas-kinetic flux (Navier-Stokes limit, Sec. 2) on x = xi + 0.05 sin(pi xi)."""
    e8, drho = _shear_error(orc, 2, 8, axis)
    e16, _ = _shear_error(orc, 2, 16, axis)
    assert e16 < 1e-2, e16
    assert e8 / e16 > 8, (e8, e16)  # P2: better than third order in the cell means
    assert drho < 1e-5  # no mass flux across the shear layers
    e3, _ = _shear_error(orc, 3, 8, axis)
    assert e3 < 5e-3, e3


def _advection_error_mapped(orc, order, n, T=0.1, nq=None):
    nodes = tuple(inputs.mapped_nodes(n) for _ in range(3))
    hmin = min(np.diff(nodes[0]))
    dt0 = 0.1 * hmin / (math.sqrt(3) + math.sqrt(1.4 / 0.8))
    ns = math.ceil(T / dt0)
    pb = orc.Problem(order=order, nq=order + 1 if nq is None else nq, n=(n, n, n), tau_eps=0.01, nodes=nodes)
    Q = orc.project(pb, orc.IC_ADVECTION, (0.2, 0.0))
    Q = orc.step(pb, Q, T / ns, ns)
    return orc.density_errors(pb, Q, orc.IC_ADVECTION, (0.2, T))


@pytest.mark.slow
@pytest.mark.parametrize("order,n0,min_order", [(1, 8, 1.8), (2, 4, 2.5)])
def test_advection_convergence_on_mapped_mesh(orc, order, n0, min_order):
    e0 = _advection_error_mapped(orc, order, n0)
    e1 = _advection_error_mapped(orc, order, 2 * n0)
    orders = np.log2(e0 / e1)
    assert orders[0] > min_order and orders[1] > min_order, orders


@pytest.mark.slow
def test_mapped_mesh_order_matches_paper_table(orc):
    """P2 with the paper's Gauss rule (n_q = k) on the mapped mesh: the L2 order from 8^3 to 16^3
    is the expected 3 and agrees with the finest order of the paper's table for this mesh (Sec. 5.1,
    Table tab-3d-3, held in tests/golden/advection_orders_nonuniform.txt; measured 3.03 against
    3.0864).  The P3 row (measured 3.97 against 4.0015) is left out to keep the CPU suite short;
    the uniform-mesh test covers P3."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "advection_orders_nonuniform.txt")) if l[0] != "#"]
    k, expected, finest = next((int(a), int(b), float(c)) for a, b, c in rows if a == "2")
    e0 = _advection_error_mapped(orc, k, 8, nq=k)
    e1 = _advection_error_mapped(orc, k, 16, nq=k)
    l2_order = math.log2(e0[1] / e1[1])
    assert l2_order > expected - 0.1, l2_order
    assert abs(l2_order - finest) < 0.15, (l2_order, finest)
