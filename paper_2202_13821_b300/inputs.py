"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds no arithmetic of the DG-HGKS method: it samples the
problems' initial conditions (Sec. 5.1 density advection, Sec. 5.3
Taylor-Green vortex) at cell centres, adds their analytic first derivatives
as the linear modal coefficients, and adds seeded random perturbations to
every modal coefficient.  The CUDA library and the oracle both consume what
it returns; neither is imported here.

Layout: ``Q[var][mode][z][y][x]`` float64 with var = (rho, rho U, rho V,
rho W, rho E); mode 0 is the cell mean, modes 1..3 the linear modes in x, y,
z (coefficients of the Legendre polynomial P_1 of each reference coordinate),
then the higher modes of P_k by total degree.
"""
from __future__ import annotations

import numpy as np

SEED = 2202_13821


def n_modes(order: int) -> int:
    return (order + 1) * (order + 2) * (order + 3) // 6


def _centres(n, lo, hi):
    h = [(hi[d] - lo[d]) / n[d] for d in range(3)]
    x = lo[0] + (np.arange(n[0]) + 0.5) * h[0]
    y = lo[1] + (np.arange(n[1]) + 0.5) * h[1]
    z = lo[2] + (np.arange(n[2]) + 0.5) * h[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return (X, Y, Z), h


def _cons_from_prim(rho, U, V, W, p, gamma):
    return np.stack([rho, rho * U, rho * V, rho * W, p / (gamma - 1.0) + 0.5 * rho * (U * U + V * V + W * W)])


def advection_prim(x, y, z, amp=0.2):
    """Sec. 5.1, 3D case: rho = 1 + amp sin(pi(x+y+z)), U=V=W=1, p=1."""
    rho = 1.0 + amp * np.sin(np.pi * (x + y + z))
    one = np.ones_like(rho)
    return rho, one, one, one, one


def tgv_prim(x, y, z, V0=1.0, rho0=1.0, p0=None, Ma=0.1, gamma=1.4, isothermal=False):
    """Sec. 5.3 Taylor-Green vortex on [-pi, pi]^3 with L = 1."""
    if p0 is None:
        p0 = rho0 * V0 * V0 / (gamma * Ma * Ma)
    U = V0 * np.sin(x) * np.cos(y) * np.cos(z)
    V = -V0 * np.cos(x) * np.sin(y) * np.cos(z)
    W = np.zeros_like(U)
    p = p0 + rho0 * V0 * V0 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    rho = rho0 * p / p0 if isothermal else np.full_like(U, rho0)
    return rho, U, V, W, p


def modal_state(prim_fn, n, order, lo, hi, gamma=1.4, perturb=0.0, seed=SEED, **kw) -> np.ndarray:
    """Cell-centre sample + analytic-gradient linear modes + seeded perturbation.

    The linear coefficient of P_1(xi_d) is (h_d / 2) dq/dx_d at the centre
    (the first-order Taylor term), with dq/dx_d taken by central differences
    of the initial condition over h_d / 1000.  ``perturb`` scales a standard
    normal perturbation added to every coefficient, relative to the largest
    |cell mean| of each variable.
    """
    n = (int(n),) * 3 if np.isscalar(n) else tuple(int(v) for v in n)
    (X, Y, Z), h = _centres(n, lo, hi)
    nm = n_modes(order)
    Q = np.zeros((5, nm, n[2], n[1], n[0]))
    Q[:, 0] = _cons_from_prim(*prim_fn(X, Y, Z, **kw), gamma)
    if order >= 1:
        for d, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            e = h[d] * 1e-3
            qp = _cons_from_prim(*prim_fn(X + dx * e, Y + dy * e, Z + dz * e, **kw), gamma)
            qm = _cons_from_prim(*prim_fn(X - dx * e, Y - dy * e, Z - dz * e, **kw), gamma)
            Q[:, 1 + d] = (qp - qm) / (2 * e) * (h[d] / 2.0)
    if perturb:
        rng = np.random.Generator(np.random.PCG64(seed))
        scale = np.abs(Q[:, 0]).reshape(5, -1).max(axis=1)
        Q += perturb * scale[:, None, None, None, None] * rng.standard_normal(Q.shape)
    return Q


def advection_state(n, order, perturb=0.0, seed=SEED, gamma=1.4, amp=0.2):
    return modal_state(advection_prim, n, order, (0.0,) * 3, (2.0,) * 3, gamma, perturb, seed, amp=amp)


def tgv_state(n, order, perturb=0.0, seed=SEED, gamma=1.4, Ma=0.1, isothermal=False):
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3

    def prim(x, y, z):
        return tgv_prim(x, y, z, Ma=Ma, gamma=gamma, isothermal=isothermal)

    return modal_state(prim, n, order, lo, hi, gamma, perturb, seed)


def random_state(n, order, seed=SEED, rho=(0.5, 2.0), vel=1.0, p=(0.5, 3.0), modes_rel=0.02, gamma=1.4):
    """Non-smooth random state: every cell mean drawn independently.

    Densities and pressures are uniform in the given ranges, velocities
    uniform in [-vel, vel]; higher modes are normal with standard deviation
    ``modes_rel`` times the cell mean of each variable.  Used to exercise the
    interface flux with large jumps between neighbouring cells.
    """
    n = tuple(int(v) for v in n)
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n[2], n[1], n[0])
    r = rng.uniform(*rho, shape)
    U, V, W = (rng.uniform(-vel, vel, shape) for _ in range(3))
    pr = rng.uniform(*p, shape)
    Q = np.zeros((5, n_modes(order)) + shape)
    Q[:, 0] = _cons_from_prim(r, U, V, W, pr, gamma)
    if order >= 1:
        Q[:, 1:] = modes_rel * np.abs(Q[:, :1]) * rng.standard_normal(Q[:, 1:].shape)
    return Q


def tgv_dt(n, order, cfl=0.15, gamma=1.4, Ma=0.1, V0=1.0):
    """dt = CFL min(h) / max(|U| + c) from the Taylor-Green initial field at cell centres."""
    (X, Y, Z), h = _centres((n, n, n), (-np.pi,) * 3, (np.pi,) * 3)
    rho, U, V, W, p = tgv_prim(X, Y, Z, V0=V0, Ma=Ma, gamma=gamma)
    c = np.sqrt(gamma * p / rho)
    return cfl * min(h) / float(np.max(np.sqrt(U * U + V * V + W * W) + c))
