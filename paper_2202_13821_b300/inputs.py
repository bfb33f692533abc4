"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds no arithmetic of the DG-HGKS method: it samples the
problems' initial conditions (Sec. 5.1 density advection, Sec. 5.3
Taylor-Green vortex) at cell centres, adds their first derivatives as the
linear modal coefficients, and adds seeded random perturbations to every
modal coefficient.  The CUDA library and the oracle both consume what it
returns; neither is imported here.

Layout: ``Q[var][mode][z][y][x]`` float64 with var = (rho, rho U, rho V,
rho W, rho E); mode 0 is the cell mean, modes 1..3 the linear modes in x, y,
z (coefficients of the Legendre polynomial P_1 of each reference coordinate),
then the higher modes of P_k by total degree.

Every generator works with numpy (host arrays, the default) or with torch
(``device=...``: the state is built directly in device memory, which the
256^3 benchmark state needs: 6.7 GB).
"""
from __future__ import annotations

import math

import numpy as np

SEED = 2202_13821


def n_modes(order: int) -> int:
    return (order + 1) * (order + 2) * (order + 3) // 6


class _NP:
    sin, cos = staticmethod(np.sin), staticmethod(np.cos)

    @staticmethod
    def stack_broadcast(q):
        return np.stack(np.broadcast_arrays(*[np.asarray(v, dtype=np.float64) for v in q]))

    @staticmethod
    def zeros(shape):
        return np.zeros(shape)

    @staticmethod
    def arange(n):
        return np.arange(n, dtype=np.float64)


class _TH:
    def __init__(self, device):
        import torch

        self.t = torch
        self.device = device

    def sin(self, x):
        return self.t.sin(x) if hasattr(x, "dim") else np.sin(x)

    def cos(self, x):
        return self.t.cos(x) if hasattr(x, "dim") else np.cos(x)

    def stack_broadcast(self, q):
        t = self.t
        q = [v if hasattr(v, "dim") else t.tensor(float(v), dtype=t.float64, device=self.device) for v in q]
        return t.stack(t.broadcast_tensors(*q))

    def zeros(self, shape):
        return self.t.zeros(shape, dtype=self.t.float64, device=self.device)

    def arange(self, n):
        return self.t.arange(n, dtype=self.t.float64, device=self.device)


def _xp(device):
    return _NP if device is None else _TH(device)


def mapped_nodes(n, lo=0.0, hi=2.0, amp=0.05):
    """Node coordinates x_q = xi_q + amp sin(pi xi_q) of the non-uniform mesh of
    Sec. 5.1 (xi_q uniform on [lo, hi]; on [0, 2] the end nodes stay fixed)."""
    xi = lo + (hi - lo) * np.arange(n + 1) / n
    return xi + amp * np.sin(np.pi * xi)


def random_nodes(n, lo=0.0, hi=2.0, spread=0.3, seed=SEED):
    """n + 1 increasing nodes on [lo, hi] whose cell widths are the mean width
    times independent uniform factors in [1 - spread, 1 + spread] (renormalised)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = 1.0 + spread * rng.uniform(-1.0, 1.0, n)
    x = np.concatenate([[0.0], np.cumsum(w)])
    x = lo + (hi - lo) * x / x[-1]
    x[-1] = hi
    return x


def _centres(xp, n, lo, hi, nodes=None):
    cen, h = [], []
    for d in range(3):
        nd = None if nodes is None else nodes[d]
        if nd is None:
            hd = (hi[d] - lo[d]) / n[d]
            cen.append(lo[d] + (xp.arange(n[d]) + 0.5) * hd)
            h.append(hd)
        else:
            nd = np.asarray(nd, dtype=np.float64)
            c, w = 0.5 * (nd[1:] + nd[:-1]), nd[1:] - nd[:-1]
            if xp is not _NP:
                c, w = (xp.t.from_numpy(np.ascontiguousarray(v)).to(xp.device) for v in (c, w))
            cen.append(c)
            h.append(w)
    # broadcastable axes: X varies along the last (x) axis, Z along the first
    shp = ((None, None, slice(None)), (None, slice(None), None), (slice(None), None, None))
    h = [v if np.isscalar(v) else v[shp[d]] for d, v in enumerate(h)]
    return tuple(cen[d][shp[d]] for d in range(3)), h


def _cons_from_prim(xp, rho, U, V, W, p, gamma):
    q = (rho, rho * U, rho * V, rho * W, p / (gamma - 1.0) + 0.5 * rho * (U * U + V * V + W * W))
    return xp.stack_broadcast(q)


def advection_prim(xp, x, y, z, amp=0.2):
    """Sec. 5.1, 3D case: rho = 1 + amp sin(pi(x+y+z)), U=V=W=1, p=1."""
    rho = 1.0 + amp * xp.sin(np.pi * (x + y + z))
    return rho, 1.0, 1.0, 1.0, 1.0


def tgv_prim(xp, x, y, z, V0=1.0, rho0=1.0, p0=None, Ma=0.1, gamma=1.4, isothermal=False):
    """Sec. 5.3 Taylor-Green vortex on [-pi, pi]^3 with L = 1."""
    if p0 is None:
        p0 = rho0 * V0 * V0 / (gamma * Ma * Ma)
    U = V0 * xp.sin(x) * xp.cos(y) * xp.cos(z)
    V = -V0 * xp.cos(x) * xp.sin(y) * xp.cos(z)
    p = p0 + rho0 * V0 * V0 / 16.0 * (xp.cos(2 * x) + xp.cos(2 * y)) * (xp.cos(2 * z) + 2.0)
    rho = rho0 * p / p0 if isothermal else rho0
    return rho, U, V, 0.0, p


def modal_state(prim_fn, n, order, lo, hi, gamma=1.4, perturb=0.0, seed=SEED, device=None, prim_kw=None,
                nodes=None):
    """Cell-centre sample + first-derivative linear modes + seeded perturbation.

    The linear coefficient of P_1(xi_d) is (h_d / 2) dq/dx_d at the centre
    (the first-order Taylor term), with dq/dx_d taken by central differences
    of the initial condition over h_d / 1000.  ``perturb`` scales a standard
    normal perturbation (numpy PCG64 stream ``seed``) added to every
    coefficient, relative to the largest |cell mean| of each variable.
    ``nodes``: optional per-axis node coordinates of a rectilinear mesh
    (then h_d is each cell's width).
    """
    xp = _xp(device)
    kw = prim_kw or {}
    n = (int(n),) * 3 if np.isscalar(n) else tuple(int(v) for v in n)
    (X, Y, Z), h = _centres(xp, n, lo, hi, nodes)
    Q = xp.zeros((5, n_modes(order), n[2], n[1], n[0]))
    Q[:, 0] = _cons_from_prim(xp, *prim_fn(xp, X, Y, Z, **kw), gamma)
    if order >= 1:
        for d, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            e = h[d] * 1e-3
            qp = _cons_from_prim(xp, *prim_fn(xp, X + dx * e, Y + dy * e, Z + dz * e, **kw), gamma)
            qm = _cons_from_prim(xp, *prim_fn(xp, X - dx * e, Y - dy * e, Z - dz * e, **kw), gamma)
            Q[:, 1 + d] = (qp - qm) * (h[d] / (4 * e))
    if perturb:
        rng = np.random.Generator(np.random.PCG64(seed))
        noise = rng.standard_normal(tuple(Q.shape))
        if device is None:
            scale = np.abs(Q[:, 0]).reshape(5, -1).max(axis=1)
            Q += perturb * scale[:, None, None, None, None] * noise
        else:
            scale = Q[:, 0].abs().reshape(5, -1).max(dim=1).values
            Q += perturb * scale[:, None, None, None, None] * xp.t.from_numpy(noise).to(device)
    return Q


def advection_state(n, order, perturb=0.0, seed=SEED, gamma=1.4, amp=0.2, device=None, nodes=None):
    return modal_state(advection_prim, n, order, (0.0,) * 3, (2.0,) * 3, gamma, perturb, seed, device,
                       dict(amp=amp), nodes)


def tgv_state(n, order, perturb=0.0, seed=SEED, gamma=1.4, Ma=0.1, isothermal=False, device=None):
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    return modal_state(tgv_prim, n, order, lo, hi, gamma, perturb, seed, device,
                       dict(Ma=Ma, gamma=gamma, isothermal=isothermal))


def random_state(n, order, seed=SEED, rho=(0.5, 2.0), vel=1.0, p=(0.5, 3.0), modes_rel=0.02, gamma=1.4):
    """Non-smooth random state (numpy): every cell mean drawn independently.

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
    Q[:, 0] = _cons_from_prim(_NP, r, U, V, W, pr, gamma)
    if order >= 1:
        Q[:, 1:] = modes_rel * np.abs(Q[:, :1]) * rng.standard_normal(Q[:, 1:].shape)
    return Q


def tgv_dt(n, order, cfl=0.15, gamma=1.4, Ma=0.1, V0=1.0):
    """dt = CFL min(h) / max(|U| + c) from the Taylor-Green initial field at cell centres."""
    (X, Y, Z), h = _centres(_NP, (n, n, n), (-np.pi,) * 3, (np.pi,) * 3)
    rho, U, V, W, p = np.broadcast_arrays(*tgv_prim(_NP, X, Y, Z, V0=V0, Ma=Ma, gamma=gamma))
    c = np.sqrt(gamma * p / rho)
    return cfl * min(h) / float(np.max(np.sqrt(U * U + V * V + W * W) + c))


def advection_dt(n, cfl=0.1, gamma=1.4, amp=0.2, T=None):
    """dt = CFL h / max(|U| + c) for the advection problem on [0,2]^3 (rho >= 1 - amp);
    if T is given, shortened so that an integer number of steps reaches T."""
    h = 2.0 / n
    dt = cfl * h / (math.sqrt(3.0) + math.sqrt(gamma / (1.0 - amp)))
    if T is not None:
        dt = T / math.ceil(T / dt)
    return dt
