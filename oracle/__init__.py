"""DG-HGKS oracle: plain FP64 CPU implementation of the per-stage residual.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA library in
``paper_2202_13821_b300``; the two meet only through the seeded input
generators and the test comparisons.

The arithmetic lives in ``dghgks_oracle.hpp`` (C++, templated on the scalar
so that forward-mode dual numbers give exact Jacobian-vector products); this
file compiles it with g++ and marshals numpy arrays through ctypes.

State layout everywhere: ``Q[var][mode][z][y][x]`` float64, var = (rho, rho U,
rho V, rho W, rho E), modes of P_k ordered by total degree with pure powers
first (Sec. 3, Eq. expansion).

Parity status: every function is pinned by ``tests/test_oracle_*.py``.  The
interface flux of Eq. (flux) is pinned at continuous states by its Euler and
Navier-Stokes limits and at discontinuous states by a brute-force
velocity/time quadrature of the distribution it integrates
(``tests/test_oracle_flux_quadrature.py``).  The Prandtl-number correction
(Pr != 1) is a reading, since the paper does not define it: it acts on F
only (see the header of dghgks_oracle.hpp), and its arithmetic is pinned by
that same quadrature of the definition taken.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, f) for f in ("oracle_capi.cpp", "dghgks_oracle.hpp", "dual.hpp")]
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (-O2 -fopenmp -ffp-contract=off)."""
    newest = max(os.path.getmtime(f) for f in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _SO + ".tmp", os.path.join(_HERE, "oracle_capi.cpp")]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


class _Cfg(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("nq", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("Pr", ctypes.c_double),
                ("tau_eps", ctypes.c_double), ("nodes", ctypes.POINTER(ctypes.c_double) * 3)]


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Problem:
    """Periodic rectilinear hexahedral grid and gas parameters (oracle side).

    ``nodes``: None (uniform cells between lo and hi) or, per axis, None or the
    n_d + 1 increasing node coordinates of that axis (lo/hi then follow them).
    """
    order: int = 1
    nq: int = 2
    n: tuple = (8, 8, 8)
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (2.0, 2.0, 2.0)
    gamma: float = 1.4
    mu: float = 0.0
    Pr: float = 1.0
    tau_eps: float = 0.0
    nodes: tuple = None

    def cfg(self) -> _Cfg:
        c = _Cfg()
        c.order, c.nq = self.order, self.nq
        c.nx, c.ny, c.nz = self.n
        for d in range(3):
            c.lo[d], c.hi[d] = self.lo[d], self.hi[d]
        c.gamma, c.mu, c.Pr, c.tau_eps = self.gamma, self.mu, self.Pr, self.tau_eps
        c._keep = []
        for d in range(3):
            nd = None if self.nodes is None else self.nodes[d]
            if nd is not None:
                a = np.ascontiguousarray(nd, dtype=np.float64)
                if a.shape != (self.n[d] + 1,):
                    raise ValueError(f"axis {d}: {self.n[d] + 1} nodes expected, got {a.shape}")
                c._keep.append(a)
                c.nodes[d] = _p(a)
        return c

    @property
    def n_modes(self) -> int:
        k = self.order
        return (k + 1) * (k + 2) * (k + 3) // 6

    @property
    def shape(self) -> tuple:
        return (5, self.n_modes, self.n[2], self.n[1], self.n[0])


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"oracle {what} failed with code {rc}")


def residual(pb: Problem, Q: np.ndarray, dt: float):
    """L = M^-1 R(Q), L_t = M^-1 R_t(Q) for the whole grid."""
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    L = np.zeros_like(Q)
    Lt = np.zeros_like(Q)
    c = pb.cfg()
    _check(lib().orc_residual(ctypes.byref(c), _p(Q), ctypes.c_double(dt), _p(L), _p(Lt)), "residual")
    return L, Lt


def residual_cells(pb: Problem, Q: np.ndarray, dt: float, cells: np.ndarray, scales: bool = False):
    """(L, L_t) of selected cells (flat index i + nx (j + ny k)), shape [n][5][modes].

    With ``scales=True`` also returns (A, A_t): M^-1 times the sums of the
    absolute values of the contributions to R and R_t (the rounding scale).
    """
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros((len(cells), 5, pb.n_modes))
    outt, A, At = np.zeros_like(out), np.zeros_like(out), np.zeros_like(out)
    c = pb.cfg()
    _check(lib().orc_residual_cells(ctypes.byref(c), _p(Q), ctypes.c_double(dt),
                                    cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    ctypes.c_int64(len(cells)), _p(out), _p(outt), _p(A), _p(At)), "residual_cells")
    return (out, outt, A, At) if scales else (out, outt)


def step(pb: Problem, Q: np.ndarray, dt: float, nsteps: int = 1) -> np.ndarray:
    """nsteps S2O4 steps (Sec. 3, Eq. two-stage); returns the new state."""
    Q = np.array(Q, dtype=np.float64, order="C", copy=True)
    c = pb.cfg()
    _check(lib().orc_step(ctypes.byref(c), _p(Q), ctypes.c_double(dt), ctypes.c_int(nsteps)), "step")
    return Q


def totals(pb: Problem, Q: np.ndarray) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    out = np.zeros(5)
    c = pb.cfg()
    _check(lib().orc_totals(ctypes.byref(c), _p(Q), _p(out)), "totals")
    return out


def kinetic_energy(pb: Problem, Q: np.ndarray, rho0: float = 1.0) -> float:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    e = ctypes.c_double()
    c = pb.cfg()
    _check(lib().orc_kinetic_energy(ctypes.byref(c), _p(Q), ctypes.c_double(rho0), ctypes.byref(e)), "kinetic_energy")
    return e.value


def enstrophy_dissipation(pb: Problem, Q: np.ndarray, rho0: float = 1.0) -> float:
    """eps(zeta) = 2 mu / (rho0 |Omega|) int rho |curl U|^2 / 2 (Sec. 5.3)."""
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    e = ctypes.c_double()
    c = pb.cfg()
    _check(lib().orc_enstrophy_dissipation(ctypes.byref(c), _p(Q), ctypes.c_double(rho0), ctypes.byref(e)),
           "enstrophy_dissipation")
    return e.value


IC_ADVECTION = 1
IC_TGV = 2
IC_VORTEX = 3
IC_SHEAR = 4  # par = (eps, axis d, lo_d, span_d, rho, p): u_{(d+1)%3} = eps sin(2 pi (x_d - lo_d)/span_d)


def project(pb: Problem, ic: int, par) -> np.ndarray:
    """L2 projection of an initial condition of Sec. 5 onto P_k ((k+3)^3 Gauss points).

    ic=1 (advection): par = (amplitude, t); ic=2 (Taylor-Green): par = (V0, rho0, p0, isothermal);
    ic=3 (isotropic vortex): par = (eps, t, xc, yc, Lx, Ly).
    """
    Q = np.zeros(pb.shape)
    par = np.ascontiguousarray(par, dtype=np.float64)
    c = pb.cfg()
    _check(lib().orc_project(ctypes.byref(c), ctypes.c_int(ic), _p(par), _p(Q)), "project")
    return Q


def density_errors(pb: Problem, Q: np.ndarray, ic: int, par) -> np.ndarray:
    """(e_L1, e_L2, e_c) of the density against the exact solution (Sec. 5.1)."""
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    par = np.ascontiguousarray(par, dtype=np.float64)
    out = np.zeros(3)
    c = pb.cfg()
    _check(lib().orc_density_errors(ctypes.byref(c), _p(Q), ctypes.c_int(ic), _p(par), _p(out)), "density_errors")
    return out


# ---- point-level functions (pins) ----

def gauss(n: int):
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().orc_gauss(ctypes.c_int(n), _p(x), _p(w)), "gauss")
    return x, w


def basis(order: int, r):
    nm = (order + 1) * (order + 2) * (order + 3) // 6
    r = np.ascontiguousarray(r, dtype=np.float64)
    b, db = np.zeros(nm), np.zeros(nm * 3)
    lib().orc_basis(ctypes.c_int(order), _p(r), _p(b), _p(db))
    return b, db.reshape(nm, 3)


def moments(U, lam: float, region: int, K: float):
    """Normalised moment tables: (m[3][10], xi[4])."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros(34)
    lib().orc_moments(_p(U), ctypes.c_double(lam), ctypes.c_int(region), ctypes.c_double(K), _p(out))
    return out[:30].reshape(3, 10), out[30:]


def slope(U, lam: float, K: float, b):
    U = np.ascontiguousarray(U, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    a = np.zeros(5)
    lib().orc_slope(_p(U), ctypes.c_double(lam), ctypes.c_double(K), _p(b), _p(a))
    return a


def fit_weights(tau: float, dt: float):
    wF, wFt = np.zeros(6), np.zeros(6)
    lib().orc_fit_weights(ctypes.c_double(tau), ctypes.c_double(dt), _p(wF), _p(wFt))
    return wF, wFt


def face_flux(d: int, QL, dQL, QR, dQR, *, gamma=1.4, mu=0.0, Pr=1.0, tau_eps=0.0, dt=1e-3):
    """Interface flux along +e_d (global frame): returns (F[5], F_t[5])."""
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (QL, dQL, QR, dQR)]
    F, Ft = np.zeros(5), np.zeros(5)
    _check(lib().orc_face_flux(ctypes.c_int(d), _p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]), ctypes.c_double(gamma),
                               ctypes.c_double(mu), ctypes.c_double(Pr), ctypes.c_double(tau_eps),
                               ctypes.c_double(dt), _p(F), _p(Ft)), "face_flux")
    return F, Ft


def cell_flux(Q, dQ, *, gamma=1.4, mu=0.0, Pr=1.0, tau_eps=0.0, dt=1e-3):
    """Interior flux of Eq. (flux-2) at a point: (F[3][5], F_t[3][5])."""
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    dQ = np.ascontiguousarray(dQ, dtype=np.float64)
    F, Ft = np.zeros((3, 5)), np.zeros((3, 5))
    _check(lib().orc_cell_flux(_p(Q), _p(dQ), ctypes.c_double(gamma), ctypes.c_double(mu), ctypes.c_double(Pr),
                               ctypes.c_double(tau_eps), ctypes.c_double(dt), _p(F), _p(Ft)), "cell_flux")
    return F, Ft


def s2o4_scalar(lam: float, q0: float, dt: float) -> float:
    """One S2O4 step of dq/dt = lam q (L = lam q, L_t = lam^2 q) through the oracle's combination."""
    out = ctypes.c_double()
    lib().orc_s2o4_scalar(ctypes.c_double(lam), ctypes.c_double(q0), ctypes.c_double(dt), ctypes.byref(out))
    return out.value


# ---- forward-mode derivatives (dual numbers) ----

def residual_jvp(pb: Problem, Q, dQ, dmu: float, dt: float):
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    dQ = np.ascontiguousarray(dQ, dtype=np.float64)
    L, Lt, dL, dLt = (np.zeros_like(Q) for _ in range(4))
    c = pb.cfg()
    _check(lib().orc_residual_jvp(ctypes.byref(c), _p(Q), _p(dQ), ctypes.c_double(dmu), ctypes.c_double(dt),
                                  _p(L), _p(Lt), _p(dL), _p(dLt)), "residual_jvp")
    return L, Lt, dL, dLt


def step_jvp(pb: Problem, Q, dQ, dmu: float, dt: float, nsteps: int, rho0: float = 1.0):
    """Returns (Q_N, dQ_N, E_k(Q_N), dE_k) along the direction (dQ, dmu)."""
    Q = np.array(Q, dtype=np.float64, order="C", copy=True)
    dQ = np.array(dQ, dtype=np.float64, order="C", copy=True)
    e, de = ctypes.c_double(), ctypes.c_double()
    c = pb.cfg()
    _check(lib().orc_step_jvp(ctypes.byref(c), _p(Q), _p(dQ), ctypes.c_double(dmu), ctypes.c_double(dt),
                              ctypes.c_int(nsteps), ctypes.c_double(rho0), ctypes.byref(e), ctypes.byref(de)),
           "step_jvp")
    return Q, dQ, e.value, de.value
