"""Thin Python binding of the C ABI in include/dghgks.h (ctypes).

Module-level functions carry the C names and only marshal arguments: torch
CUDA tensors become device pointers, the current torch stream becomes the
cudaStream_t.  Every step of the computation runs in libdghgks.so; there is
no Python or CPU fallback, and a missing library raises immediately.

``Solver`` bundles a context with its mesh and convenience allocators.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libdghgks.so")

DGHGKS_FP64 = 0
DGHGKS_FP32_MIXED = 1
DGHGKS_FP32_STAGE64 = 2  # FP32 flux and projection; FP64 M^-1 and S2O4 stage combination
ERRORS = {-1: "bad argument", -2: "unsupported", -3: "CUDA error", -4: "non-physical state", -5: "out of memory",
          -6: "problem exceeds the fixed scratch of dghgks_residual_static"}


class DghgksError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dghgks error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("periodic", ctypes.c_int * 3),
                ("nodes", ctypes.POINTER(ctypes.c_double) * 3)]


class Opts(ctypes.Structure):
    _fields_ = [("n_q", ctypes.c_int), ("precision", ctypes.c_int), ("tau_eps", ctypes.c_double)]


_lib = None
_VP = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_DP = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "dghgks_init": (_I, [ctypes.POINTER(Mesh), _I, _D, _D, _D, ctypes.POINTER(Opts), ctypes.POINTER(_VP)]),
    "dghgks_destroy": (None, [_VP]),
    "dghgks_last_error": (ctypes.c_char_p, [_VP]),
    "dghgks_n_modes": (_I, [_VP]),
    "dghgks_set_mu": (_I, [_VP, _D]),
    "dghgks_residual": (_I, [_VP, _VP, _D, _VP, _VP, _VP]),
    "dghgks_step": (_I, [_VP, _VP, _D, _VP]),
    "dghgks_steps": (_I, [_VP, _VP, _D, _I, _VP]),
    "dghgks_run_host": (_I, [_VP, _DP, _D, _I, _D, _DP, _VP]),
    "dghgks_totals": (_I, [_VP, _VP, _DP, _VP]),
    "dghgks_kinetic_energy": (_I, [_VP, _VP, _D, _DP, _VP]),
    "dghgks_l2_diff": (_I, [_VP, _VP, _VP, _I, _DP, _VP]),
    "dghgks_enstrophy_dissipation": (_I, [_VP, _VP, _D, _DP, _VP]),
    "dghgks_status": (_I, [_VP, _VP]),
    "dghgks_launch_count": (ctypes.c_int64, [_VP]),
    "dghgks_gauss_rule": (_I, [_I, _DP, _DP]),
    "dghgks_residual_static": (_I, [ctypes.POINTER(Mesh), _I, _D, _D, _D, ctypes.POINTER(Opts), _VP, _D, _VP, _VP,
                                    _VP]),
    "dghgks_residual_vjp": (_I, [_VP, _VP, _D, _VP, _VP, _VP, _VP, _VP]),
    "dghgks_adjoint_step": (_I, [_VP, _VP, _VP, _D, _VP, _VP, _VP]),
    "dghgks_kinetic_energy_vjp": (_I, [_VP, _VP, _D, _VP, _VP]),
    "dghgks_profile": (_I, [_VP, _I]),
    "dghgks_profile_read": (_I, [_VP, _DP, ctypes.POINTER(ctypes.c_int64)]),
    "dghgks_pipe_rates": (_I, [_DP, _I]),
}

NKINDS = 7
KIND_NAMES = ("face_x", "face_y", "face_z", "cell_residual", "cell_stage1", "cell_stage2", "reduction")


def load():
    """Load libdghgks.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise RuntimeError(f"{_SO} is missing: build it with `python -m paper_2202_13821_b300.build`")
        lib = ctypes.CDLL(_SO)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def _ptr(t) -> int:
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


def _stream(stream=None):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(ctx, rc: int):
    if rc != 0:
        raise DghgksError(rc, load().dghgks_last_error(ctx).decode())


# ---- functions with the C names ----

def dghgks_init(n, lo, hi, order: int, gamma: float, mu: float, Pr: float, n_q: int = 0,
                precision: int = DGHGKS_FP64, tau_eps: float = 0.0, nodes=None):
    """nodes: None, or per axis None / the n_d + 1 increasing node coordinates (host)."""
    m = Mesh()
    m.nx, m.ny, m.nz = (int(v) for v in n)
    keep = []
    for d in range(3):
        m.lo[d], m.hi[d], m.periodic[d] = lo[d], hi[d], 1
        nd = None if nodes is None else nodes[d]
        if nd is not None:
            a = np.ascontiguousarray(nd, dtype=np.float64)
            if a.shape != (int(n[d]) + 1,):
                raise ValueError(f"axis {d}: wrong number of mesh nodes {a.shape}")
            keep.append(a)
            m.nodes[d] = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    o = Opts(int(n_q), int(precision), float(tau_eps))
    ctx = _VP()
    rc = load().dghgks_init(ctypes.byref(m), int(order), gamma, mu, Pr, ctypes.byref(o), ctypes.byref(ctx))
    if rc != 0:
        raise DghgksError(rc, load().dghgks_last_error(None).decode())
    return ctx


def dghgks_residual_static(n, lo, hi, order: int, gamma: float, mu: float, Pr: float, Q, dt: float, L, Lt,
                           n_q: int = 0, precision: int = DGHGKS_FP64, tau_eps: float = 0.0, stream=None):
    """Residual without allocation or context (scratch in a fixed device array); see include/dghgks.h."""
    m = Mesh()
    m.nx, m.ny, m.nz = (int(v) for v in n)
    for d in range(3):
        m.lo[d], m.hi[d], m.periodic[d] = lo[d], hi[d], 1
    o = Opts(int(n_q), int(precision), float(tau_eps))
    rc = load().dghgks_residual_static(ctypes.byref(m), int(order), gamma, mu, Pr, ctypes.byref(o), _ptr(Q), dt,
                                       _ptr(L), _ptr(Lt), _stream(stream))
    if rc != 0:
        raise DghgksError(rc, "dghgks_residual_static")


def dghgks_pipe_rates() -> dict:
    """Measured FP32/FP64 FMA FLOP/s, operations/s of the FP32 flux's division, rsqrt, exp and erfc,
    and the SM count of the current device (see include/dghgks.h)."""
    out = np.zeros(7)
    rc = load().dghgks_pipe_rates(out.ctypes.data_as(_DP), 7)
    if rc != 0:
        raise DghgksError(rc, "dghgks_pipe_rates")
    keys = ("ffma_flops", "dfma_flops", "div_ops", "rsqrt_ops", "exp_ops", "erfc_ops", "sms")
    return dict(zip(keys, out.tolist()))


def dghgks_destroy(ctx):
    load().dghgks_destroy(ctx)


def dghgks_residual(ctx, Q, dt: float, L, Lt, stream=None):
    _check(ctx, load().dghgks_residual(ctx, _ptr(Q), dt, _ptr(L), _ptr(Lt), _stream(stream)))


def dghgks_step(ctx, Q, dt: float, stream=None):
    _check(ctx, load().dghgks_step(ctx, _ptr(Q), dt, _stream(stream)))


def dghgks_steps(ctx, Q, dt: float, nsteps: int, stream=None):
    _check(ctx, load().dghgks_steps(ctx, _ptr(Q), dt, int(nsteps), _stream(stream)))


def dghgks_run_host(ctx, Q_host: np.ndarray, dt: float, nsteps: int, rho0: float = 1.0, ek_host=None, stream=None):
    assert Q_host.dtype == np.float64 and Q_host.flags.c_contiguous
    ekp = None if ek_host is None else ek_host.ctypes.data_as(_DP)
    _check(ctx, load().dghgks_run_host(ctx, Q_host.ctypes.data_as(_DP), dt, int(nsteps), rho0, ekp, _stream(stream)))


def dghgks_totals(ctx, Q, stream=None) -> np.ndarray:
    out = np.zeros(5)
    _check(ctx, load().dghgks_totals(ctx, _ptr(Q), out.ctypes.data_as(_DP), _stream(stream)))
    return out


def dghgks_kinetic_energy(ctx, Q, rho0: float = 1.0, stream=None) -> float:
    e = ctypes.c_double()
    _check(ctx, load().dghgks_kinetic_energy(ctx, _ptr(Q), rho0, ctypes.byref(e), _stream(stream)))
    return e.value


def dghgks_enstrophy_dissipation(ctx, Q, rho0: float = 1.0, stream=None) -> float:
    e = ctypes.c_double()
    _check(ctx, load().dghgks_enstrophy_dissipation(ctx, _ptr(Q), rho0, ctypes.byref(e), _stream(stream)))
    return e.value


def dghgks_l2_diff(ctx, A, B, var: int = 0, stream=None) -> float:
    e = ctypes.c_double()
    _check(ctx, load().dghgks_l2_diff(ctx, _ptr(A), _ptr(B), int(var), ctypes.byref(e), _stream(stream)))
    return e.value


def dghgks_status(ctx, stream=None):
    _check(ctx, load().dghgks_status(ctx, _stream(stream)))


def dghgks_set_mu(ctx, mu: float):
    _check(ctx, load().dghgks_set_mu(ctx, mu))


def dghgks_launch_count(ctx) -> int:
    return int(load().dghgks_launch_count(ctx))


def dghgks_gauss_rule(n: int):
    x, w = np.zeros(n), np.zeros(n)
    rc = load().dghgks_gauss_rule(n, x.ctypes.data_as(_DP), w.ctypes.data_as(_DP))
    if rc:
        raise DghgksError(rc, "gauss rule")
    return x, w


def dghgks_residual_vjp(ctx, Q, dt: float, lamL, lamLt, lamQ, dmu, stream=None):
    """lamQ <- (dL/dQ)^T lamL + (dLt/dQ)^T lamLt; dmu (1-element CUDA tensor) += viscosity part."""
    _check(ctx, load().dghgks_residual_vjp(ctx, _ptr(Q), dt, _ptr(lamL), _ptr(lamLt), _ptr(lamQ), _ptr(dmu),
                                           _stream(stream)))


def dghgks_adjoint_step(ctx, Qn, lam_next, dt: float, lam_n, dJ_dmu, stream=None):
    _check(ctx, load().dghgks_adjoint_step(ctx, _ptr(Qn), _ptr(lam_next), dt, _ptr(lam_n), _ptr(dJ_dmu),
                                           _stream(stream)))


def dghgks_kinetic_energy_vjp(ctx, Q, rho0: float, out, stream=None):
    _check(ctx, load().dghgks_kinetic_energy_vjp(ctx, _ptr(Q), rho0, _ptr(out), _stream(stream)))


def dghgks_profile(ctx, enable: bool):
    _check(ctx, load().dghgks_profile(ctx, 1 if enable else 0))


def dghgks_profile_read(ctx):
    ms = np.zeros(NKINDS)
    n = np.zeros(NKINDS, dtype=np.int64)
    _check(ctx, load().dghgks_profile_read(ctx, ms.ctypes.data_as(_DP), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return {KIND_NAMES[k]: (float(ms[k]), int(n[k])) for k in range(NKINDS)}


# ---- convenience wrapper ----

@dataclass
class Solver:
    """A DG-HGKS context on the current CUDA device."""
    n: tuple
    lo: tuple
    hi: tuple
    order: int = 2
    gamma: float = 1.4
    mu: float = 0.0
    Pr: float = 1.0
    n_q: int = 0
    precision: int = DGHGKS_FP64
    tau_eps: float = 0.0
    nodes: tuple = None  # rectilinear mesh: per axis None or n_d + 1 node coordinates

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        self.ctx = dghgks_init(self.n, self.lo, self.hi, self.order, self.gamma, self.mu, self.Pr, self.n_q,
                               self.precision, self.tau_eps, self.nodes)
        self.n_modes = load().dghgks_n_modes(self.ctx)

    @property
    def shape(self):
        return (5, self.n_modes, self.n[2], self.n[1], self.n[0])

    def close(self):
        if getattr(self, "ctx", None):
            dghgks_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self):
        import torch

        return torch.empty(self.shape, dtype=torch.float64, device="cuda")

    def residual(self, Q, dt, L=None, Lt=None, stream=None):
        L = self.empty() if L is None else L
        Lt = self.empty() if Lt is None else Lt
        dghgks_residual(self.ctx, Q, dt, L, Lt, stream)
        return L, Lt

    def step(self, Q, dt, nsteps: int = 1, stream=None):
        for _ in range(nsteps):
            dghgks_step(self.ctx, Q, dt, stream)
        return Q

    def steps(self, Q, dt, nsteps: int, stream=None):
        """nsteps steps by CUDA-graph replay (dghgks_steps)."""
        dghgks_steps(self.ctx, Q, dt, nsteps, stream)
        return Q

    def run_host(self, Q_host, dt, nsteps, rho0=1.0, with_ek=True, stream=None):
        ek = np.zeros(nsteps) if with_ek else None
        dghgks_run_host(self.ctx, Q_host, dt, nsteps, rho0, ek, stream)
        return ek

    def totals(self, Q, stream=None):
        return dghgks_totals(self.ctx, Q, stream)

    def kinetic_energy(self, Q, rho0=1.0, stream=None):
        return dghgks_kinetic_energy(self.ctx, Q, rho0, stream)

    def enstrophy_dissipation(self, Q, rho0=1.0, stream=None):
        return dghgks_enstrophy_dissipation(self.ctx, Q, rho0, stream)

    def l2_diff(self, A, B, var=0, stream=None):
        return dghgks_l2_diff(self.ctx, A, B, var, stream)

    def status(self, stream=None):
        dghgks_status(self.ctx, stream)

    def set_mu(self, mu):
        dghgks_set_mu(self.ctx, mu)
        self.mu = mu

    def profile(self, enable: bool):
        dghgks_profile(self.ctx, enable)

    def profile_read(self):
        return dghgks_profile_read(self.ctx)

    @property
    def launches(self) -> int:
        return dghgks_launch_count(self.ctx)
