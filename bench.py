#!/usr/bin/env python
"""Throughput of the DG-HGKS per-stage residual on one B300 (or N replicas).

Workload: Taylor-Green vortex (Sec. 5.3 of arXiv:2202.13821) on a periodic
256^3 uniform grid, P2 elements (10 modes x 5 variables per cell), 3x3 face and
3^3 cell Gauss points, Re = 1600, Ma = 0.1, Pr = 0.72, gamma = 1.4, dt from
CFL 0.15.  A step is one S2O4 time step = two full residual stages over the
whole grid (3 face launches + 1 cell launch per stage).

Metric: DOF-stage-updates/s = 5 * N_modes * N_cells * 2 / (time per step),
whole job (sum over ranks).  The headline value is the FP32-mixed path, timed
as a user runs it: one dghgks_steps call of K steps (CUDA-graph replay) between
two CUDA events, after W untimed steps; per-kernel times for the roofline come
from a separate profiled pass.  Beside it: the FP32 flux with FP64 stage
arithmetic and the FP64 path on the same state, the errors of the FP32 paths
against FP64 (L2 density difference, relative kinetic-energy history; over
the bench's steps at 256^3 and over a 400-step run at 64^3) and against the
oracle (the oracle steps 9^3 boxes cut around sampled cells; that is also the
CPU baseline), the end-to-end rate through dghgks_run_host with
host buffers, the measured FMA and transcendental rates of the GPU, and the
adjoint leg (Taylor-Green 64^3 P2 FP64, 100 checkpointed steps).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the method written plainly from
the paper): each step is a whole S2O4 step of the oracle on a periodic 16^3
Taylor-Green grid (P2, n_q = 3), the workload at a size the host cores step
in seconds.
Multi-GPU: one replica per rank ("replicas only": independent problems, no
data-path collective), weak scaling; barrier + max over ranks for timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-stage-updates/s, TGV P2 256^3: FP32-mixed vs FP64, at stated L2/KE error"
UNIT = "DOF-stage-updates/s"
N_CELLS_1D = 256
ORDER, NQ = 2, 3
MU, PR, GAMMA, MA = 1.0 / 1600.0, 0.72, 1.4, 0.1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_CELLS_1D, help="cells per direction")
    ap.add_argument("--fp64-steps", type=int, default=None, help="timed FP64 steps (default: --steps)")
    ap.add_argument("--boxes", type=int, default=24, help="9^3 boxes the oracle steps for the CPU baseline and the "
                                                        "error against the oracle")
    ap.add_argument("--ref-n", type=int, default=16, help="grid of the reference arm's oracle steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stage64", action="store_true", help="skip the FP32-flux / FP64-stage leg")
    ap.add_argument("--cpu-config2", action="store_true",
                    help="also time the oracle on BASELINE configuration 2 in full (64^3 P2, 2 steps; ~2 min)")
    ap.add_argument("--adjoint-n", type=int, default=64, help="cells per direction of the adjoint leg (0: skip)")
    ap.add_argument("--adjoint-steps", type=int, default=100, help="checkpointed steps of the adjoint leg")
    ap.add_argument("--long-error-n", type=int, default=64, help="cells per direction of the long-run error leg")
    ap.add_argument("--long-error-steps", type=int, default=400,
                    help="steps of the long-run FP32-vs-FP64 error leg (0: skip)")
    return ap.parse_args()


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Ranks:
    """Replica bookkeeping across ranks: barrier, max over ranks, whole-job sums.

    Each rank runs an independent replica of the workload (no data-path
    collective); timing takes the slowest rank, throughput counts every
    rank's units.  backend "nccl" on GPUs, "gloo" for the CPU tests."""

    def __init__(self, world: int, backend: str = "nccl", device=None):
        self.world = world
        self.dist = None
        self.device = device
        if world > 1:
            import torch.distributed as dist

            if not dist.is_initialized():
                kw = {"device_id": device} if backend == "nccl" and device is not None else {}
                dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch

        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def job_rate(self, units_per_rank: float, seconds_max: float) -> float:
        """Whole-job throughput: every rank processed units_per_rank in at most seconds_max."""
        return units_per_rank * self.world / seconds_max

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def workload_config(n, dt):
    return {
        "workload": f"Taylor-Green vortex {n}^3 cells, P2 (10 modes x 5 vars), 3x3 face / 3^3 cell Gauss points, "
                    f"Re=1600, Ma=0.1, Pr=0.72, CFL 0.15, one S2O4 step per iteration",
        "cells": n ** 3,
        "dofs": 5 * 10 * n ** 3,
        "order": ORDER,
        "n_q": NQ,
        "dt": dt,
        "l2_policy": f"inputs larger than L2: state {5 * 10 * n ** 3 * 8 / 1e9:.2f} GB per buffer, no flush",
        "parallelism": "replicas",
    }


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------
def sample_cells(n, count):
    """Cells (i, j, k) of the n^3 grid whose 9^3 boxes the oracle steps: the corners and an interior
    cell, then seeded random ones."""
    import numpy as np

    rng = np.random.default_rng(5)
    fixed = [(0, 0, 0), (n - 1, n - 1, n - 1), (131 % n, 7 % n, 200 % n)]
    return fixed + [tuple(int(x) for x in rng.integers(0, n, 3)) for _ in range(max(0, count - len(fixed)))]


def box_of(Q0, n, cell):
    """The periodic 9^3 box of the n^3 state around `cell` (device tensor in, numpy out) and its lower corner.

    After 2 S2O4 steps (4 stages) a cell depends only on the cells within 4 face-neighbour hops, so
    the oracle stepping the box reproduces the full-grid result at its centre exactly."""
    import torch

    i, j, k = cell
    ix, iy, iz = (torch.tensor([(c + d) % n for d in range(-4, 5)], device=Q0.device) for c in (i, j, k))
    sub = Q0.index_select(2, iz).index_select(3, iy).index_select(4, ix).cpu().numpy()
    h = 2 * math.pi / n
    lo = tuple(-math.pi + (c - 4) * h for c in (i, j, k))
    return sub, lo


def oracle_boxes(boxes, n, dt, nsteps=2):
    """The oracle's nsteps S2O4 steps of each 9^3 box; returns (centre coefficients [cells][5][10], seconds,
    threads)."""
    import numpy as np

    import oracle

    oracle.build()
    h = 2 * math.pi / n
    out = []
    t0 = time.perf_counter()
    for sub, lo in boxes:
        pb = oracle.Problem(order=ORDER, nq=NQ, n=(9, 9, 9), lo=lo, hi=tuple(x + 9 * h for x in lo), mu=MU, Pr=PR,
                            gamma=GAMMA)
        out.append(oracle.step(pb, sub, dt, nsteps)[:, :, 4, 4, 4])
    el = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return np.array(out), el, threads


def oracle_config1():
    """BASELINE configuration 1 run in full by the oracle: 3D density advection, 8^3 P1, n_q = 2,
    tau = 0.01 dt, CFL 0.1, S2O4 to t = 0.1.  Returns (DOF-stage-updates/s, seconds, steps)."""
    import oracle
    from paper_2202_13821_b300 import inputs

    oracle.build()
    T = 0.1
    dt = inputs.advection_dt(8, T=T)
    ns = round(T / dt)
    pb = oracle.Problem(order=1, nq=2, n=(8, 8, 8), lo=(0.0,) * 3, hi=(2.0,) * 3, tau_eps=0.01)
    Q = oracle.project(pb, oracle.IC_ADVECTION, (0.2, 0.0))
    t0 = time.perf_counter()
    oracle.step(pb, Q, dt, ns)
    el = time.perf_counter() - t0
    return 8 ** 3 * 5 * 4 * 2 * ns / el, el, ns


def oracle_config2(nsteps=2):
    """BASELINE configuration 2 run by the oracle: Taylor-Green 64^3 P2, n_q = 3, dt from CFL 0.15, nsteps
    S2O4 steps from the projected initial state.  Returns (DOF-stage-updates/s, seconds)."""
    import oracle
    from paper_2202_13821_b300 import inputs

    oracle.build()
    n = 64
    dt = inputs.tgv_dt(n, ORDER)
    pb = oracle.Problem(order=ORDER, nq=NQ, n=(n, n, n), lo=(-math.pi,) * 3, hi=(math.pi,) * 3, mu=MU, Pr=PR,
                        gamma=GAMMA)
    Q = inputs.tgv_state(n, ORDER, device="cpu").numpy()
    t0 = time.perf_counter()
    oracle.step(pb, Q, dt, nsteps)
    el = time.perf_counter() - t0
    return n ** 3 * 50 * 2 * nsteps / el, el


def run_reference(args):
    """The reference arm: the FP64 oracle (the method written plainly from the paper), timed on the host
    cores.  Each step is one whole S2O4 step of the oracle on a periodic Taylor-Green grid of
    --ref-n^3 cells (P2, n_q = 3, the workload's physics and dt rule at a size the CPU steps in a few
    seconds; the per-DOF cost does not depend on the grid size)."""
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    from paper_2202_13821_b300 import inputs

    oracle.build()
    m = args.ref_n
    dt = inputs.tgv_dt(m, ORDER)
    pb = oracle.Problem(order=ORDER, nq=NQ, n=(m, m, m), lo=(-math.pi,) * 3, hi=(math.pi,) * 3, mu=MU, Pr=PR,
                        gamma=GAMMA)
    Q = inputs.tgv_state(m, ORDER, device="cpu").numpy()
    times = []
    for _ in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        Q = oracle.step(pb, Q, dt, 1)
        times.append(time.perf_counter() - t0)
    timed = times[args.warmup:] or times
    sec = statistics.mean(timed)
    value = 5 * 10 * m ** 3 * 2 / sec
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"oracle (FP64, each cell evaluating its own six faces), whole S2O4 steps of the Taylor-Green "
              f"vortex on a periodic {m}^3 grid, P2, n_q = 3, dt from CFL 0.15 ({dt:.3e}); "
              f"DOF-stage-updates/s = {m}^3 x 50 x 2 / step time")
    cfg = workload_config(args.n, inputs.tgv_dt(args.n, ORDER))
    cfg["reference_sample"] = {"cells": m ** 3, "dt": dt}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [l.strip().split(", ") for l in open(self.f.name) if l.strip() and not l.startswith("index")]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1].split()[0]))
                smax.append(float(r[2].split()[0]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip() == "Active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash() -> str:
    """Hash of the forward kernel sources and of their compiler options; a profile summary is valid
    only for the same hash."""
    import hashlib

    from paper_2202_13821_b300 import build

    h = hashlib.sha1()
    for f in ("dg_kernels.cuh", "gks_point.cuh", "dg_tables.cuh"):
        with open(os.path.join(ROOT, "paper_2202_13821_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(build.NVCC_FLAGS + build.EXTRA.get("dghgks_api.cu", [])).encode())
    return h.hexdigest()[:12]


def profiled_traffic(kernel: str, n: int):
    """DRAM bytes per launch of `kernel` from a committed ncu summary (profiles/<kernel>_*.md),
    scaled to n^3 cells; None if no summary matches the current kernel sources."""
    import glob
    import re

    cur = kernel_source_hash()
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_*.md"))):
        txt = open(f).read()
        mh = re.search(r"source-hash:\s*([0-9a-f]+)", txt)
        mb = re.search(r"dram-bytes-per-cell:\s*([0-9.eE+]+)", txt)
        if mh and mb and mh.group(1) == cur:
            return float(mb.group(1)) * n ** 3, os.path.relpath(f, ROOT)
    return None, None


def run_leg(torch, api, precision, Q0, dt, warmup, steps, barrier, clock=None, prof_steps=3, cells=()):
    """One precision on the workload: the states after 2 steps at the sampled cells (for the error against
    the oracle), `warmup` untimed steps, `steps` timed steps of the production path (one dghgks_steps call,
    CUDA-graph replay, no per-launch events), then a separate profiled pass of `prof_steps` steps on a copy
    (each launch bracketed by CUDA events) for the per-kernel times of the roofline."""
    n = Q0.shape[4]
    s = api.Solver((n, Q0.shape[3], Q0.shape[2]), (-math.pi,) * 3, (math.pi,) * 3, order=ORDER,
                   gamma=GAMMA, mu=MU, Pr=PR, n_q=NQ, precision=precision)
    centres = None
    if cells:
        Q2 = Q0.clone()
        s.steps(Q2, dt, 2)
        s.status()
        centres = torch.stack([Q2[:, :, k, j, i] for (i, j, k) in cells]).cpu().numpy()
        del Q2
    Q = Q0.clone()
    ek = [s.kinetic_energy(Q)]
    for _ in range(warmup):
        s.steps(Q, dt, 1)
        ek.append(s.kinetic_energy(Q))
    s.status()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.steps(Q.clone(), dt, 2)  # capture both step graphs of this dt outside the timed region
    torch.cuda.synchronize()
    barrier()
    launches0 = s.launches
    if clock is not None:
        clock.start()
    e0.record(stream)
    s.steps(Q, dt, steps)  # FP32 contexts: the state rounded to FP32 carries over between the steps
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clock.stop() if clock is not None else None
    barrier()
    ms = e0.elapsed_time(e1)
    launches = s.launches - launches0
    s.status()
    ek.append(s.kinetic_energy(Q))
    prof = None
    if prof_steps > 0:
        Qp = Q.clone()
        s.profile(True)
        s.steps(Qp, dt, prof_steps)
        prof = s.profile_read()
        s.profile(False)
        s.status()
        del Qp
    return {"solver": s, "Q": Q, "ms": ms, "prof": prof, "launches": launches, "ek": ek, "clocks": clocks,
            "centres": centres}


def long_run_error(torch, api, n, steps):
    """FP32-mixed and FP32-flux / FP64-stage runs against an FP64 run of the same Taylor-Green state over
    `steps` S2O4 steps at n^3: the L2 density difference to FP64 against the FP64 density change from t = 0
    at checkpoints (the early density change of this initial field is small and not monotonic, so the
    256^3 comparison over the bench's few steps divides by a near-zero signal), and the E_k difference."""
    lo, hi = (-math.pi,) * 3, (math.pi,) * 3
    kw = dict(order=ORDER, gamma=GAMMA, mu=MU, Pr=PR, n_q=NQ)
    from paper_2202_13821_b300 import inputs
    Q0 = inputs.tgv_state(n, ORDER, device="cuda")
    dt = inputs.tgv_dt(n, ORDER)
    sol = {p: api.Solver((n,) * 3, lo, hi, precision=p, **kw) for p in (0, 1, 2)}
    Q = {p: Q0.clone() for p in sol}
    out = {"workload": f"Taylor-Green {n}^3 P2, n_q = 3, dt from CFL 0.15", "checkpoints": []}
    done = 0
    for target in sorted({max(1, steps // 16), max(1, steps // 4), steps}):
        for p in sol:
            sol[p].steps(Q[p], dt, target - done)
        done = target
        chg = sol[0].l2_diff(Q[0], Q0, 0)
        ek64 = sol[0].kinetic_energy(Q[0])
        row = {"steps": target, "t": target * dt, "l2_rho_change_fp64": chg}
        for p, tag in ((1, "fp32"), (2, "fp32_stage64")):
            d = sol[0].l2_diff(Q[p], Q[0], 0)
            row[tag] = {"l2_rho_vs_fp64": d, "ratio_rho": d / chg,
                        "ek_rel_diff": abs(sol[0].kinetic_energy(Q[p]) - ek64) / ek64}
        out["checkpoints"].append(row)
    for p in sol:
        sol[p].status()
        sol[p].close()
    return out


def algorithmic_bytes(kernel, precision):
    """HBM bytes per cell of one launch, mean of the two stages of a step (P2: 50 state coefficients,
    60 face moments per face): each value read or written once, neighbours' data counted once.

    k_face stage 1 reads the state and writes the F and F_t moments; stage 2 reads Q* (flux
    precision) and writes the F_t moments.  k_cell stage 1 reads the state and the moments of its
    faces and writes Q* and inc; stage 2 reads Q*, inc, the F_t moments and the FP64 state and
    writes the state.  FP32 steps read the state rounded to FP32 at stage 1, which stage 2 writes
    besides the FP64 state (the rounding kernel at the start of a call is not counted); with FP64
    stage arithmetic (precision 2) inc is FP64 and stage 1 also reads the FP64 state for Q*."""
    r = 4 if precision in (1, 2) else 8
    e = 8 if precision in (0, 2) else 4
    coef, mom = 5 * 10, 10 * 6
    state_in = coef * r  # FP32 copy (FP32 contexts) or the FP64 state
    copy_out = coef * 4 if precision in (1, 2) else 0
    if kernel == "k_face":
        s1 = state_in + mom * r
        s2 = coef * r + mom // 2 * r
    else:
        s1 = state_in + 3 * mom * r + coef * r + coef * e + (coef * 8 if precision == 2 else 0)
        s2 = coef * r + coef * e + 3 * (mom // 2) * r + 2 * coef * 8 + copy_out
    return (s1 + s2) / 2


def charged_flops(point, rates):
    """Work of one flux point in FP32 FMA-equivalent FLOP: the counted additions and multiplications, and
    each division, reciprocal square root, exponential and erfc at its measured cost (the FMA FLOPs the
    GPU issues in the time of one such operation, from dghgks_pipe_rates).  The counter records a
    reciprocal square root as a square root and a division by it; on the GPU it is one instruction."""
    c = {k: rates["ffma_flops"] / rates[k + "_ops"] for k in ("div", "rsqrt", "exp", "erfc")}
    base = point["total_flops"] - point["div"]
    extra = (point["div"] - point["sqrt"]) * c["div"] + point["sqrt"] * c["rsqrt"] + point["exp"] * c["exp"] + \
        point["erfc"] * c["erfc"]
    return base, extra, c


def roofline_entry(prof, precision, n, rates, clocks):
    """Roofline of the dominant kernel: algorithmic FLOPs per launch (value-numbered counts of the flux,
    trace and projection arithmetic; FP32 contexts also charge the transcendentals at their measured
    cost) over the kernel's mean CUDA-event launch time in the profiled pass, against the measured FMA
    rate of this GPU (dghgks_pipe_rates)."""
    from paper_2202_13821_b300 import build

    oc = build.opcounts(ORDER, NQ, PR != 1.0)
    face_ms = sum(prof[k][0] for k in ("face_x", "face_y", "face_z"))
    face_n = sum(prof[k][1] for k in ("face_x", "face_y", "face_z"))
    cell_ms = prof["cell_stage1"][0] + prof["cell_stage2"][0]
    cell_n = prof["cell_stage1"][1] + prof["cell_stage2"][1]
    pts = n ** 3 * NQ * NQ  # face points of one face launch (one normal direction)
    cpts = n ** 3 * NQ ** 3
    fp32 = precision in (1, 2)
    kernels = {}
    for name, npts, ms_, nl, key in (("k_face", pts, face_ms, face_n, "face_point"),
                                     ("k_cell", cpts, cell_ms, cell_n, "cell_point")):
        pt = oc[key]
        # a step launches each kernel once per stage; the stage-2 launches need F_t only (the counts keep
        # only the operations F_t depends on; the transcendentals are needed by both), so the per-launch
        # figure is the mean of the two
        counted = npts * (pt["total_flops"] + pt["total_flops_ft"]) / 2
        charged = counted
        if fp32:
            base, extra, _ = charged_flops(pt, rates)
            charged = counted - npts * pt["div"] + npts * extra
        kernels[name] = {"launches": nl, "avg_ms": ms_ / max(nl, 1), "flops_per_launch": counted,
                         "charged_flops_per_launch": charged}
    dom = max(kernels, key=lambda k: kernels[k]["avg_ms"] * kernels[k]["launches"])
    kd = kernels[dom]
    achieved = kd["charged_flops_per_launch"] / (kd["avg_ms"] * 1e-3) / 1e12
    achieved_counted = kd["flops_per_launch"] / (kd["avg_ms"] * 1e-3) / 1e12
    sms = rates.get("sms", 148)
    smax = (clocks or {}).get("sm_max_mhz") or 2032.0
    if fp32:
        peak = rates["ffma_flops"] / 1e12
        derived = sms * 128 * 2 * smax * 1e6 / 1e12
        peak_src = (f"measured: FP32 FMA loop (dghgks_pipe_rates, {int(sms)} SMs) = {peak:.1f} TFLOP/s; "
                    f"derived {int(sms)} SMs x 128 lanes x 2 x {smax:.0f} MHz = {derived:.1f}")
        charges = charged_flops(oc["face_point"], rates)[2]
    else:
        peak = rates["dfma_flops"] / 1e12
        derived = None
        peak_src = f"measured: FP64 FMA loop (dghgks_pipe_rates) = {peak:.3f} TFLOP/s (B300 nominal 1.25)"
        charges = None
    traffic, traffic_src = profiled_traffic(dom, n) if precision == 1 else (None, None)
    entry = {
        "bound": "alu", "kernel": dom, "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
        "frac": round(achieved / peak, 4), "traffic": traffic, "traffic_source": traffic_src,
        "traffic_algorithmic": n ** 3 * algorithmic_bytes(dom, precision),
        "peak_source": peak_src, "peak_derived": derived,
        "achieved_counted_only": round(achieved_counted, 3), "frac_counted_only": round(achieved_counted / peak, 4),
        "algorithmic_flops": "value-numbered op count per point x points per launch, mean of the two stages "
                             f"(face point {oc['face_point']['total_flops']} / {oc['face_point']['total_flops_ft']} "
                             f"F_t only; cell point {oc['cell_point']['total_flops']} / "
                             f"{oc['cell_point']['total_flops_ft']} F_t only)" +
                             ("; achieved charges each div / rsqrt / exp / erfc at its measured cost in FMA FLOPs "
                              "(charged_flops_per_launch), achieved_counted_only counts each as 1" if fp32 else ""),
        "transcendental_charge_flops": ({k: round(v, 2) for k, v in charges.items()} if charges else None),
        "kernels": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                    for k, v in kernels.items()},
    }
    return entry


def run_adjoint(torch, api, n, nsteps):
    """Gradient of the final E_k w.r.t. the initial state and mu over nsteps checkpointed FP64 steps
    (Taylor-Green P2): measured time per forward and per adjoint step, checkpoint bytes, peak device
    memory of torch's allocator (the checkpoints and the adjoint state) and the device memory in use
    after the forward pass (cudaMemGetInfo: also the library's own scratch)."""
    from paper_2202_13821_b300 import autograd, inputs

    dt = inputs.tgv_dt(n, ORDER)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    base_alloc = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    s = api.Solver((n,) * 3, (-math.pi,) * 3, (math.pi,) * 3, order=ORDER, gamma=GAMMA, mu=MU, Pr=PR, n_q=NQ,
                   precision=api.DGHGKS_FP64)
    Q0 = inputs.tgv_state(n, ORDER, device="cuda").requires_grad_(True)
    mu = torch.tensor(MU, dtype=torch.float64, device="cuda", requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = autograd.kinetic_energy(autograd.rollout(Q0, mu, s, dt, nsteps), s)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    free1, _ = torch.cuda.mem_get_info()  # checkpoints, state and the library's scratch are held here
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    state = Q0.numel() * 8
    fwd, adj = 1e3 * (t1 - t0) / nsteps, 1e3 * (t2 - t1) / nsteps
    out = {"workload": f"Taylor-Green {n}^3 P2 FP64, {nsteps} checkpointed S2O4 steps, dE_k/d(Q0, mu)",
           "steps": nsteps, "forward_ms_per_step": fwd, "adjoint_ms_per_step": adj, "adjoint_over_forward": adj / fwd,
           "checkpoint_bytes_per_step": state, "checkpoint_bytes": nsteps * state,
           "torch_peak_bytes": torch.cuda.max_memory_allocated() - base_alloc,
           "device_bytes_after_forward": free0 - free1, "dJ_dmu": float(mu.grad.item()),
           "grad_norm": float(Q0.grad.norm().item())}
    s.close()
    del Q0, mu, J
    torch.cuda.empty_cache()
    return out


def pipe_rates(api, local):
    """Measured FMA and transcendental rates of this GPU, with the SM clock sampled meanwhile."""
    clock = ClockSampler(local)
    clock.start()
    r = api.dghgks_pipe_rates()
    r["clocks"] = clock.stop()
    return r


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    ranks = Ranks(world, "nccl", torch.device("cuda", local))
    barrier, max_over_ranks = ranks.barrier, ranks.max

    from paper_2202_13821_b300 import api, build, inputs

    build.build()
    api.load()
    n = args.n
    dt = inputs.tgv_dt(n, ORDER)
    dof_step = 5 * 10 * n ** 3 * 2
    flux_step = 2 * (3 * n ** 3 * NQ ** 2 + n ** 3 * NQ ** 3)
    Q0 = inputs.tgv_state(n, ORDER, device="cuda")
    torch.cuda.synchronize()
    rates = pipe_rates(api, local)
    do_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    cells = sample_cells(n, args.boxes) if do_cpu else ()

    # --- FP32-mixed (headline) ---
    m32 = run_leg(torch, api, api.DGHGKS_FP32_MIXED, Q0, dt, args.warmup, args.steps, barrier,
                  ClockSampler(local), cells=cells)
    clocks = m32["clocks"]
    ms32 = max_over_ranks(m32["ms"]) / args.steps
    value = ranks.job_rate(dof_step, ms32 * 1e-3)
    m32["solver"].close()  # free its scratch; the final state Q stays

    # --- FP32 flux with FP64 stage arithmetic ---
    ms_s = m_s = None
    if not args.no_stage64:
        m_s = run_leg(torch, api, api.DGHGKS_FP32_STAGE64, Q0, dt, args.warmup, args.steps, barrier, cells=cells)
        ms_s = max_over_ranks(m_s["ms"]) / args.steps
        m_s["solver"].close()

    # --- FP64 on the same state ---
    k64 = args.fp64_steps if args.fp64_steps is not None else args.steps
    m64 = run_leg(torch, api, api.DGHGKS_FP64, Q0, dt, args.warmup, k64, barrier, prof_steps=1, cells=cells)
    ms64 = max_over_ranks(m64["ms"]) / k64
    value64 = ranks.job_rate(dof_step, ms64 * 1e-3)

    # --- errors of the FP32 paths against FP64 after the same steps (when the step counts agree) ---
    s64 = m64["solver"]
    err = {"steps_compared": args.warmup + args.steps if k64 == args.steps else None}
    l2_change = s64.l2_diff(m64["Q"], Q0, 0) if k64 == args.steps else None
    for tag, m in (("fp32", m32), ("fp32_stage64", m_s)):
        if m is None:
            continue
        e = {}
        if k64 == args.steps:
            e["l2_rho_vs_fp64"] = s64.l2_diff(m["Q"], m64["Q"], 0)
            e["l2_rhoE_vs_fp64"] = s64.l2_diff(m["Q"], m64["Q"], 4)
            e["l2_rho_change_over_run"] = l2_change
            e["ratio_rho"] = e["l2_rho_vs_fp64"] / l2_change
        dek = [abs(a - b) / abs(b) for a, b in zip(m["ek"], m64["ek"])]
        e["ek_rel_diff_max"] = max(dek)
        e["ek_decay_rel_diff"] = (abs((m["ek"][-1] - m["ek"][0]) - (m64["ek"][-1] - m64["ek"][0])) /
                                  abs(m64["ek"][-1] - m64["ek"][0])
                                  if k64 == args.steps and m64["ek"][-1] != m64["ek"][0] else None)
        err[tag] = e
    err["ek_history_fp64"] = m64["ek"]
    s64.close()
    m64["solver"] = None
    if args.long_error_steps > 0:
        err["long_run"] = long_run_error(torch, api, args.long_error_n, args.long_error_steps)

    roof = roofline_entry(m32["prof"], 1, n, rates, clocks)
    roof64 = roofline_entry(m64["prof"], 0, n, rates, None)
    roof_s = roofline_entry(m_s["prof"], 2, n, rates, None) if m_s is not None else None

    # --- end to end through the C ABI with host buffers (FP32-mixed) ---
    host = torch.empty(Q0.shape, dtype=torch.float64, pin_memory=True)
    host.copy_(Q0)
    Qh = host.numpy()
    s_e2e = api.Solver((n, n, n), (-math.pi,) * 3, (math.pi,) * 3, order=ORDER, gamma=GAMMA, mu=MU, Pr=PR,
                       n_q=NQ, precision=api.DGHGKS_FP32_MIXED)
    s_e2e.run_host(Qh, dt, 1)  # allocates the device state, warms up
    host.copy_(Q0)
    barrier()
    t0 = time.perf_counter()
    ek_e2e = s_e2e.run_host(Qh, dt, args.steps)
    el = max_over_ranks(time.perf_counter() - t0)
    state_bytes = Q0.numel() * 8
    e2e = {"value": ranks.job_rate(dof_step * args.steps, el), "unit": UNIT,
           "h2d_bytes_per_step": state_bytes / args.steps,
           "d2h_bytes_per_step": (state_bytes + 8 * args.steps) / args.steps,
           "api": "dghgks_run_host (H2D of the state, K steps with E_k read back after each, D2H of the state)",
           "ek_last": float(ek_e2e[-1])}
    s_e2e.close()
    del host

    adj = run_adjoint(torch, api, args.adjoint_n, args.adjoint_steps) if args.adjoint_n > 0 else None

    # --- CPU baseline: the oracle on 9^3 boxes of the workload (2 steps each), and BASELINE config 1 ---
    cpu = None
    if do_cpu:
        boxes = [box_of(Q0, n, c) for c in cells]
        want, sec, threads = oracle_boxes(boxes, n, dt)
        cfg1_rate, cfg1_s, cfg1_steps = oracle_config1()
        nb = len(cells)
        cpu = {"value": nb * 9 ** 3 * 50 * 2 * 2 / sec, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"oracle (FP64) stepping {nb} periodic 9^3 boxes cut from the {n}^3 workload around sampled "
                         f"cells, 2 S2O4 steps each, {sec:.1f} s; DOF-stage-updates/s = boxes x 729 x 50 x 2 stages x "
                         f"2 steps / time",
               "config1_full_run": {"value": cfg1_rate, "seconds": cfg1_s, "steps": cfg1_steps,
                                    "workload": "3D density advection 8^3 P1, n_q = 2, S2O4 to t = 0.1"}}
        if args.cpu_config2:
            c2_rate, c2_s = oracle_config2()
            cpu["config2_full_run"] = {"value": c2_rate, "seconds": c2_s, "steps": 2,
                                       "workload": "Taylor-Green 64^3 P2, n_q = 3, dt from CFL 0.15, 2 S2O4 steps"}
        # error of each GPU path against the oracle at the box centres after 2 steps (the 9^3 box holds every
        # cell a centre depends on after 4 stages, so the oracle's centre values are those of the full grid)
        Q0c = torch.stack([Q0[:, :, k, j, i] for (i, j, k) in cells]).cpu().numpy()
        w = np.array([(2 * a + 1) * (2 * b + 1) * (2 * c + 1) for (a, b, c) in
                      ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0),
                       (1, 0, 1), (0, 1, 1))], dtype=float)
        rms = lambda d: float(np.sqrt(np.mean(np.sum(d[:, 0, :] ** 2 / w, axis=1))))  # density, cell-mean L2
        vo = {"cells": nb, "steps": 2, "rms_rho_change": rms(want - Q0c)}
        for tag, m in (("fp64", m64), ("fp32", m32), ("fp32_stage64", m_s)):
            if m is None or m["centres"] is None:
                continue
            d = m["centres"] - want
            vo[tag] = {"rms_rho_err": rms(d), "ratio_rho": rms(d) / vo["rms_rho_change"],
                       "max_abs_err_per_var": np.abs(d).max(axis=(0, 2)).tolist()}
        err["vs_oracle"] = vo

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-mixed (f32 flux/quadrature/projection/stage increments, f64 state "
                                          "accumulation + reductions)",
            "data": "synthetic", "config": workload_config(n, dt),
            "timing": "one dghgks_steps call of K steps (CUDA-graph replay), CUDA events on the stream; per-kernel "
                      "times from a separate profiled pass",
            "fp64": {"value": value64, "unit": UNIT, "ms_per_step": ms64, "steps": k64, "dtype": "f64",
                     "roofline": roof64},
            "fp32_stage64": (None if m_s is None else
                             {"value": ranks.job_rate(dof_step, ms_s * 1e-3), "unit": UNIT, "ms_per_step": ms_s,
                              "dtype": "f32 flux/quadrature/projection, f64 M^-1 + S2O4 combination",
                              "roofline": roof_s}),
            "error": err, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": m32["launches"],
            "pipe_rates": rates,
            "adjoint": adj,
            # companion metric: gas-kinetic flux evaluations (face and cell Gauss points, both stages;
            # one face point counts once, with both of its time integrals)
            "flux_evaluations_per_s": {"fp32_mixed": ranks.job_rate(flux_step, ms32 * 1e-3),
                                       "fp64": ranks.job_rate(flux_step, ms64 * 1e-3)},
        }
        print(json.dumps(line), flush=True)
    ranks.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
