#!/usr/bin/env python
"""Throughput of the DG-HGKS per-stage residual on one B300 (or N replicas).

Workload: Taylor-Green vortex (Sec. 5.3 of arXiv:2202.13821) on a periodic
256^3 uniform grid, P2 elements (10 modes x 5 variables per cell), 3x3 face and
3^3 cell Gauss points, Re = 1600, Ma = 0.1, Pr = 0.72, gamma = 1.4, dt from
CFL 0.15.  A step is one S2O4 time step = two full residual stages over the
whole grid (3 face launches + 1 cell launch per stage).

Metric: DOF-stage-updates/s = 5 * N_modes * N_cells * 2 / (time per step),
whole job (sum over ranks).  The headline value is the FP32-mixed path (flux
and quadrature in FP32, stage accumulation and reductions in FP64); the FP64
path is measured on the same state and reported beside it, with the error
of FP32-mixed against FP64 (L2 density difference, relative kinetic-energy
history difference).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the method written plainly from
the paper) on a bounded sample of cells of the same workload.
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
FP32_PEAK_NOTE = "148 SMs x 128 FP32 lanes x 2 flop x sm_max_mhz"
FP64_PEAK_TFLOPS = 1.25  # B300 nominal FP64 (non-tensor) rate


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_CELLS_1D, help="cells per direction")
    ap.add_argument("--fp64-steps", type=int, default=None, help="timed FP64 steps (default: --steps)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU-baseline sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--adjoint-n", type=int, default=64, help="cells per direction of the adjoint leg (0: skip)")
    ap.add_argument("--adjoint-steps", type=int, default=4, help="checkpointed steps of the adjoint leg")
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
def oracle_sample(n, seconds, reps=1, Q=None):
    """Time the oracle's residual on a bounded sample of cells of the workload.

    Returns (DOF-stage-updates/s per repetition, threads, sample description)."""
    import numpy as np

    import oracle
    from paper_2202_13821_b300 import inputs

    oracle.build()
    if Q is None:
        Q = inputs.tgv_state(n, ORDER, device="cpu").numpy()
    dt = inputs.tgv_dt(n, ORDER)
    pb = oracle.Problem(order=ORDER, nq=NQ, n=(n, n, n), lo=(-math.pi,) * 3, hi=(math.pi,) * 3, mu=MU, Pr=PR,
                        gamma=GAMMA)
    rng = np.random.default_rng(0)
    # calibrate on 64 cells, then size the sample to the time budget
    cells = rng.integers(0, n ** 3, 64)
    t0 = time.perf_counter()
    oracle.residual_cells(pb, Q, dt, cells)
    per_cell = (time.perf_counter() - t0) / len(cells)
    ncells = int(max(64, min(n ** 3, seconds / max(per_cell, 1e-9) / reps)))
    cells = rng.integers(0, n ** 3, ncells)
    rates = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.residual_cells(pb, Q, dt, cells)
        el = time.perf_counter() - t0
        rates.append(ncells * 5 * 10 / el)  # one stage of 50 DOFs per cell residual
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"oracle residual (FP64, L and L_t, each cell evaluating its own six faces) of {ncells} random cells "
              f"of the {n}^3 workload, {reps} repetition(s); DOF-stage-updates/s = cells x 50 / time")
    return rates, threads, sample


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    n = args.n
    from paper_2202_13821_b300 import inputs

    dt = inputs.tgv_dt(n, ORDER)
    budget = max(4.0, min(15.0, 100.0 / max(1, args.steps + args.warmup)))
    rates, threads, sample = oracle_sample(n, budget, reps=args.steps + args.warmup)
    timed = rates[args.warmup:] or rates
    value = statistics.mean(timed)  # rank 0 alone runs the CPU oracle
    ms_per_step = 5 * 10 * n ** 3 * 2 / value * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(n, dt),
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


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def run_leg(torch, api, precision, Q0, dt, warmup, steps, barrier, clock=None):
    s = api.Solver((Q0.shape[4], Q0.shape[3], Q0.shape[2]), (-math.pi,) * 3, (math.pi,) * 3, order=ORDER,
                   gamma=GAMMA, mu=MU, Pr=PR, n_q=NQ, precision=precision)
    Q = Q0.clone()
    ek = [s.kinetic_energy(Q)]
    for _ in range(warmup):
        s.step(Q, dt)
        ek.append(s.kinetic_energy(Q))
    s.status()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    launches0 = s.launches
    s.profile(True)
    if clock is not None:
        clock.start()
    e0.record(stream)
    s.steps(Q, dt, steps)  # FP32-mixed: the state rounded to FP32 carries over between the steps
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clock.stop() if clock is not None else None
    barrier()
    ms = e0.elapsed_time(e1)
    prof = s.profile_read()
    s.profile(False)
    launches = s.launches - launches0
    s.status()
    ek.append(s.kinetic_energy(Q))
    return {"solver": s, "Q": Q, "ms": ms, "prof": prof, "launches": launches, "ek": ek, "clocks": clocks}


def algorithmic_bytes(kernel, precision):
    """HBM bytes per cell of one launch, mean of the two stages of a step (P2: 50 state coefficients,
    60 face moments per face): each value read or written once, neighbours' data counted once.

    k_face stage 1 reads the state and writes the F and F_t moments; stage 2 reads Q* (flux
    precision) and writes the F_t moments.  k_cell stage 1 reads the state and the moments of its
    faces and writes Q* and inc; stage 2 reads Q*, inc, the F_t moments and the FP64 state and
    writes the state.  FP32-mixed steps read the state rounded to FP32 at stage 1, which stage 2
    writes besides the FP64 state (the rounding kernel at the start of a call is not counted)."""
    r = 4 if precision == 1 else 8
    coef, mom = 5 * 10, 10 * 6
    state_in = coef * r  # FP32 copy (FP32-mixed) or the FP64 state
    copy_out = coef * 4 if precision == 1 else 0
    if kernel == "k_face":
        s1 = state_in + mom * r
        s2 = coef * r + mom // 2 * r
    else:
        s1 = state_in + 3 * mom * r + 2 * coef * r  # six faces, each shared by two cells
        s2 = 2 * coef * r + 3 * (mom // 2) * r + 2 * coef * 8 + copy_out
    return (s1 + s2) / 2


def roofline_entry(prof, precision, n, peaks, clocks):
    from paper_2202_13821_b300 import build

    oc = build.opcounts(ORDER, NQ, PR != 1.0)
    face_ms = sum(prof[k][0] for k in ("face_x", "face_y", "face_z"))
    face_n = sum(prof[k][1] for k in ("face_x", "face_y", "face_z"))
    cell_ms = prof["cell_stage1"][0] + prof["cell_stage2"][0]
    cell_n = prof["cell_stage1"][1] + prof["cell_stage2"][1]
    pts = n ** 3 * NQ * NQ  # face points of one face launch (one normal direction)
    cpts = n ** 3 * NQ ** 3
    # a step launches each kernel once per stage; the stage-2 launches need
    # F_t only (the counts keep only the operations F_t depends on), so the
    # per-launch figure is the mean of the two
    face_flops = pts * (oc["face_point"]["total_flops"] + oc["face_point"]["total_flops_ft"]) // 2
    cell_flops = cpts * (oc["cell_point"]["total_flops"] + oc["cell_point"]["total_flops_ft"]) // 2
    kernels = {
        "k_face": {"launches": face_n, "avg_ms": face_ms / max(face_n, 1), "flops_per_launch": face_flops},
        "k_cell": {"launches": cell_n, "avg_ms": cell_ms / max(cell_n, 1), "flops_per_launch": cell_flops},
    }
    dom = max(kernels, key=lambda k: kernels[k]["avg_ms"] * kernels[k]["launches"])
    kd = kernels[dom]
    achieved = kd["flops_per_launch"] / (kd["avg_ms"] * 1e-3) / 1e12
    smax = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2032.0)
    if precision == 1:
        peak = 148 * 128 * 2 * smax * 1e6 / 1e12
        peak_src = f"derived: {FP32_PEAK_NOTE} = {peak:.1f} TFLOP/s (FP32)"
    else:
        peak = FP64_PEAK_TFLOPS
        peak_src = "B300 FP64 1.25 TFLOP/s nominal (a DFMA loop measured 0.95 on a B300)"
    traffic, traffic_src = profiled_traffic(dom, n) if precision == 1 else (None, None)
    return {
        "bound": "alu", "kernel": dom, "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
        "frac": round(achieved / peak, 4), "traffic": traffic, "traffic_source": traffic_src,
        "traffic_algorithmic": n ** 3 * algorithmic_bytes(dom, precision),
        "peak_source": peak_src,
        "algorithmic_flops": "value-numbered op count per point x points per launch, mean of the two stages "
                             f"(face point {oc['face_point']['total_flops']} / {oc['face_point']['total_flops_ft']} "
                             f"F_t only; cell point {oc['cell_point']['total_flops']} / "
                             f"{oc['cell_point']['total_flops_ft']} F_t only)",
        "kernels": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                    for k, v in kernels.items()},
    }


def run_adjoint(torch, api, n, nsteps):
    """Gradient of the final E_k w.r.t. the initial state and mu over nsteps checkpointed FP64 steps
    (Taylor-Green P2): time per forward and per adjoint step, checkpoint and device memory."""
    from paper_2202_13821_b300 import autograd, inputs

    dt = inputs.tgv_dt(n, ORDER)
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
    out = {"workload": f"Taylor-Green {n}^3 P2 FP64, {nsteps} checkpointed S2O4 steps, dE_k/d(Q0, mu)",
           "forward_ms_per_step": 1e3 * (t1 - t0) / nsteps, "adjoint_ms_per_step": 1e3 * (t2 - t1) / nsteps,
           "checkpoint_bytes_per_step": state, "checkpoint_bytes_100_steps": 100 * state,
           "device_bytes_after_forward": free0 - free1, "dJ_dmu": float(mu.grad.item()),
           "grad_norm": float(Q0.grad.norm().item())}
    s.close()
    del Q0, mu, J
    torch.cuda.empty_cache()
    return out


def run_ours(args):
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
    peaks = measured_peaks()

    # --- FP32-mixed (headline) ---
    m32 = run_leg(torch, api, api.DGHGKS_FP32_MIXED, Q0, dt, args.warmup, args.steps, barrier, ClockSampler(local))
    clocks = m32["clocks"]
    ms32 = max_over_ranks(m32["ms"]) / args.steps
    value = ranks.job_rate(dof_step, ms32 * 1e-3)
    m32["solver"].close()  # free its scratch; the final state Q stays

    # --- FP64 on the same state ---
    k64 = args.fp64_steps if args.fp64_steps is not None else args.steps
    m64 = run_leg(torch, api, api.DGHGKS_FP64, Q0, dt, args.warmup, k64, barrier)
    ms64 = max_over_ranks(m64["ms"]) / k64
    value64 = ranks.job_rate(dof_step, ms64 * 1e-3)

    # --- error of FP32-mixed against FP64 after the same steps (when the step counts agree) ---
    s64 = m64["solver"]
    err = {"steps_compared": args.warmup + args.steps if k64 == args.steps else None}
    if k64 == args.steps:
        l2 = s64.l2_diff(m32["Q"], m64["Q"], 0)
        l2E = s64.l2_diff(m32["Q"], m64["Q"], 4)
        l2_change = s64.l2_diff(m64["Q"], Q0, 0)
        err.update({"l2_rho_fp32_vs_fp64": l2, "l2_rhoE_fp32_vs_fp64": l2E,
                    "l2_rho_change_over_run": l2_change})
    s64.close()
    m64["solver"] = None
    ek32, ek64 = m32["ek"], m64["ek"]
    dek = [abs(a - b) / abs(b) for a, b in zip(ek32, ek64)]
    err["ek_rel_diff_max"] = max(dek)
    err["ek_history_fp64"] = ek64
    err["ek_decay_rel_diff"] = (abs((ek32[-1] - ek32[0]) - (ek64[-1] - ek64[0])) / abs(ek64[-1] - ek64[0])
                                if k64 == args.steps and ek64[-1] != ek64[0] else None)

    roof = roofline_entry(m32["prof"], 1, n, peaks, clocks)
    roof64 = roofline_entry(m64["prof"], 0, n, peaks, None)

    # --- end to end through the C ABI with host buffers (FP32-mixed) ---
    e2e = None
    if True:  # every rank measures its own replica end to end
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

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rates, threads, sample = oracle_sample(n, args.cpu_seconds, Q=Q0.cpu().numpy())
        cpu = {"value": rates[0], "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-mixed (f32 flux/quadrature, f64 stage + reductions)",
            "data": "synthetic", "config": workload_config(n, dt),
            "fp64": {"value": value64, "unit": UNIT, "ms_per_step": ms64, "steps": k64, "dtype": "f64",
                     "roofline": roof64},
            "error": err, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": m32["launches"],
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
