"""The hand-written reverse mode of the point fluxes (csrc/gks_point_adj.cuh, used by the adjoint
kernels) against forward-mode dual numbers through the forward flux templates, compiled for the
host: every component of J^T w, for random physical states and cotangents, Pr = 1 and 0.72,
mu > 0 and mu = 0 with tau_eps > 0, for the full sweeps and for the F_t-only sweeps of the adjoint's
second stage (tests/native/point_vjp_check.cpp)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_point_flux_vjp_matches_dual_numbers(tmp_path):
    exe = str(tmp_path / "point_vjp_check")
    cuda_inc = "/usr/local/cuda/include"
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wno-unknown-pragmas", "-I", cuda_inc, "-I",
                    os.path.join(ROOT, "paper_2202_13821_b300", "csrc"), "-o", exe,
                    os.path.join(HERE, "native", "point_vjp_check.cpp")], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
    worst = float(r.stdout.strip().splitlines()[-1].split()[-1])
    assert worst < 1e-11
