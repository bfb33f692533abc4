"""The bounded shared-memory barrier wait of the persistent cell kernel gives up and reports.

The cell kernel orders its tile loop with mbarriers; every wait on one is bounded (2 s of global
time) and, when it gives up, sets bit 1 of the device error flag and lets the kernel return, so a
barrier that never completes cannot hang the GPU.  tests/native/mbar_timeout_check.cu runs the same
wait on a barrier that never completes (one of two expected arrivals) and on one that completes
(control), then launches a third kernel: the first must time out in about 2 s with the flag set,
the second succeed at once, and the context stay usable.  No fault, trap or unbounded wait is
involved.
"""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.gpu
def test_bounded_barrier_wait_times_out_and_reports(tmp_path):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_13821_b300 import build

    exe = str(tmp_path / "mbar_timeout_check")
    subprocess.run([build.nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "paper_2202_13821_b300", "csrc"),
                    "-o", exe, os.path.join(HERE, "native", "mbar_timeout_check.cu")], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    f = r.stdout.split()
    assert f[1:4] == ["2", "0", "7"]
