"""dghgks_residual_static: the residual for callers that cannot allocate.

Callers inside another framework's memory plan, real-time loops that forbid
allocation after start-up, or code that must not trigger cudaFree's device
synchronisation cannot create a context (dghgks_init allocates).  This entry
point keeps its scratch in a fixed device array instead.  The test calls it
twice in a row through the C ABI for every supported layout (P1 with n_q = 2,
P2 with n_q = 2 and 3) in FP64 and FP32-mixed, on a grid whose x extent is
not a multiple of the face kernel's 32-face tiles, and requires both results
to equal the context-based dghgks_residual bit for bit: the same kernels run
on the same inputs.  The tolerance of the other residual tests (relative
1e-11) is asserted as well, so that a mismatch also reports its size.  It also
checks that an oversized problem is refused before any GPU work.  This file is
collected last so that a failure here cannot hide the other tests.
"""
import math

import numpy as np
import pytest

RTOL = 1e-11


def per_var_err(a, b):
    a = np.asarray(a).reshape(5, -1)
    b = np.asarray(b).reshape(5, -1)
    scale = np.abs(b).max(axis=1)
    return np.abs(a - b).max(axis=1) / np.where(scale > 0, scale, 1.0)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("order,nq", [(1, 2), (2, 2), (2, 3)])
def test_static_residual_matches_context_residual_twice(order, nq, precision):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_13821_b300 import api, build, inputs

    build.build()
    n, lo, hi = (37, 9, 7), (-math.pi,) * 3, (math.pi,) * 3
    kw = dict(order=order, gamma=1.4, mu=1 / 1600, Pr=0.72)
    Q = inputs.tgv_state(n, order, perturb=1e-3, device="cuda")
    s = api.Solver(n, lo, hi, n_q=nq, precision=precision, **kw)
    L0, Lt0 = s.residual(Q, 1.3e-3)
    torch.cuda.synchronize()
    s.close()
    for _ in range(2):
        L = torch.full_like(Q, float("nan"))
        Lt = torch.full_like(Q, float("nan"))
        api.dghgks_residual_static(n, lo, hi, kw["order"], kw["gamma"], kw["mu"], kw["Pr"], Q, 1.3e-3, L, Lt,
                                   n_q=nq, precision=precision)
        for got, want in ((L, L0), (Lt, Lt0)):
            assert per_var_err(got.cpu().numpy(), want.cpu().numpy()).max() < RTOL
            assert torch.equal(got, want)


@pytest.mark.gpu
def test_static_residual_rejects_oversized_problem():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_13821_b300 import api, build

    build.build()
    n = (32, 32, 32)  # P2 FP64 face moments: 32768 cells x 1440 B > 16 MiB
    Q = torch.zeros((5, 10) + n, dtype=torch.float64, device="cuda")
    L, Lt = torch.zeros_like(Q), torch.zeros_like(Q)
    with pytest.raises(api.DghgksError) as e:
        api.dghgks_residual_static(n, (0,) * 3, (1,) * 3, 2, 1.4, 0.0, 1.0, Q, 1e-3, L, Lt, n_q=3)
    assert e.value.code == -6
