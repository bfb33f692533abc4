"""CPU-side checks of the C-ABI library: it loads, exports every symbol the
header declares, and its host-only Gauss rule matches numpy (no GPU needed)."""
import os
import re

import numpy as np
import numpy.polynomial.legendre as npl
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2202_13821_b300 import api, build

    build.build()
    return api.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dghgks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dghgks_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dghgks_init", "dghgks_residual", "dghgks_step", "dghgks_totals", "dghgks_kinetic_energy",
                 "dghgks_last_error", "dghgks_destroy", "dghgks_run_host", "dghgks_status"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2202_13821_b300 import api

    assert set(declared_functions()) <= set(api.exported_symbols())


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_device_gauss_rule_matches_numpy(lib, n):
    from paper_2202_13821_b300 import api

    x, w = api.dghgks_gauss_rule(n)
    xr, wr = npl.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=2e-16)
    np.testing.assert_allclose(w, wr / 2, rtol=2e-16, atol=2e-16)


def test_init_rejects_bad_arguments_without_gpu(lib):
    from paper_2202_13821_b300 import api

    # argument checks run before any CUDA call
    with pytest.raises(api.DghgksError) as e:
        api.dghgks_init((0, 4, 4), (0, 0, 0), (1, 1, 1), 2, 1.4, 0.0, 1.0)
    assert e.value.code == -1
    with pytest.raises(api.DghgksError) as e:
        api.dghgks_init((4, 4, 4), (0, 0, 0), (1, 1, 1), 5, 1.4, 0.0, 1.0)
    assert e.value.code == -2
    with pytest.raises(api.DghgksError) as e:
        api.dghgks_init((4, 4, 4), (0, 0, 0), (1, 1, 1), 2, 1.4, -1.0, 1.0)
    assert e.value.code == -1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2202_13821_b300 import api

    monkeypatch.setattr(api, "_lib", None)
    monkeypatch.setattr(api, "_SO", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        api.load()


def _static_call(lib, n, order, nq=0, precision=0, nodes=None):
    """dghgks_residual_static with placeholder device pointers: every case below is rejected by
    the argument checks, which run before the first CUDA call, so the pointers are never used."""
    import ctypes

    from paper_2202_13821_b300 import api

    m = api.Mesh()
    m.nx, m.ny, m.nz = n
    keep = []
    for d in range(3):
        m.lo[d], m.hi[d], m.periodic[d] = 0.0, 1.0, 1
        if nodes is not None:
            arr = (ctypes.c_double * (n[d] + 1))(*np.linspace(0.0, 1.0, n[d] + 1) ** 1.1)
            keep.append(arr)
            m.nodes[d] = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
    o = api.Opts(nq, precision, 0.0)
    fake = ctypes.c_void_p(0x1000)
    return lib.dghgks_residual_static(ctypes.byref(m), order, 1.4, 0.0, 1.0, ctypes.byref(o), fake, 1e-3,
                                      ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000), None)


def test_static_residual_rejects_unsupported_cases_without_gpu(lib):
    # order 3, an n_q the static path does not carry, a rectilinear mesh: DGHGKS_EUNSUP
    assert _static_call(lib, (4, 4, 4), 3, 3) == -2
    assert _static_call(lib, (4, 4, 4), 1, 3) == -2
    assert _static_call(lib, (4, 4, 4), 2, 3, nodes=True) == -2
    # the FP32-flux / FP64-stage precision is a context option only: DGHGKS_EARG
    assert _static_call(lib, (4, 4, 4), 2, 3, precision=2) == -1
    # face moments above the fixed 16 MiB scratch: DGHGKS_ESCRATCH (P2 FP64: 1440 B per cell)
    assert _static_call(lib, (32, 32, 32), 2, 3) == -6
    assert _static_call(lib, (64, 64, 64), 1, 2, precision=1) == -6
