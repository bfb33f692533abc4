"""Taylor-Green vortex histories in the paper's setting (Sec. 5.3: P2, n_q = k = 2, Pr = 1,
Re = 1600, Ma = 0.1), 64^3 cells to t = 10, FP32-mixed path, through the C ABI.

* E_k(0) = 1/8 (closed form of the initial field; cell-centre sampling at 64^3);
* E_k decreases monotonically;
* while the flow is smooth and resolved (t <= 3) the kinetic-energy dissipation
  eps(E_k) = -dE_k/dt (central differences, as in the paper) equals the enstrophy
  form eps(zeta) = 2 mu / (rho0 Omega) int 1/2 rho |curl U|^2 of the incompressible
  limit, computed independently from the element gradients;
* eps(E_k) peaks during the vortex breakdown, between t = 7 and t = 10.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def history():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_13821_b300 import api, build, tgv

    build.build()
    api.load()
    return tgv.run(n=64, order=2, t_end=10.0, precision=1)


def test_initial_kinetic_energy(history):
    assert abs(history["ek"][0] - 0.125) < 1e-3


def test_kinetic_energy_decreases(history):
    assert np.all(np.diff(history["ek"]) < 0)


def test_dissipation_equals_enstrophy_form_while_resolved(history):
    t, eek, ez = history["t"], history["eps_ek"], history["eps_zeta"]
    sel = (t >= 0.5) & (t <= 3.0)
    rel = np.abs(ez[sel] / eek[sel] - 1.0)
    print(f"max |eps(zeta)/eps(E_k) - 1| for t in [0.5, 3]: {rel.max():.3f}")
    assert rel.max() < 0.06


def test_dissipation_peak_during_breakdown(history):
    i = int(np.nanargmax(history["eps_ek"]))
    print(f"max eps(E_k) = {history['eps_ek'][i]:.5f} at t = {history['t'][i]:.2f}")
    assert 7.0 <= history["t"][i] <= 10.0
