"""Properties of the CUDA path that hold at any size (GPU, through the C ABI).

* optimal order k+1 on the 3D density advection (Sec. 5.1) against its exact
  solution, on finer grids than the oracle reaches, on uniform and on the
  mapped non-uniform mesh of the same section;
* conservation of mass, momentum and energy to rounding over many steps
  (FP64 rounding on the FP64 path, FP32 rounding of the per-step increments
  on the FP32-mixed path);
* uniform flow preserved; bitwise determinism run to run;
* graph replay (dghgks_steps) bitwise equal to single steps;
* FP32-mixed error against the FP64 path on the Taylor-Green vortex, stated
  and bounded;
* error paths: non-physical state -> DGHGKS_EPHYS via the device flag (the
  context stays usable), bad arguments -> DGHGKS_EARG.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def api(torch):
    from paper_2202_13821_b300 import api, build

    build.build()
    api.load()
    return api


TGV = dict(lo=(-math.pi,) * 3, hi=(math.pi,) * 3)


def advection_error(api, torch, order, n, T=0.1, mapped=False):
    import oracle
    from paper_2202_13821_b300 import inputs

    nodes = (inputs.mapped_nodes(n),) * 3 if mapped else None
    dt = inputs.advection_dt(n, T=T)
    if mapped:  # CFL on the smallest cell
        dt = T / math.ceil(T / (dt * min(np.diff(nodes[0])) / (2.0 / n)))
    s = api.Solver((n,) * 3, (0,) * 3, (2,) * 3, order=order, n_q=order + 1, tau_eps=0.01, nodes=nodes)
    pb = oracle.Problem(order=order, nq=order + 1, n=(n,) * 3, tau_eps=0.01, nodes=nodes)
    Q = torch.from_numpy(oracle.project(pb, oracle.IC_ADVECTION, (0.2, 0.0))).cuda()
    s.step(Q, dt, round(T / dt))
    s.status()
    return oracle.density_errors(pb, Q.cpu().numpy(), oracle.IC_ADVECTION, (0.2, T))


@pytest.mark.parametrize("order,sizes,lo_order", [(1, (16, 32), 1.9), (2, (8, 16), 2.85), (3, (8, 16), 3.6)])
def test_advection_convergence_order(torch, api, order, sizes, lo_order):
    e = [advection_error(api, torch, order, n) for n in sizes]
    orders = np.log2(e[0] / e[1])
    assert orders[0] > lo_order and orders[1] > lo_order, orders


@pytest.mark.parametrize("order,sizes,lo_order", [(2, (8, 16), 2.85), (3, (8, 16), 3.6)])
def test_advection_convergence_order_mapped_mesh(torch, api, order, sizes, lo_order):
    """Sec. 5.1 non-uniform mesh x = xi + 0.05 sin(pi xi) (Tables tab-3d-3, tab-3d-4: L2 orders
    3.70 (P2) and 4.22 (P3) at 8^3 -> 16^3)."""
    e = [advection_error(api, torch, order, n, mapped=True) for n in sizes]
    orders = np.log2(e[0] / e[1])
    print(f"P{order} mapped-mesh advection errors {e[0]} -> {e[1]}, orders {orders}")
    assert orders[0] > lo_order and orders[1] > lo_order, orders


def vortex_errors_gpu(api, torch, order, n, T=1.0, cfl=0.1):
    import oracle

    h = 10.0 / n
    dt0 = cfl * h / (math.sqrt(2) + 1.0 + math.sqrt(1.4))
    ns = math.ceil(T / dt0)
    lo, hi = (0.0, 0.0, 0.0), (10.0, 10.0, h)
    s = api.Solver((n, n, 1), lo, hi, order=order, n_q=order + 1)
    pb = oracle.Problem(order=order, nq=order + 1, n=(n, n, 1), lo=lo, hi=hi)
    Q = torch.from_numpy(oracle.project(pb, oracle.IC_VORTEX, (5.0, 0.0, 5.0, 5.0, 10.0, 10.0))).cuda()
    s.step(Q, T / ns, ns)
    s.status()
    return oracle.density_errors(pb, Q.cpu().numpy(), oracle.IC_VORTEX, (5.0, T, 5.0, 5.0, 10.0, 10.0))


@pytest.mark.parametrize("order,lo_order", [(2, 2.6), (3, 3.6)])
def test_isotropic_vortex_order(torch, api, order, lo_order):
    """Nonlinear accuracy test of Sec. 5.1 (isotropic vortex moving with (1, 1)), one cell in z.
    The paper's L2 orders at 20^2 -> 40^2 are 2.76 (P2) and 4.33 (P3); the cell-average error
    e_c converges faster than k+1 (super-convergence, Tables iso-vor-1/2)."""
    e0, e1 = vortex_errors_gpu(api, torch, order, 20), vortex_errors_gpu(api, torch, order, 40)
    orders = np.log2(e0 / e1)
    print(f"P{order} vortex errors {e0} -> {e1}, orders {orders}")
    assert orders[1] > lo_order, orders
    assert orders[2] > order + 1, orders


def test_conservation_over_steps(torch, api):
    from paper_2202_13821_b300 import inputs

    for prec in (0, 1, 2):
        s = api.Solver((24, 20, 16), **TGV, order=2, mu=1 / 1600, Pr=0.72, n_q=3, precision=prec)
        Q = inputs.tgv_state((24, 20, 16), 2, perturb=1e-3, device="cuda")
        t0 = s.totals(Q)
        s.step(Q, 5e-3, 10)
        s.status()
        t1 = s.totals(Q)
        scale = np.array([1.0, 1.0, 1.0, 1.0, 180.0]) * (2 * math.pi) ** 3
        # FP64: every face moment enters its two cells with opposite signs and the
        # sums are FP64.  FP32-mixed: the same antisymmetry, but each cell's stage
        # increment is rounded to FP32 before the FP64 accumulation, so totals
        # move by FP32 rounding of the increments (~1e-7 of |dt L| per cell).
        # FP32 flux with FP64 stage arithmetic: the FP32 face moments are summed
        # in FP64 (exactly, for a few terms) and the increments stay FP64, so the
        # totals hold as in FP64.
        tol = 1e-10 if prec == 1 else 1e-13
        assert np.all(np.abs(t1 - t0) <= tol * scale), (prec, (t1 - t0) / scale)


def test_uniform_flow_preserved(torch, api):
    for prec in (0, 1, 2):
        s = api.Solver((8, 9, 10), (0,) * 3, (1,) * 3, order=2, mu=1e-3, Pr=0.72, precision=prec)
        Q = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
        rho, u, p = 1.3, (0.2, -0.4, 0.7), 2.0
        Q[0, 0], Q[1, 0], Q[2, 0], Q[3, 0] = rho, rho * u[0], rho * u[1], rho * u[2]
        Q[4, 0] = p / 0.4 + 0.5 * rho * sum(x * x for x in u)
        dt = 1e-2
        L, Lt = s.residual(Q, dt)
        if prec == 0:
            assert float(L.abs().max()) < 1e-12 and float(Lt.abs().max()) < 1e-11
        else:
            # FP32: the face and interior fluxes of the uniform state agree to rounding, so L is
            # a few ulps of the largest flux component over the smallest cell width (times the
            # basis factor 3 of the linear modes); F_t = 4 (I(dt) - 2 I(dt/2)) / dt^2 cancels
            # the free-transport and equilibrium terms with the fit weight q = 4 x s^2 / dt
            # (x = tau / dt, s = 1 - exp(-dt / (2 tau))), which multiplies that rounding
            eps, fmax = 2.0 ** -24, 0.7 * (Q[4, 0, 0, 0, 0].item() + p)  # energy flux u_z (rho E + p)
            h = 1 / 10
            tau = 1e-3 / p
            x, s_ = tau / dt, 1 - math.exp(-dt / (2 * tau))
            q = 4 * x * s_ * s_ / dt
            tol = 64 * eps * fmax * 3 / h
            assert float(L.abs().max()) < tol and float(Lt.abs().max()) < q * tol


def test_deterministic_and_graph_replay_bitwise(torch, api):
    from paper_2202_13821_b300 import inputs

    for prec in (0, 1, 2):
        s = api.Solver((20, 12, 9), **TGV, order=2, mu=1 / 1600, Pr=0.72, precision=prec)
        Q0 = inputs.tgv_state((20, 12, 9), 2, perturb=1e-3, device="cuda")
        A, B, C = Q0.clone(), Q0.clone(), Q0.clone()
        s.step(A, 4e-3, 3)
        s.step(B, 4e-3, 3)
        s.steps(C, 4e-3, 3)
        s.status()
        assert torch.equal(A, B) and torch.equal(A, C)
        # a new dt re-captures the graph
        D, E = Q0.clone(), Q0.clone()
        s.steps(D, 2e-3, 2)
        s.step(E, 2e-3, 2)
        s.status()
        assert torch.equal(D, E)


def test_fp32_state_copy_stays_within_one_call(torch, api):
    """FP32-mixed dghgks_steps: the steps after the first read the FP32 copy of the state that the
    step before wrote; the first step of every call rounds the FP64 state into it afresh, so a
    state changed between calls is what the next call steps, and a profiled call (launches enqueued
    directly, each recorded) gives the graph replay's result."""
    from paper_2202_13821_b300 import inputs

    s = api.Solver((20, 12, 9), **TGV, order=2, mu=1 / 1600, Pr=0.72, precision=1)
    Q0 = inputs.tgv_state((20, 12, 9), 2, perturb=1e-3, device="cuda")
    Q1 = Q0.clone()
    Q1[0, 0] *= 1.01  # another state: density raised by 1 %
    A = Q0.clone()
    s.steps(A, 4e-3, 3)  # leaves the FP32 copy of A behind
    B, C, D = Q1.clone(), Q1.clone(), Q1.clone()
    s.steps(B, 4e-3, 2)
    s.step(C, 4e-3, 2)
    s.profile(True)
    s.steps(D, 4e-3, 2)
    prof = s.profile_read()
    s.profile(False)
    s.status()
    assert torch.equal(B, C) and torch.equal(B, D)
    assert sum(n for _, n in prof.values()) == 16  # 8 launches per step, all recorded
    assert not torch.equal(A, B)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("order,nq", [(1, 2), (2, 2), (2, 3), (3, 3), (3, 4)])
def test_fp32_steps_with_state_copy_bitwise_every_layout(torch, api, order, nq, precision):
    """dghgks_steps (FP32 contexts: later steps read the FP32 copy of the state written by the step
    before) equals dghgks_step bitwise for every cell-kernel layout: four cells per warp (n_q = 2),
    a warp per cell (n_q = 3) and two warps per cell (n_q = 4), on a ragged grid; FP32-mixed and
    FP32 flux with FP64 stage arithmetic."""
    from paper_2202_13821_b300 import inputs

    n = (19, 6, 5)
    s = api.Solver(n, **TGV, order=order, mu=1 / 1600, Pr=0.72, n_q=nq, precision=precision)
    Q0 = inputs.tgv_state(n, order, perturb=1e-3, device="cuda")
    A, B = Q0.clone(), Q0.clone()
    s.step(A, 3e-3, 3)
    s.steps(B, 3e-3, 3)
    s.status()
    assert torch.equal(A, B)
    assert not torch.equal(A, Q0)


def test_fp32_steps_on_an_8_byte_aligned_state(torch, api):
    """The C ABI takes any contiguous FP64 state: a view that starts one value into its storage (8-byte,
    not 16-byte aligned) steps to the same result as an aligned copy."""
    from paper_2202_13821_b300 import inputs

    n = (12, 5, 4)
    s = api.Solver(n, **TGV, order=2, mu=1 / 1600, Pr=0.72, n_q=3, precision=1)
    Q0 = inputs.tgv_state(n, 2, perturb=1e-3, device="cuda")
    buf = torch.empty(Q0.numel() + 1, dtype=torch.float64, device="cuda")
    V = buf[1:].view(Q0.shape)
    V.copy_(Q0)
    assert V.data_ptr() % 16 == 8
    A = Q0.clone()
    s.steps(A, 3e-3, 2)
    s.steps(V, 3e-3, 2)
    s.status()
    assert torch.equal(A, V)


def test_run_host_matches_device_steps(torch, api):
    """dghgks_run_host (host state in and out, E_k of each step on a second stream beside the next
    step) gives bitwise the state and E_k history of device steps with E_k after each."""
    from paper_2202_13821_b300 import inputs

    n = (24, 20, 16)
    for prec in (0, 1, 2):
        s = api.Solver(n, **TGV, order=2, mu=1 / 1600, Pr=0.72, precision=prec)
        Q0 = inputs.tgv_state(n, 2, perturb=1e-3, device="cuda")
        Qd = Q0.clone()
        ek_dev = []
        for _ in range(11):
            s.step(Qd, 3e-3)
            ek_dev.append(s.kinetic_energy(Qd))
        host = torch.empty(Q0.shape, dtype=torch.float64, pin_memory=True)
        host.copy_(Q0)
        ek_host = s.run_host(host.numpy(), 3e-3, 11)
        s.status()
        assert torch.equal(host.cuda(), Qd)
        assert np.array_equal(ek_host, np.array(ek_dev))


def test_graph_replay_follows_set_mu(torch, api):
    """dghgks_steps after dghgks_set_mu uses the new viscosity (the graph is captured again)."""
    from paper_2202_13821_b300 import inputs

    s = api.Solver((12, 10, 8), **TGV, order=2, mu=1 / 1600, Pr=0.72)
    Q0 = inputs.tgv_state((12, 10, 8), 2, perturb=1e-3, device="cuda")
    A, B = Q0.clone(), Q0.clone()
    s.steps(A, 4e-3, 2)  # capture with the first viscosity
    s.set_mu(1 / 400)
    A = Q0.clone()
    s.steps(A, 4e-3, 2)
    s.step(B, 4e-3, 2)
    s.status()
    assert torch.equal(A, B)


def test_fp32_mixed_error_against_fp64(torch, api):
    """Stated error of the FP32-mixed path on the Taylor-Green vortex (48^3, 10 steps)."""
    from paper_2202_13821_b300 import inputs

    n = 48
    dt = inputs.tgv_dt(n, 2)
    Q0 = inputs.tgv_state(n, 2, device="cuda")
    res = {}
    for prec in (0, 1):
        s = api.Solver((n,) * 3, **TGV, order=2, mu=1 / 1600, Pr=0.72, precision=prec)
        Q = Q0.clone()
        ek = [s.kinetic_energy(Q)]
        for _ in range(10):
            s.step(Q, dt)
            ek.append(s.kinetic_energy(Q))
        s.status()
        res[prec] = (Q, np.array(ek), s)
    s64 = res[0][2]
    l2 = s64.l2_diff(res[1][0], res[0][0], 0)
    change = s64.l2_diff(res[0][0], Q0, 0)
    dek = np.abs(res[1][1] - res[0][1]) / res[0][1]
    decay = abs((res[1][1][-1] - res[1][1][0]) - (res[0][1][-1] - res[0][1][0])) / abs(res[0][1][-1] - res[0][1][0])
    print(f"FP32-mixed vs FP64: L2(rho) {l2:.3e} (change {change:.3e}), E_k rel {dek.max():.2e}, decay rel {decay:.2e}")
    assert dek.max() < 1e-6
    assert decay < 1e-3
    assert l2 < 0.5 * change


def test_fp32_mixed_error_128_cubed(torch, api):
    """The FP32-mixed configuration: Taylor-Green 128^3 P2, 20 steps in FP32-mixed, in FP32 flux with
    FP64 stage arithmetic and in FP64 on the same GPU (the FP64 path equals the oracle to 1e-11):
    stated L2 density difference and relative E_k-history difference of both FP32 variants."""
    from paper_2202_13821_b300 import inputs

    n, N = 128, 20
    dt = inputs.tgv_dt(n, 2)
    Q0 = inputs.tgv_state(n, 2, device="cuda")
    res = {}
    for prec in (0, 1, 2):
        s = api.Solver((n,) * 3, **TGV, order=2, mu=1 / 1600, Pr=0.72, precision=prec)
        Q = Q0.clone()
        ek = [s.kinetic_energy(Q)]
        for _ in range(N):
            s.steps(Q, dt, 1)
            ek.append(s.kinetic_energy(Q))
        s.status()
        res[prec] = (Q, np.array(ek), s)
        if prec:
            s.close()
    s64 = res[0][2]
    change = s64.l2_diff(res[0][0], Q0, 0)
    for prec in (1, 2):
        l2 = s64.l2_diff(res[prec][0], res[0][0], 0)
        dek = np.abs(res[prec][1] - res[0][1]) / res[0][1]
        print(f"128^3, {N} steps, precision {prec}: L2(rho) vs FP64 {l2:.3e} (FP64 change {change:.3e}), "
              f"max relative E_k difference {dek.max():.3e}")
        assert dek.max() < 1e-8
        assert l2 < 0.5 * change


@pytest.mark.parametrize("order,nq,precision,nsteps", [(2, 3, 1, 400), (2, 3, 0, 300), (1, 2, 1, 400),
                                                   (3, 3, 1, 300), (3, 4, 1, 300), (2, 3, 2, 400)])
def test_prandtl_072_long_run_stays_bounded(torch, api, order, nq, precision, nsteps):
    """Taylor-Green at Pr = 0.72 over hundreds of steps, every cell-kernel layout (P1 n_q = 2, P2 n_q = 3,
    P3 n_q = 3 and 4) and all three precisions for P2: the highest modes must stay at the size of the
    resolved flow.  With the Prandtl correction also applied to the fitted time derivative F_t
    (a reading since dropped: the heat flux about the velocity of t_n, differentiated in time,
    carries a frame-shift term in d_t U) both precisions doubled their largest P2 coefficient every
    ~20 steps from step ~60 and failed with non-physical states before step 300; with the correction
    on F only the largest P2 coefficient grows by 10 % over 400 steps, as with Pr = 1."""
    from paper_2202_13821_b300 import inputs

    n = 64 if order < 3 else 48
    dt = inputs.tgv_dt(n, order, cfl=0.09 if order == 3 else 0.15)  # the paper's CFL numbers (Sec. 5.3)
    s = api.Solver((n,) * 3, **TGV, order=order, mu=1 / 1600, Pr=0.72, n_q=nq, precision=precision)
    Q = inputs.tgv_state(n, order, device="cuda")
    hi = slice(1, None) if order == 1 else slice(4, None)  # the highest-degree modes present
    s.steps(Q, dt, 50)
    a50 = float(Q[:, hi].abs().max())
    s.steps(Q, dt, nsteps - 50)
    s.status()
    assert bool(torch.isfinite(Q).all())
    a_end = float(Q[:, hi].abs().max())
    print(f"P{order} n_q={nq} precision {precision}: largest high-mode coefficient {a50:.3e} after 50 steps, "
          f"{a_end:.3e} after {nsteps}")
    assert a_end < 1.5 * a50


def test_nonphysical_state_sets_flag_and_context_survives(torch, api):
    from paper_2202_13821_b300 import inputs

    s = api.Solver((8, 8, 8), **TGV, order=2, mu=1 / 1600)
    Q = inputs.tgv_state(8, 2, device="cuda")
    bad = Q.clone()
    bad[0, 0, 3, 4, 5] = -1.0  # negative density in one cell
    L, Lt = s.residual(bad, 1e-3)
    with pytest.raises(api.DghgksError) as e:
        s.status()
    assert e.value.code == -4
    # the flag was cleared and the context still works
    L, Lt = s.residual(Q, 1e-3)
    s.status()
    assert torch.isfinite(L).all()


def test_bad_arguments(torch, api):
    s = api.Solver((4, 4, 4), (0,) * 3, (1,) * 3, order=1)
    Q = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(api.DghgksError) as e:
        api.dghgks_step(s.ctx, Q, -1.0)
    assert e.value.code == -1
    with pytest.raises(api.DghgksError) as e:
        api.dghgks_residual(s.ctx, Q, 1e-3, Q, Q)  # aliasing outputs
    assert e.value.code == -1
