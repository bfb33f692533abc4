"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance (FP64 path), relative 1e-11 per variable:
  * residuals L, L_t: max |gpu - oracle| <= 1e-11 * S_v, where S_v is the
    largest coefficient of variable v of M^-1 sum |contribution| (the oracle's
    absolute-value residual, the scale of the summands).  The residual is a sum
    with heavy cancellation: in the low-Mach Taylor-Green flow the pressure
    fluxes (~p0 = 71) of opposite faces cancel to O(1), and the cancellation
    grows like 1/h, so two FP64 evaluations that differ only in operation
    order (closed-form vs LU slope solves, compile-time moment products vs
    expanded monomials, CUDA vs glibc exp/erfc) agree to ~eps * S_v, not to
    ~eps * |L|.  The result-relative error max|gpu - oracle| / max|oracle| is
    also asserted below 1e-11 on the grids up to 37 cells wide.
  * S2O4 state increments Q^{n+2} - Q^n: max |gpu - oracle| <= 1e-11 * max
    |oracle increment| per variable.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL = 1e-11


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


def per_var_err(a, b):
    a = np.asarray(a).reshape(5, -1)
    b = np.asarray(b).reshape(5, -1)
    scale = np.abs(b).max(axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    return np.abs(a - b).max(axis=1) / scale


def make(api, orc, n, lo, hi, order, nq, mu=0.0, Pr=1.0, tau_eps=0.0, precision=0, nodes=None):
    s = api.Solver(n, lo, hi, order=order, mu=mu, Pr=Pr, n_q=nq, precision=precision, tau_eps=tau_eps, nodes=nodes)
    pb = orc.Problem(order=order, nq=nq, n=tuple(n), lo=tuple(lo), hi=tuple(hi), mu=mu, Pr=Pr, tau_eps=tau_eps,
                     nodes=nodes)
    return s, pb


def oracle_residual(orc, pb, Q, dt):
    """Oracle (L, L_t, A, A_t) in the state layout."""
    nc = int(np.prod(pb.n))
    out = orc.residual_cells(pb, Q, dt, np.arange(nc), scales=True)
    return [x.transpose(1, 2, 0).reshape(pb.shape) for x in out]


def assert_residual_parity(L, Lt, ref):
    Lo, Lto, A, At = ref
    for a, b, sc in ((L, Lo, A), (Lt, Lto, At)):
        err = np.abs(a - b).reshape(5, -1).max(axis=1)
        scale = np.abs(sc).reshape(5, -1).max(axis=1)
        assert np.all(err <= RTOL * scale), (err / scale)
        assert per_var_err(a, b).max() < RTOL


def residual_pair(torch, s, pb, orc, Q, dt):
    Qd = torch.from_numpy(Q).cuda()
    L, Lt = s.residual(Qd, dt)
    torch.cuda.synchronize()
    s.status()
    return L.cpu().numpy(), Lt.cpu().numpy(), oracle_residual(orc, pb, Q, dt)


ADV = dict(lo=(0.0,) * 3, hi=(2.0,) * 3)
TGV = dict(lo=(-math.pi,) * 3, hi=(math.pi,) * 3)


@pytest.mark.parametrize("n", [(8, 8, 8), (37, 5, 6), (1, 3, 2)])
def test_advection_p1_residual(torch, api, orc, n):
    from paper_2202_13821_b300 import inputs

    s, pb = make(api, orc, n, order=1, nq=2, tau_eps=0.01, **ADV)
    Q = inputs.modal_state(inputs.advection_prim, n, 1, ADV["lo"], ADV["hi"], perturb=1e-3)
    L, Lt, ref = residual_pair(torch, s, pb, orc, Q, 8.2e-3)
    assert_residual_parity(L, Lt, ref)


@pytest.mark.parametrize("nq", [3, 2])
@pytest.mark.parametrize("Pr", [1.0, 0.72])
@pytest.mark.parametrize("n", [(8, 8, 8), (35, 9, 4)])
def test_tgv_p2_residual(torch, api, orc, n, Pr, nq):
    from paper_2202_13821_b300 import inputs

    s, pb = make(api, orc, n, order=2, nq=nq, mu=1 / 1600, Pr=Pr, **TGV)
    Q = inputs.modal_state(inputs.tgv_prim, n, 2, TGV["lo"], TGV["hi"], perturb=1e-3)
    dt = 1.3e-3
    L, Lt, ref = residual_pair(torch, s, pb, orc, Q, dt)
    assert_residual_parity(L, Lt, ref)


@pytest.mark.parametrize("order,nq", [(1, 2), (2, 3), (2, 2)])
@pytest.mark.parametrize("mu,tau_eps,Pr", [(0.0, 0.0, 1.0), (5e-3, 0.05, 1.0), (2e-3, 0.0, 0.72)])
def test_random_discontinuous_states(torch, api, orc, order, nq, mu, tau_eps, Pr):
    from paper_2202_13821_b300 import inputs

    n = (5, 4, 3)
    s, pb = make(api, orc, n, lo=(0, 0, 0), hi=(1.0, 0.8, 0.6), order=order, nq=nq, mu=mu, Pr=Pr, tau_eps=tau_eps)
    Q = inputs.random_state(n, order, seed=7 + order)
    L, Lt, ref = residual_pair(torch, s, pb, orc, Q, 2e-3)
    assert_residual_parity(L, Lt, ref)


@pytest.mark.parametrize("nq", [3, 4])
@pytest.mark.parametrize("state", ["tgv", "random"])
def test_p3_residual(torch, api, orc, nq, state):
    """P3 elements (20 modes), the paper's fourth-order case, with n_q = 3 (the paper's rule) and 4."""
    from paper_2202_13821_b300 import inputs

    if state == "tgv":
        n = (9, 5, 6)
        s, pb = make(api, orc, n, order=3, nq=nq, mu=1 / 1600, Pr=0.72, **TGV)
        Q = inputs.modal_state(inputs.tgv_prim, n, 3, TGV["lo"], TGV["hi"], perturb=1e-3)
    else:
        n = (5, 3, 4)
        s, pb = make(api, orc, n, lo=(0, 0, 0), hi=(1.0, 0.8, 0.6), order=3, nq=nq, mu=3e-3, tau_eps=0.02)
        Q = inputs.random_state(n, 3, seed=5)
    L, Lt, ref = residual_pair(torch, s, pb, orc, Q, 1.5e-3)
    assert_residual_parity(L, Lt, ref)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("order,nq", [(1, 2), (2, 2), (2, 3), (3, 3), (3, 4)])
def test_fp32_mixed_residual_every_layout(torch, api, orc, order, nq, precision):
    """FP32-mixed residual (Sec. 3, Eq. (flux) and (flux-2) in FP32 arithmetic) against the FP64
    oracle for every FP32 face layout (a thread per row of n_q Gauss points) and cell layout, on a
    perturbed Taylor-Green state with 35 cells along x (one full 32-face CTA and a ragged one).

    Bound per variable: 2e-5 of the oracle's magnitude scale (the sum of the absolute values of the
    terms that make up the residual).  FP32 rounds each of the few hundred terms of a point flux and
    of the projections to 6e-8 of its size; 2e-5 = 335 units of FP32 rounding of the scale leaves
    room for their accumulation and for the divisions and exponentials of the flux.  Measured on a
    B300: L within 2.5e-7 of its scale for every layout; L_t, formed from the time fit of the face
    flux, within 1.6e-5 at P1 (the fewest terms per scale), 9e-6 at P2 and 5e-6 at P3.  The same
    bound holds for the FP32 flux with FP64 assembly and M^-1 (precision 2)."""
    from paper_2202_13821_b300 import inputs

    n = (35, 5, 3)
    s, pb = make(api, orc, n, order=order, nq=nq, mu=1 / 1600, Pr=0.72, precision=precision, **TGV)
    Q = inputs.modal_state(inputs.tgv_prim, n, order, TGV["lo"], TGV["hi"], perturb=1e-3)
    L, Lt, ref = residual_pair(torch, s, pb, orc, Q, 1.5e-3)
    worst = []
    for a, b, sc in ((L, ref[0], ref[2]), (Lt, ref[1], ref[3])):
        err = np.abs(a - b).reshape(5, -1).max(axis=1)
        scale = np.abs(sc).reshape(5, -1).max(axis=1)
        worst.append((err / scale).max())
        assert np.all(err <= 2e-5 * scale), err / scale
    print(f"P{order} n_q={nq} precision {precision}: max err / scale L {worst[0]:.2e}, L_t {worst[1]:.2e}")


@pytest.mark.parametrize("precision", [0, 1])
def test_rows_longer_than_the_grid(torch, api, orc, precision):
    """Persistent cell CTAs take the tiles of 8 cells gridDim.x apart and step a tile's coordinates
    from the previous one.  2400 x 1 x 2 cells: 300 tiles per row, more than the resident CTAs of a
    B300 (148 in FP64, 296 in FP32), so a CTA's next tile lies in the same row or, past the row's end,
    in the next row, which here is the next z plane (the row index wraps into the plane index).  FP64:
    the parity bound of the other residual tests; FP32-mixed: 2e-5 of the oracle's magnitude scale."""
    from paper_2202_13821_b300 import inputs

    n = (2400, 1, 2)
    s, pb = make(api, orc, n, order=2, nq=3, mu=1 / 1600, Pr=0.72, precision=precision, **TGV)
    Q = inputs.modal_state(inputs.tgv_prim, n, 2, TGV["lo"], TGV["hi"], perturb=1e-3)
    L, Lt, ref = residual_pair(torch, s, pb, orc, Q, 1.3e-3)
    if precision == 0:
        assert_residual_parity(L, Lt, ref)
    else:
        for a, b, sc in ((L, ref[0], ref[2]), (Lt, ref[1], ref[3])):
            err = np.abs(a - b).reshape(5, -1).max(axis=1)
            scale = np.abs(sc).reshape(5, -1).max(axis=1)
            assert np.all(err <= 2e-5 * scale), err / scale


@pytest.mark.parametrize("order,nq,case", [(1, 2, "adv"), (2, 3, "tgv"), (3, 4, "tgv")])
def test_s2o4_step_parity(torch, api, orc, order, nq, case):
    from paper_2202_13821_b300 import inputs

    n = (6, 7, 5)
    if case == "adv":
        s, pb = make(api, orc, n, order=order, nq=nq, tau_eps=0.01, **ADV)
        Q = inputs.modal_state(inputs.advection_prim, n, order, ADV["lo"], ADV["hi"], perturb=1e-3)
        dt = 8e-3
    else:
        s, pb = make(api, orc, n, order=order, nq=nq, mu=1 / 1600, Pr=0.72, **TGV)
        Q = inputs.modal_state(inputs.tgv_prim, n, order, TGV["lo"], TGV["hi"], perturb=1e-3)
        dt = 5e-3
    Qd = torch.from_numpy(Q).cuda()
    s.step(Qd, dt, 2)
    s.status()
    Qo = orc.step(pb, Q, dt, 2)
    dg = Qd.cpu().numpy() - Q
    do = Qo - Q
    assert per_var_err(dg, do).max() < RTOL


def test_sampled_cells_full_size_tgv_256(torch, api, orc):
    """Bench launch configuration (TGV 256^3, P2, n_q = 3, FP64) on sampled cells."""
    from paper_2202_13821_b300 import inputs

    n = (256, 256, 256)
    s, pb = make(api, orc, n, order=2, nq=3, mu=1 / 1600, Pr=0.72, **TGV)
    Qd = inputs.tgv_state(256, 2, device="cuda")
    Q = Qd.cpu().numpy()
    dt = inputs.tgv_dt(256, 2)
    L, Lt = s.residual(Qd, dt)
    torch.cuda.synchronize()
    s.status()
    rng = np.random.default_rng(0)
    cells = np.concatenate([[0, 255, 256 * 256 - 1, 256 ** 3 - 1, 256 * 255 + 31, 256 * 256 * 128 + 33],
                            rng.integers(0, 256 ** 3, 40)])
    Lo, Lto, Ao, Ato = orc.residual_cells(pb, Q, dt, cells, scales=True)
    Lc = L.reshape(5, 10, -1)[:, :, cells].permute(2, 0, 1).cpu().numpy()
    Ltc = Lt.reshape(5, 10, -1)[:, :, cells].permute(2, 0, 1).cpu().numpy()
    # scale per variable over the sampled cells
    for a, b, sc in ((Lc, Lo, Ao), (Ltc, Lto, Ato)):
        err = np.abs(a - b).max(axis=(0, 2))
        scale = np.abs(sc).max(axis=(0, 2))
        assert np.all(err <= RTOL * scale), err / scale


@pytest.mark.parametrize("precision", [1, 2])
def test_fp32_mixed_steps_sampled_full_size_tgv_256(torch, api, orc, precision):
    """Bench configuration of the timed leg (TGV 256^3, P2, n_q = 3, FP32-mixed, one dghgks_steps call
    of 2 steps, the second reading the FP32 copy of the state) against the FP64 oracle on sampled
    cells; the same for the FP32 flux with FP64 stage arithmetic (precision 2).  After 2 S2O4 steps (4 stages) a cell depends only on the cells within 4 face-neighbour
    hops, so the oracle steps a periodic 9^3 box cut around each sampled cell from the same initial
    state; the box's wrap reaches the centre only after 5 hops, so the centre's result is exact.

    Tolerance, per variable: the FP32 residual of a cell sums a few hundred terms of size up to its
    absolute-value scale A (the oracle's M^-1 sum |contribution|), so its rounding error is bounded by
    about 300 u A = 2e-5 A (u = 2^-24); the two steps' increment dt (L(Q^0) + L(Q^1)) + O(dt^2 L_t)
    carries at most 2.5 such errors in dt A plus 2 in dt^2 A_t."""
    from paper_2202_13821_b300 import inputs

    n = 256
    s = api.Solver((n,) * 3, TGV["lo"], TGV["hi"], order=2, mu=1 / 1600, Pr=0.72, n_q=3, precision=precision)
    Q0 = inputs.tgv_state(n, 2, device="cuda")
    dt = inputs.tgv_dt(n, 2)
    Qd = Q0.clone()
    s.steps(Qd, dt, 2)
    torch.cuda.synchronize()
    s.status()
    h = 2 * math.pi / n
    rng = np.random.default_rng(5)
    cells = [(0, 0, 0), (255, 255, 255), (131, 7, 200)] + [tuple(int(x) for x in rng.integers(0, n, 3)) for _ in range(5)]
    worst = np.zeros(5)
    for (i, j, k) in cells:
        ix, iy, iz = (torch.tensor((c + np.arange(-4, 5)) % n, device="cuda") for c in (i, j, k))
        sub = Q0.index_select(2, iz).index_select(3, iy).index_select(4, ix).cpu().numpy()
        lo = tuple(TGV["lo"][d] + (c - 4) * h for d, c in enumerate((i, j, k)))
        pb = orc.Problem(order=2, nq=3, n=(9, 9, 9), lo=lo, hi=tuple(x + 9 * h for x in lo), mu=1 / 1600, Pr=0.72)
        want = orc.step(pb, sub, dt, 2)[:, :, 4, 4, 4]
        _, _, A, At = orc.residual_cells(pb, sub, dt, np.array([4 + 9 * (4 + 9 * 4)]), scales=True)
        got = Qd[:, :, k, j, i].cpu().numpy()
        tol = 2e-5 * (2.5 * dt * A[0].max(axis=1) + 2 * dt * dt * At[0].max(axis=1))
        err = np.abs(got - want).max(axis=1)
        assert np.all(err <= tol), (i, j, k, err / tol)
        worst = np.maximum(worst, err / tol)
    s.close()
    print(f"precision {precision}: max error / tolerance per variable:", worst)


def test_totals_and_kinetic_energy(torch, api, orc):
    from paper_2202_13821_b300 import inputs

    n = (12, 10, 9)
    s, pb = make(api, orc, n, order=2, nq=3, mu=1 / 1600, **TGV)
    Q = inputs.modal_state(inputs.tgv_prim, n, 2, TGV["lo"], TGV["hi"], perturb=1e-3)
    Qd = torch.from_numpy(Q).cuda()
    np.testing.assert_allclose(s.totals(Qd), orc.totals(pb, Q), rtol=1e-13, atol=1e-13)
    assert abs(s.kinetic_energy(Qd) - orc.kinetic_energy(pb, Q)) < 1e-14
    e_gpu, e_orc = s.enstrophy_dissipation(Qd), orc.enstrophy_dissipation(pb, Q)
    assert abs(e_gpu - e_orc) <= 1e-12 * abs(e_orc)
    # L2 difference through the mass matrix against a direct numpy evaluation
    Q2 = Q.copy()
    Q2[0] += 1e-3 * np.random.default_rng(1).standard_normal(Q2[0].shape)
    h = [(TGV["hi"][d] - TGV["lo"][d]) / n[d] for d in range(3)]
    md = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    M = np.array([np.prod(h) / np.prod([2 * e + 1 for e in m]) for m in md])
    want = math.sqrt(np.sum(M[:, None, None, None] * (Q2[0] - Q[0]) ** 2))
    got = s.l2_diff(torch.from_numpy(Q2).cuda(), Qd, 0)
    assert abs(got - want) <= 1e-12 * want


# ---- rectilinear (non-uniform) meshes ----

def random_mesh(n, lo, hi, seed=40, spread=0.4):
    from paper_2202_13821_b300 import inputs

    return tuple(inputs.random_nodes(n[d], lo[d], hi[d], spread=spread, seed=seed + d) for d in range(3))


@pytest.mark.parametrize("order,nq", [(1, 2), (2, 3), (2, 2), (3, 3), (3, 4)])
@pytest.mark.parametrize("n", [(37, 5, 6), (3, 4, 2)])
def test_rectilinear_residual(torch, api, orc, order, nq, n):
    """Random cell widths (+-40%) on every axis; x spans two face tiles with a ragged tail."""
    from paper_2202_13821_b300 import inputs

    nodes = random_mesh(n, TGV["lo"], TGV["hi"])
    s, pb = make(api, orc, n, order=order, nq=nq, mu=1 / 1600, Pr=0.72, nodes=nodes, **TGV)
    Q = inputs.modal_state(inputs.tgv_prim, n, order, TGV["lo"], TGV["hi"], perturb=1e-3, nodes=nodes)
    L, Lt, ref = residual_pair(torch, s, pb, orc, Q, 1.3e-3)
    assert_residual_parity(L, Lt, ref)


def test_rectilinear_mapped_mesh_one_axis(torch, api, orc):
    """The mapped grid of Sec. 5.1 along y only (x, z uniform), random discontinuous state."""
    from paper_2202_13821_b300 import inputs

    n = (6, 9, 4)
    nodes = (None, inputs.mapped_nodes(9), None)
    s, pb = make(api, orc, n, lo=(0.0,) * 3, hi=(1.0, 2.0, 0.5), order=2, nq=3, mu=2e-3, Pr=0.72, tau_eps=0.01,
                 nodes=nodes)
    Q = inputs.random_state(n, 2, seed=17)
    L, Lt, ref = residual_pair(torch, s, pb, orc, Q, 2e-3)
    assert_residual_parity(L, Lt, ref)


@pytest.mark.parametrize("order,nq", [(2, 3), (3, 4)])
def test_rectilinear_step_parity(torch, api, orc, order, nq):
    from paper_2202_13821_b300 import inputs

    n = (6, 7, 5)
    nodes = tuple(inputs.mapped_nodes(v) for v in n)
    s, pb = make(api, orc, n, order=order, nq=nq, tau_eps=0.01, nodes=nodes, **ADV)
    Q = inputs.advection_state(n, order, perturb=1e-3, nodes=nodes)
    Qd = torch.from_numpy(Q).cuda()
    s.step(Qd, 6e-3, 2)
    s.status()
    Qo = orc.step(pb, Q, 6e-3, 2)
    assert per_var_err(Qd.cpu().numpy() - Q, Qo - Q).max() < RTOL


def test_rectilinear_reductions(torch, api, orc):
    from paper_2202_13821_b300 import inputs

    n = (12, 10, 9)
    nodes = random_mesh(n, TGV["lo"], TGV["hi"], seed=50)
    s, pb = make(api, orc, n, order=2, nq=3, mu=1 / 1600, nodes=nodes, **TGV)
    Q = inputs.modal_state(inputs.tgv_prim, n, 2, TGV["lo"], TGV["hi"], perturb=1e-3, nodes=nodes)
    Qd = torch.from_numpy(Q).cuda()
    np.testing.assert_allclose(s.totals(Qd), orc.totals(pb, Q), rtol=1e-13, atol=1e-13)
    assert abs(s.kinetic_energy(Qd) - orc.kinetic_energy(pb, Q)) < 1e-14
    e_gpu, e_orc = s.enstrophy_dissipation(Qd), orc.enstrophy_dissipation(pb, Q)
    assert abs(e_gpu - e_orc) <= 1e-12 * abs(e_orc)
    Q2 = Q.copy()
    Q2[0] += 1e-3 * np.random.default_rng(2).standard_normal(Q2[0].shape)
    w = [np.diff(x) for x in nodes]
    vol = w[2][:, None, None] * w[1][None, :, None] * w[0][None, None, :]
    md = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    norm = np.array([1.0 / np.prod([2 * e + 1 for e in m]) for m in md])
    want = math.sqrt(np.sum(norm[:, None, None, None] * vol[None] * (Q2[0] - Q[0]) ** 2))
    got = s.l2_diff(torch.from_numpy(Q2).cuda(), Qd, 0)
    assert abs(got - want) <= 1e-12 * want


def test_rectilinear_fp32_mixed_close_to_fp64(torch, api, orc):
    from paper_2202_13821_b300 import inputs

    n = (20, 12, 9)
    nodes = random_mesh(n, TGV["lo"], TGV["hi"], seed=60)
    Q = inputs.modal_state(inputs.tgv_prim, n, 2, TGV["lo"], TGV["hi"], perturb=1e-3, nodes=nodes)
    out = []
    for prec in (0, 1):
        s = api.Solver(n, TGV["lo"], TGV["hi"], order=2, mu=1 / 1600, Pr=0.72, n_q=3, precision=prec, nodes=nodes)
        L, Lt = s.residual(torch.from_numpy(Q).cuda(), 1.3e-3)
        s.status()
        out.append((L.cpu().numpy(), Lt.cpu().numpy()))
    ref = oracle_residual(orc, orc.Problem(order=2, nq=3, n=n, mu=1 / 1600, Pr=0.72, nodes=nodes), Q, 1.3e-3)
    for a, b, sc in ((out[1][0], out[0][0], ref[2]), (out[1][1], out[0][1], ref[3])):
        err = np.abs(a - b).reshape(5, -1).max(axis=1)
        scale = np.abs(sc).reshape(5, -1).max(axis=1)
        assert np.all(err <= 2e-5 * scale), err / scale


def test_rectilinear_rejects_bad_nodes(torch, api):
    from paper_2202_13821_b300 import inputs

    n = (4, 4, 4)
    bad = inputs.mapped_nodes(4)[::-1].copy()
    with pytest.raises(api.DghgksError) as e:
        api.Solver(n, (0,) * 3, (2,) * 3, order=2, nodes=(bad, None, None))
    assert e.value.code == -1
