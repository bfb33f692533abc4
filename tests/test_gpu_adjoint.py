"""Adjoint (reverse-mode) kernels against the oracle's forward-mode dual numbers
and against central finite differences (GPU, FP64, through the C ABI).

* residual VJP: <lamL, dL> + <lamLt, dLt> (oracle dual-number JVP along
  (dQ, dmu)) equals <lamQ, dQ> + dmu_bar * dmu (GPU VJP), relative 1e-10;
* adjoint step: <lam_{n+1}, dQ^{n+1}> (oracle JVP of one S2O4 step) equals
  <lam_n, dQ^n> + dJ/dmu * dmu;
* E_k after N steps: the directional derivative from the GPU gradient
  (torch.autograd through rollout + kinetic_energy) matches the oracle's
  dual-number derivative and a central finite difference of the GPU forward
  (8^3 P1 advection-type state, seeded Gaussian direction; FD to 1e-6).
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


def direction(shape, seed, Q):
    rng = np.random.default_rng(seed)
    scale = np.abs(Q).reshape(5, -1).max(axis=1)[:, None, None, None, None]
    return rng.standard_normal(shape) * scale * 1e-2


CASES = [
    dict(order=1, nq=2, n=(5, 4, 3), mu=5e-3, Pr=1.0, tau_eps=0.0, state="random"),
    dict(order=2, nq=3, n=(4, 5, 3), mu=1e-2, Pr=0.72, tau_eps=0.0, state="random", nodes=True),
    dict(order=1, nq=2, n=(6, 5, 4), mu=2e-3, Pr=1.0, tau_eps=0.01, state="adv", nodes=True),
    dict(order=3, nq=3, n=(5, 4, 3), mu=1e-2, Pr=0.72, tau_eps=0.0, state="tgv"),
    dict(order=3, nq=3, n=(4, 3, 4), mu=5e-3, Pr=0.72, tau_eps=0.0, state="random", nodes=True),
    dict(order=2, nq=3, n=(4, 3, 5), mu=1e-2, Pr=0.72, tau_eps=0.0, state="random"),
    dict(order=2, nq=2, n=(6, 5, 4), mu=1 / 1600, Pr=0.72, tau_eps=0.0, state="tgv"),
    dict(order=1, nq=2, n=(6, 6, 6), mu=0.0, Pr=1.0, tau_eps=0.01, state="adv"),
    # P3 with n_q = 4: a cell's 64 points over two warps, cell CTAs of 4 cells
    # (ragged at nx = 5 and 3)
    dict(order=3, nq=4, n=(5, 3, 3), mu=1e-2, Pr=0.72, tau_eps=0.0, state="tgv"),
    dict(order=3, nq=4, n=(3, 4, 3), mu=5e-3, Pr=0.72, tau_eps=0.0, state="random", nodes=True),
]


def make_case(api, orc, c):
    from paper_2202_13821_b300 import inputs

    if c["state"] == "tgv":
        lo, hi = (-math.pi,) * 3, (math.pi,) * 3
        Q = inputs.modal_state(inputs.tgv_prim, c["n"], c["order"], lo, hi, perturb=1e-3)
    elif c["state"] == "adv":
        lo, hi = (0.0,) * 3, (2.0,) * 3
        Q = inputs.modal_state(inputs.advection_prim, c["n"], c["order"], lo, hi, perturb=1e-3)
    else:
        lo, hi = (0.0,) * 3, (1.0, 0.8, 0.6)
        Q = inputs.random_state(c["n"], c["order"], seed=21)
    nodes = None
    if c.get("nodes"):  # rectilinear mesh: random widths (+-40 %) on every axis
        nodes = tuple(inputs.random_nodes(c["n"][d], lo[d], hi[d], spread=0.4, seed=70 + d) for d in range(3))
        if c["state"] == "adv":
            Q = inputs.advection_state(c["n"], c["order"], perturb=1e-3, nodes=nodes)
    s = api.Solver(c["n"], lo, hi, order=c["order"], mu=c["mu"], Pr=c["Pr"], n_q=c["nq"], tau_eps=c["tau_eps"],
                   nodes=nodes)
    pb = orc.Problem(order=c["order"], nq=c["nq"], n=tuple(c["n"]), lo=lo, hi=hi, mu=c["mu"], Pr=c["Pr"],
                     tau_eps=c["tau_eps"], nodes=nodes)
    return s, pb, Q


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"P{c['order']}nq{c['nq']}-{c['state']}-Pr{c['Pr']}"
                                                    + ("-rect" if c.get("nodes") else ""))
def test_residual_vjp_dot_product(torch, api, orc, case):
    s, pb, Q = make_case(api, orc, case)
    dt = 3e-3
    dQ = direction(Q.shape, 1, Q)
    dmu = 1e-3
    _, _, dL, dLt = orc.residual_jvp(pb, Q, dQ, dmu, dt)
    rng = np.random.default_rng(2)
    lamL, lamLt = rng.standard_normal(Q.shape), rng.standard_normal(Q.shape)
    lamQ = torch.empty(Q.shape, dtype=torch.float64, device="cuda")
    mu_bar = torch.zeros(1, dtype=torch.float64, device="cuda")
    api.dghgks_residual_vjp(s.ctx, torch.from_numpy(Q).cuda(), dt, torch.from_numpy(lamL).cuda(),
                            torch.from_numpy(lamLt).cuda(), lamQ, mu_bar)
    torch.cuda.synchronize()
    lhs = np.sum(lamL * dL) + np.sum(lamLt * dLt)
    rhs = np.sum(lamQ.cpu().numpy() * dQ) + float(mu_bar.item()) * dmu
    scale = np.sum(np.abs(lamL * dL)) + np.sum(np.abs(lamLt * dLt))
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("case", CASES[1:7] + CASES[8:10], ids=lambda c: f"P{c['order']}nq{c['nq']}-{c['state']}"
                                                                        + ("-rect" if c.get("nodes") else ""))
def test_adjoint_step_dot_product(torch, api, orc, case):
    s, pb, Q = make_case(api, orc, case)
    dt = 2e-3
    dQ = direction(Q.shape, 3, Q)
    dmu = 1e-3
    _, dQ1, _, _ = orc.step_jvp(pb, Q, dQ, dmu, dt, 1)
    lam = np.random.default_rng(4).standard_normal(Q.shape)
    lam_n = torch.from_numpy(lam).cuda()
    g_mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    api.dghgks_adjoint_step(s.ctx, torch.from_numpy(Q).cuda(), lam_n, dt, lam_n, g_mu)  # in place
    torch.cuda.synchronize()
    lhs = np.sum(lam * dQ1)
    rhs = np.sum(lam_n.cpu().numpy() * dQ) + float(g_mu.item()) * dmu
    scale = np.sum(np.abs(lam * dQ1))
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs)


@pytest.mark.parametrize("rect", [False, True], ids=["uniform", "rect"])
def test_kinetic_energy_gradient_vs_dual_numbers_and_fd(torch, api, orc, rect):
    """E_k after 4 steps, 8^3 P1, gradient w.r.t. Q^0 and mu (FD along a seeded Gaussian direction);
    uniform mesh, and the mapped grid of Sec. 5.1 on the three axes."""
    from paper_2202_13821_b300 import autograd, inputs

    n, lo, hi = (8, 8, 8), (-math.pi,) * 3, (math.pi,) * 3
    nodes = tuple(-math.pi + math.pi * inputs.mapped_nodes(8) for _ in range(3)) if rect else None
    mu0, dt, N = 2e-2, 4e-3, 4
    Q0 = inputs.modal_state(inputs.tgv_prim, n, 1, lo, hi, perturb=1e-3, prim_kw=dict(Ma=0.3), nodes=nodes)
    s = api.Solver(n, lo, hi, order=1, mu=mu0, Pr=0.72, n_q=2, nodes=nodes)
    pb = orc.Problem(order=1, nq=2, n=n, lo=lo, hi=hi, mu=mu0, Pr=0.72, nodes=nodes)
    Qt = torch.from_numpy(Q0).cuda().requires_grad_(True)
    mu = torch.tensor(mu0, dtype=torch.float64, device="cuda", requires_grad=True)
    J = autograd.kinetic_energy(autograd.rollout(Qt, mu, s, dt, N), s)
    J.backward()
    gQ, gmu = Qt.grad.cpu().numpy(), float(mu.grad.item())
    dQ = np.random.default_rng(7).standard_normal(Q0.shape) * np.abs(Q0).reshape(5, -1).max(axis=1)[:, None, None, None, None] * 1e-3
    dmu = 1e-3
    directional = np.sum(gQ * dQ) + gmu * dmu
    # exact directional derivative from the oracle's dual numbers
    _, _, Ek, dEk = orc.step_jvp(pb, Q0, dQ, dmu, dt, N)
    assert abs(float(J.item()) - Ek) <= 1e-12 * abs(Ek)
    assert abs(directional - dEk) <= 1e-9 * abs(dEk), (directional, dEk)
    # central finite difference of the GPU forward
    h = 1e-4

    def Ek_at(eps):
        s.set_mu(mu0 + eps * dmu)
        Q = torch.from_numpy(Q0 + eps * dQ).cuda()
        s.step(Q, dt, N)
        return s.kinetic_energy(Q)

    fd = (Ek_at(h) - Ek_at(-h)) / (2 * h)
    assert abs(directional - fd) <= 1e-6 * abs(fd), (directional, fd)


def test_adjoint_configuration_tgv32_p2_50_steps(torch, api):
    """The adjoint configuration: Taylor-Green 32^3, P2, FP64, 50 S2O4 steps, gradient of the final
    E_k with respect to every initial modal coefficient and mu (per-step checkpoints, stage
    recomputation), checked against a central finite difference of the forward run along a
    seeded Gaussian direction."""
    from paper_2202_13821_b300 import autograd, inputs

    n, N = 32, 50
    lo, hi = (-math.pi,) * 3, (math.pi,) * 3
    mu0 = 1 / 1600
    dt = inputs.tgv_dt(n, 2)
    s = api.Solver((n,) * 3, lo, hi, order=2, mu=mu0, Pr=0.72, n_q=3)
    Q0 = inputs.tgv_state(n, 2, perturb=1e-4, device="cuda")
    Qt = Q0.clone().requires_grad_(True)
    mu = torch.tensor(mu0, dtype=torch.float64, device="cuda", requires_grad=True)
    J = autograd.kinetic_energy(autograd.rollout(Qt, mu, s, dt, N), s)
    J.backward()
    gQ, gmu = Qt.grad, float(mu.grad.item())
    assert torch.isfinite(gQ).all()
    g = torch.Generator(device="cpu").manual_seed(11)
    scale = Q0.reshape(5, -1).abs().amax(dim=1).reshape(5, 1, 1, 1, 1)
    dQ = (torch.randn(Q0.shape, generator=g, dtype=torch.float64) * 1e-3).cuda() * scale
    dmu = 1e-4 * mu0
    directional = float((gQ * dQ).sum()) + gmu * dmu
    h = 1e-3

    def Ek_at(eps):
        s.set_mu(mu0 + eps * dmu)
        Q = Q0 + eps * dQ
        s.steps(Q, dt, N)
        return s.kinetic_energy(Q)

    fd = (Ek_at(h) - Ek_at(-h)) / (2 * h)
    print(f"directional derivative: adjoint {directional:.12e}, finite difference {fd:.12e}, dJ/dmu {gmu:.6e}")
    assert abs(directional - fd) <= 1e-6 * abs(fd), (directional, fd)
