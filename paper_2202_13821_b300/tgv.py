"""Taylor-Green vortex time histories (Sec. 5.3): E_k(t), eps(E_k) = -dE_k/dt and
eps(zeta) = 2 mu / (rho0 Omega) int 1/2 rho |curl U|^2.

The paper's setting is Pr = 1 and n_q = k Gauss points per direction (P2: 2, P3: 3),
on 32^3 to 96^3 cells, to t = 10.  Every step runs on the GPU through the C ABI
(graph replay between samples); E_k and eps(zeta) are the library's FP64
reductions; eps(E_k) is the second-order central difference of the sampled E_k,
as in the paper.

    python -m paper_2202_13821_b300.tgv --n 64 --order 2 --t-end 10 --out tgv64.csv
"""
from __future__ import annotations

import argparse
import math

import numpy as np


def run(n: int = 64, order: int = 2, n_q: int = 0, t_end: float = 10.0, cfl: float = 0.15, Pr: float = 1.0,
        Re: float = 1600.0, Ma: float = 0.1, precision: int = 1, sample_dt: float = 0.1, device: str = "cuda"):
    """Returns a dict of numpy arrays t, ek, eps_ek (central difference; NaN at the ends), eps_zeta."""
    from . import api, inputs

    n_q = n_q or order  # the paper's rule
    mu = 1.0 / Re  # rho0 V0 L / Re with rho0 = V0 = L = 1
    s = api.Solver((n,) * 3, (-math.pi,) * 3, (math.pi,) * 3, order=order, mu=mu, Pr=Pr, n_q=n_q,
                   precision=precision)
    Q = inputs.tgv_state(n, order, Ma=Ma, device=device)
    dt0 = inputs.tgv_dt(n, order, cfl=cfl, Ma=Ma)
    per = max(1, math.ceil(sample_dt / dt0))  # steps per sample
    dt = sample_dt / per
    nsamp = int(round(t_end / sample_dt))
    t = [0.0]
    ek = [s.kinetic_energy(Q)]
    ez = [s.enstrophy_dissipation(Q)]
    for m in range(nsamp):
        s.steps(Q, dt, per)
        t.append((m + 1) * sample_dt)
        ek.append(s.kinetic_energy(Q))
        ez.append(s.enstrophy_dissipation(Q))
    s.status()
    t, ek, ez = np.array(t), np.array(ek), np.array(ez)
    eps_ek = np.full_like(ek, np.nan)
    eps_ek[1:-1] = -(ek[2:] - ek[:-2]) / (t[2:] - t[:-2])
    return {"t": t, "ek": ek, "eps_ek": eps_ek, "eps_zeta": ez, "dt": dt, "steps": per * nsamp}


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--order", type=int, default=2)
    ap.add_argument("--n-q", type=int, default=0, help="Gauss points per direction (0: the paper's k)")
    ap.add_argument("--t-end", type=float, default=10.0)
    ap.add_argument("--precision", type=int, default=1, help="0 FP64, 1 FP32-mixed")
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    h = run(a.n, a.order, a.n_q, a.t_end, precision=a.precision)
    rows = np.stack([h["t"], h["ek"], h["eps_ek"], h["eps_zeta"]], axis=1)
    if a.out:
        np.savetxt(a.out, rows, delimiter=",", header="t,E_k,eps(E_k),eps(zeta)", comments="")
    i = int(np.nanargmax(h["eps_ek"]))
    print(f"{h['steps']} steps of dt {h['dt']:.4e}; E_k(t_end) {h['ek'][-1]:.5f}; "
          f"max eps(E_k) {h['eps_ek'][i]:.5f} at t = {h['t'][i]:.2f}; "
          f"max eps(zeta) {h['eps_zeta'].max():.5f} at t = {h['t'][int(np.argmax(h['eps_zeta']))]:.2f}")


if __name__ == "__main__":
    main()
