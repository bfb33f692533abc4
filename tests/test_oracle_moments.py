"""Pins of the oracle's Maxwellian moments and slope solves (Sec. 2).

References are brute-force velocity-space quadratures in numpy: Gauss-Hermite
for the full space, Gauss-Legendre on a truncated half line for u > 0 / u < 0,
the Gamma-function moments of a chi-square variable for xi^2, and a direct
5-dimensional quadrature of the moment matrix <psi_k psi_m> for K = 2.
"""
import itertools
import math

import numpy as np
import pytest
from scipy.special import gamma as Gamma


def _full_1d(U, lam, n):
    x, w = np.polynomial.hermite.hermgauss(60)
    u = U + x / np.sqrt(lam)
    return np.sum(w * u ** n) / np.sqrt(np.pi)


def _half_1d(U, lam, n, sign):
    # integrate sqrt(lam/pi) exp(-lam (u-U)^2) u^n over u>0 (sign=+1) or u<0 (sign=-1)
    L = abs(U) + 14.0 / np.sqrt(lam)
    x, w = np.polynomial.legendre.leggauss(400)
    # two panels for accuracy
    tot = 0.0
    for a, b in ((0.0, L / 4), (L / 4, L)):
        s = 0.5 * (b - a) * x + 0.5 * (b + a)
        u = sign * s
        tot += 0.5 * (b - a) * np.sum(w * np.sqrt(lam / np.pi) * np.exp(-lam * (u - U) ** 2) * u ** n)
    return tot


CASES = [(0.3, 0.7), (-1.2, 2.5), (2.0, 0.35), (0.0, 1.0), (-0.05, 7.0)]


@pytest.mark.parametrize("U,lam", CASES)
def test_full_and_half_space_moments(orc, U, lam):
    for region in (0, 1, -1):
        m, xi = orc.moments([U, -0.4, 0.9], lam, region, 2.0)
        for n in range(10):
            ref = _full_1d(U, lam, n) if region == 0 else _half_1d(U, lam, n, region)
            assert abs(m[0, n] - ref) <= 1e-12 * max(1.0, abs(ref)), (region, n, m[0, n], ref)
        for n in range(10):  # v, w always full space
            assert abs(m[1, n] - _full_1d(-0.4, lam, n)) <= 1e-12 * max(1, abs(m[1, n]))
            assert abs(m[2, n] - _full_1d(0.9, lam, n)) <= 1e-12 * max(1, abs(m[2, n]))
    # half spaces add to the full space
    mf, _ = orc.moments([U, 0, 0], lam, 0, 2.0)
    mp, _ = orc.moments([U, 0, 0], lam, 1, 2.0)
    mn, _ = orc.moments([U, 0, 0], lam, -1, 2.0)
    np.testing.assert_allclose(mp[0] + mn[0], mf[0], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("K", [2.0, 0.0, 3.0, 1.5])
def test_internal_dof_moments(orc, K):
    lam = 0.8
    _, xi = orc.moments([0, 0, 0], lam, 0, K)
    sig2 = 1 / (2 * lam)
    for d in range(4):
        # xi^2 = sig2 * chi2_K; E[chi2_K^d] = 2^d Gamma(K/2 + d) / Gamma(K/2)
        ref = sig2 ** d * (2 ** d * Gamma(K / 2 + d) / Gamma(K / 2) if K > 0 else (1.0 if d == 0 else 0.0))
        assert abs(xi[d] - ref) <= 1e-14 * max(1, ref)


def _moment_matrix_bruteforce(U, lam):
    """<psi_k psi_m> for K = 2 by a tensor Gauss-Hermite rule in (u, v, w, xi_1, xi_2)."""
    x, w = np.polynomial.hermite.hermgauss(8)
    s = 1 / np.sqrt(lam)
    M = np.zeros((5, 5))
    for (a, wa), (b, wb), (c, wc) in itertools.product(zip(x, w), repeat=3):
        u, v, ww = U[0] + a * s, U[1] + b * s, U[2] + c * s
        X1, X2 = np.meshgrid(x * s, x * s, indexing="ij")
        W12 = np.outer(w, w)
        xi2 = X1 ** 2 + X2 ** 2
        psi = [np.ones_like(xi2), u + 0 * xi2, v + 0 * xi2, ww + 0 * xi2, 0.5 * (u * u + v * v + ww * ww + xi2)]
        for k in range(5):
            for m in range(5):
                M[k, m] += wa * wb * wc * np.sum(W12 * psi[k] * psi[m])
    return M / np.pi ** 2.5


@pytest.mark.parametrize("U,lam", [((0.3, -0.5, 1.1), 0.9), ((-2.0, 0.1, 0.0), 3.0), ((0, 0, 0), 0.25)])
def test_slope_solve_residual(orc, U, lam):
    M = _moment_matrix_bruteforce(np.array(U), lam)
    rng = np.random.default_rng(5)
    for _ in range(3):
        b = rng.standard_normal(5)
        a = orc.slope(U, lam, 2.0, b)
        np.testing.assert_allclose(M @ a, b, rtol=1e-11, atol=1e-11 * np.abs(b).max())
