"""Pins of the oracle's basis, mass matrix and Gauss rules (Sec. 3, Eqs. expansion, surface, volume).

Independent references: numpy's Legendre module and Gauss-Legendre rule.
"""
import itertools

import numpy as np
import numpy.polynomial.legendre as npl
import pytest


def _leg(n, x):
    c = np.zeros(n + 1)
    c[n] = 1
    return npl.legval(x, c)


def _dleg(n, x):
    c = np.zeros(n + 1)
    c[n] = 1
    return npl.legval(x, npl.legder(c))


MODES = {
    0: [(0, 0, 0)],
    1: [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)],
    2: [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)],
}


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_gauss_rule_matches_numpy(orc, n):
    x, w = orc.gauss(n)
    xr, wr = npl.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=1e-15)
    np.testing.assert_allclose(w, wr / 2, rtol=1e-14)  # normalised: sum to 1
    assert abs(w.sum() - 1) < 1e-15


@pytest.mark.parametrize("order", [1, 2, 3])
def test_mode_count_and_set(orc, order):
    nm = (order + 1) * (order + 2) * (order + 3) // 6
    want = {m for m in itertools.product(range(order + 1), repeat=3) if sum(m) <= order}
    assert len(want) == nm
    # identify each oracle mode by its values at random points (unique for distinct modes)
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1, 1, (12, 3))
    got = []
    for m in range(nm):
        vals = np.array([orc.basis(order, p)[0][m] for p in pts])
        match = [t for t in want if np.allclose(vals, [_leg(t[0], p[0]) * _leg(t[1], p[1]) * _leg(t[2], p[2]) for p in pts],
                                               rtol=1e-13, atol=1e-14)]
        assert len(match) == 1
        got.append(match[0])
    assert set(got) == want
    degs = [sum(t) for t in got]
    assert degs == sorted(degs)  # ordered by total degree
    if order <= 2:
        assert got == MODES[order]


@pytest.mark.parametrize("order", [1, 2, 3])
def test_basis_gradients_and_orthogonality(orc, order):
    nm = (order + 1) * (order + 2) * (order + 3) // 6
    xg, wg = npl.leggauss(order + 2)
    M = np.zeros((nm, nm))
    for (a, wa), (b, wb), (c, wc) in itertools.product(zip(xg, wg), repeat=3):
        B, dB = orc.basis(order, [a, b, c])
        M += wa * wb * wc * np.outer(B, B)
        # gradient check against numpy derivatives (mode identification via values)
        for m in range(nm):
            for d in range(3):
                h = 1e-6
                p1, p0 = np.array([a, b, c]), np.array([a, b, c])
                p1[d] += h
                p0[d] -= h
                fd = (orc.basis(order, p1)[0][m] - orc.basis(order, p0)[0][m]) / (2 * h)
                assert abs(dB[m, d] - fd) < 1e-7
    # int_{[-1,1]^3} B_m B_n = delta_mn 8 / prod(2 n_d + 1)  ->  M_nn = |K| / prod(2n_d+1) per unit volume
    assert np.allclose(M - np.diag(np.diag(M)), 0, atol=1e-13)
    if order <= 2:
        want = [8.0 / ((2 * t[0] + 1) * (2 * t[1] + 1) * (2 * t[2] + 1)) for t in MODES[order]]
        np.testing.assert_allclose(np.diag(M), want, rtol=1e-13)


def test_derivatives_exact_at_endpoints(orc):
    # P_n'(+-1) = (+-1)^(n+1) n(n+1)/2 (closed form)
    for r in (-1.0, 1.0):
        B, dB = orc.basis(2, [r, 0.3, -0.2])
        # mode (2,0,0) is index 4: d/dxi P_2(xi) P_0 P_0 = 3 xi
        assert abs(dB[4, 0] - 3 * r) < 1e-15
        assert abs(dB[1, 0] - 1.0) < 1e-15
        assert abs(B[4] - 1.0) < 1e-15  # P_2(+-1) = 1
