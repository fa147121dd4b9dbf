"""Pins for the oracle's 1D rules and Lagrange bases (Sec. 2.5, Eq. colocated;
Sec. 1.2, Eq. tpps).  Closed forms, exactness on monomials, the paper's RTCF_2
figure, and a library routine (numpy's Gauss-Legendre) as an outside check."""
import os
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")

s3, s15, s5, s21 = np.sqrt(3.0), np.sqrt(15.0), np.sqrt(5.0), np.sqrt(21.0)
CLOSED_GL = {
    1: ([0.5], [1.0]),
    2: ([0.5 - s3 / 6, 0.5 + s3 / 6], [0.5, 0.5]),
    3: ([0.5 - s15 / 10, 0.5, 0.5 + s15 / 10], [5 / 18, 4 / 9, 5 / 18]),
}
CLOSED_GLL = {
    2: ([0.0, 1.0], [0.5, 0.5]),
    3: ([0.0, 0.5, 1.0], [1 / 6, 2 / 3, 1 / 6]),
    4: ([0.0, 0.5 - s5 / 10, 0.5 + s5 / 10, 1.0], [1 / 12, 5 / 12, 5 / 12, 1 / 12]),
    5: ([0.0, 0.5 - s21 / 14, 0.5, 0.5 + s21 / 14, 1.0], [1 / 20, 49 / 180, 16 / 45, 49 / 180, 1 / 20]),
}


@pytest.mark.parametrize("n", sorted(CLOSED_GL))
def test_gauss_legendre_closed_forms(orc, n):
    x, w = orc.gauss_legendre(n)
    np.testing.assert_allclose(x, CLOSED_GL[n][0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, CLOSED_GL[n][1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", sorted(CLOSED_GLL))
def test_gauss_lobatto_closed_forms(orc, n):
    x, w = orc.gauss_lobatto(n)
    np.testing.assert_allclose(x, CLOSED_GLL[n][0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, CLOSED_GLL[n][1], rtol=0, atol=1e-15)


def test_rtcf2_figure_nodes(orc):
    """The RTCF_2 figure (Sec. 3.5) fixes the reference interval [0,1], GLL
    nodes for the continuous P_2 factor and Gauss nodes for the dP_1 factor."""
    rows = [l.split() for l in open(os.path.join(GOLD, "rtcf2_nodes.txt")) if l.strip() and l[0] != "#"]
    for kind, n, v in rows:
        x, _ = (orc.gauss_lobatto if kind == "GLL" else orc.gauss_legendre)(int(n))
        assert np.min(np.abs(x - float(v))) < 5e-4, (kind, n, v, x)


@pytest.mark.parametrize("n", range(1, 17))
def test_gauss_legendre_exactness(orc, n):
    x, w = orc.gauss_legendre(n)
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.all(np.diff(x) > 0) and x[0] > 0 and x[-1] < 1
    for k in range(2 * n):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 5e-15, k
    # the error on x^(2n) is the closed form (n!)^4 / ((2n+1) ((2n)!)^2)
    # (the Gauss remainder term on [0,1] with f^(2n) = (2n)!)
    err = 1.0 / (2 * n + 1) - np.dot(w, x ** (2 * n))
    exact = float(Fraction(factorial(n) ** 4, (2 * n + 1) * factorial(2 * n) ** 2))
    assert abs(err - exact) < 1e-6 * exact + 5e-15


@pytest.mark.parametrize("n", range(2, 17))
def test_gauss_lobatto_exactness(orc, n):
    x, w = orc.gauss_lobatto(n)
    assert x[0] == 0.0 and x[-1] == 1.0
    assert abs(w.sum() - 1.0) < 1e-14
    for k in range(2 * n - 2):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 5e-15, k
    # Lobatto remainder on [0,1] for x^(2n-2): -n (n-1)^3 ((n-2)!)^4 / ((2n-1) ((2n-2)!)^2)
    err = 1.0 / (2 * n - 1) - np.dot(w, x ** (2 * n - 2))
    exact = -float(Fraction(n * (n - 1) ** 3 * factorial(n - 2) ** 4,
                            (2 * n - 1) * factorial(2 * n - 2) ** 2))
    assert abs(err - exact) < 1e-6 * abs(exact) + 5e-15


@pytest.mark.parametrize("n", [4, 9, 17, 24])
def test_gauss_legendre_matches_numpy(orc, n):
    t, v = np.polynomial.legendre.leggauss(n)
    x, w = orc.gauss_legendre(n)
    np.testing.assert_allclose(x, 0.5 * (t + 1), rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, 0.5 * v, rtol=0, atol=2e-15)


@pytest.mark.parametrize("kind,n", [("GLL", 2), ("GLL", 5), ("GLL", 9), ("GL", 1), ("GL", 4), ("GL", 8)])
def test_lagrange_basis(orc, kind, n):
    nodes, _ = (orc.gauss_lobatto if kind == "GLL" else orc.gauss_legendre)(n)
    for i in range(n):
        for j in range(n):
            assert abs(orc.lagrange(nodes, i, nodes[j]) - (1.0 if i == j else 0.0)) < 1e-14
    rng = np.random.default_rng(0)
    for t in rng.random(7):
        assert abs(sum(orc.lagrange(nodes, i, t) for i in range(n)) - 1.0) < 1e-13
        assert abs(sum(orc.lagrange(nodes, i, t, deriv=True) for i in range(n))) < 1e-11
        # derivative of the interpolant of t^k is k t^(k-1) for k < n
        for k in range(1, n):
            d = sum(nodes[i] ** k * orc.lagrange(nodes, i, t, deriv=True) for i in range(n))
            assert abs(d - k * t ** (k - 1)) < 1e-10 * max(1, k * k)


def test_lagrange_exact_rational(orc):
    """On the rational GLL_3 nodes {0, 1/2, 1} the basis and its derivative at
    t = 1/3 are known exactly."""
    nodes = [0.0, 0.5, 1.0]
    t = Fraction(1, 3)
    xs = [Fraction(0), Fraction(1, 2), Fraction(1)]
    for i in range(3):
        v = Fraction(1)
        for k in range(3):
            if k != i:
                v *= (t - xs[k]) / (xs[i] - xs[k])
        assert abs(orc.lagrange(nodes, i, 1 / 3) - float(v)) < 1e-15
    # phi_0 = (2t-1)(t-1) -> phi_0' = 4t - 3 ; phi_1 = 4t(1-t) -> 4 - 8t ; phi_2 = t(2t-1) -> 4t - 1
    for i, d in enumerate([4 / 3 - 3, 4 - 8 / 3, 4 / 3 - 1]):
        assert abs(orc.lagrange(nodes, i, 1 / 3, deriv=True) - d) < 1e-14


def test_paper_dense_tensor_size(orc):
    """Sec. 4.2: the dense local Laplace tensor at degree 16 takes 193 MB."""
    facts = dict(l.split() for l in open(os.path.join(GOLD, "paper_facts.txt")) if l.strip() and l[0] != "#")
    _, nloc = orc.space_size("Q", 16, (1, 1, 1))
    assert round(nloc * nloc * 8 / 1e6) == int(facts["dense_local_tensor_MB_degree16"])
