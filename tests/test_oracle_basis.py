"""Pins of the oracle's 1D building blocks against closed forms and numpy's
Legendre routines (reading R1/R2: Gauss-Lobatto H1 nodes, Gauss-Legendre L2
nodes and quadrature)."""
import numpy as np
import pytest

import oracle as O
from tests import _fem_ref as R


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre(n)
    xr, wr = R.gauss_legendre01(n)
    assert np.allclose(x, xr, atol=1e-15, rtol=0)
    assert np.allclose(w, wr, atol=1e-15, rtol=0)


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_exact_for_degree_2n_minus_1(n):
    x, w = O.gauss_legendre(n)
    for p in range(2 * n):
        assert abs(np.dot(w, x ** p) - 1.0 / (p + 1)) < 2e-15
    # and not exact one degree higher (the rule has exactly that degree)
    assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-10


def test_gauss_lobatto_closed_forms():
    assert np.array_equal(O.gauss_lobatto(2), [0.0, 1.0])
    assert np.allclose(O.gauss_lobatto(3), [0.0, 0.5, 1.0], atol=1e-16)
    a = (1.0 - 1.0 / np.sqrt(5.0)) / 2.0
    assert np.allclose(O.gauss_lobatto(4), [0.0, a, 1.0 - a, 1.0], atol=1e-15)
    b = (1.0 - np.sqrt(3.0 / 7.0)) / 2.0
    assert np.allclose(O.gauss_lobatto(5), [0.0, b, 0.5, 1.0 - b, 1.0], atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_gauss_lobatto_matches_numpy_roots(n):
    assert np.allclose(O.gauss_lobatto(n), R.gauss_lobatto01(n), atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_lagrange_cardinal_partition_and_reproduction(n):
    nodes = O.gauss_lobatto(n) if n >= 2 else np.array([0.5])
    for a, xa in enumerate(nodes):
        val, _ = O.lagrange(nodes, xa)
        assert np.allclose(val, np.eye(n)[a], atol=1e-15)
    rng = np.random.default_rng(0)
    for t in rng.uniform(0, 1, 7):
        val, der = O.lagrange(nodes, t)
        assert abs(val.sum() - 1.0) < 1e-14
        assert abs(der.sum()) < 1e-12
        for p in range(n):
            # interpolation of t^p is exact up to degree n-1
            assert abs(np.dot(val, nodes ** p) - t ** p) < 1e-14
            if p >= 1:
                assert abs(np.dot(der, nodes ** p) - p * t ** (p - 1)) < 1e-12


def test_lagrange_matches_numpy_polynomials():
    nodes = O.gauss_lobatto(4)
    polys = R.lagrange_polys(nodes)
    from numpy.polynomial import polynomial as P
    for t in (0.0, 0.13, 0.5, 0.77, 1.0):
        val, der = O.lagrange(nodes, t)
        assert np.allclose(val, [P.polyval(t, c) for c in polys], atol=1e-14)
        assert np.allclose(der, [P.polyval(t, P.polyder(c)) for c in polys], atol=1e-12)


def test_sym_min_eig_vs_numpy():
    rng = np.random.default_rng(1)
    for d in (2, 3):
        for _ in range(200):
            A = rng.normal(size=(d, d))
            A = A + A.T
            lam, s = O.sym_min_eig(A)
            w, V = np.linalg.eigh(A)
            assert abs(lam - w[0]) < 1e-13 * max(1.0, abs(w).max())
            assert abs(np.linalg.norm(s) - 1.0) < 1e-14
            if w[1] - w[0] > 1e-6:
                assert abs(abs(np.dot(s, V[:, 0])) - 1.0) < 1e-10


def test_sym_min_eig_ties_take_lowest_index():
    lam, s = O.sym_min_eig(np.diag([2.0, 2.0]))
    assert lam == 2.0 and np.array_equal(s, [1.0, 0.0])
    lam, s = O.sym_min_eig(np.zeros((3, 3)))
    assert lam == 0.0 and np.array_equal(s, [1.0, 0.0, 0.0])
    lam, s = O.sym_min_eig(np.diag([3.0, -1.0, 5.0]))
    assert lam == -1.0 and np.allclose(np.abs(s), [0.0, 1.0, 0.0])
