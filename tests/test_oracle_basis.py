"""Pins of the oracle's 1D tables against library routines and closed forms (CPU)."""
import math

import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_legendre_matches_numpy_and_is_exact(n):
    g, w = basis.gauss_legendre(n)
    x, ww = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(g, 0.5 * (x + 1.0), rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * ww, rtol=0, atol=2e-15)
    # exact for monomials up to degree 2n - 1 on [0, 1]
    for k in range(2 * n):
        assert abs(np.sum(w * g ** k) - 1.0 / (k + 1)) < 1e-15


def test_gauss_lobatto_closed_forms():
    np.testing.assert_allclose(basis.gauss_lobatto_nodes(2), [0.0, 1.0], atol=0)
    np.testing.assert_allclose(basis.gauss_lobatto_nodes(3), [0.0, 0.5, 1.0], atol=1e-16)
    a = 0.5 / math.sqrt(5.0)
    np.testing.assert_allclose(basis.gauss_lobatto_nodes(4), [0.0, 0.5 - a, 0.5 + a, 1.0], atol=1e-16)
    b = 0.5 * math.sqrt(3.0 / 7.0)
    np.testing.assert_allclose(basis.gauss_lobatto_nodes(5), [0.0, 0.5 - b, 0.5, 0.5 + b, 1.0],
                               atol=1e-16)


@pytest.mark.parametrize("n", range(2, 10))
def test_gauss_lobatto_nodes_are_roots_of_legendre_derivative(n):
    """Interior nodes are the roots of P'_{n-1}; the Lobatto rule is then exact to degree 2n-3."""
    nodes = basis.gauss_lobatto_nodes(n)
    t = 2.0 * nodes - 1.0
    dP = np.polynomial.legendre.Legendre.basis(n - 1).deriv()
    if n > 2:
        assert np.max(np.abs(dP(t[1:-1]))) < 1e-11 * max(1.0, np.max(np.abs(dP.coef)))
    P = np.polynomial.legendre.Legendre.basis(n - 1)
    w = 2.0 / (n * (n - 1) * P(t) ** 2)  # weights on [-1, 1]
    for k in range(2 * n - 2):
        exact = (1.0 - (-1.0) ** (k + 1)) / (k + 1)
        assert abs(np.sum(w * t ** k) - exact) < 1e-13


@pytest.mark.parametrize("n", range(2, 10))
def test_lagrange_delta_and_monomial_reproduction(n):
    nodes = basis.gauss_lobatto_nodes(n)
    np.testing.assert_allclose(basis.lagrange_eval(nodes, nodes), np.eye(n), atol=1e-14)
    xs = np.linspace(-0.1, 1.1, 13)
    for order in range(0, n + 1):
        V = basis.lagrange_eval(nodes, xs, order)
        for k in range(n):
            # sum_i x_i^k phi_i^(order)(x) = d^order/dx^order x^k  (exact for k <= n - 1)
            got = V @ nodes ** k
            if order > k:
                want = np.zeros_like(xs)
            else:
                want = math.factorial(k) / math.factorial(k - order) * xs ** (k - order)
            scale = max(1.0, np.max(np.abs(V)))
            assert np.max(np.abs(got - want)) < 1e-12 * scale


def test_lagrange_matches_independent_polynomial_fit():
    """Derivatives of every order vs numpy.polynomial fitted through the delta conditions."""
    n = 6
    nodes = basis.gauss_lobatto_nodes(n)
    xs = np.linspace(0.0, 1.0, 11)
    for i in range(n):
        yi = np.zeros(n)
        yi[i] = 1.0
        poly = np.polynomial.Polynomial.fit(nodes, yi, n - 1, domain=[0, 1], window=[0, 1])
        for order in range(n):
            got = basis.lagrange_eval(nodes, xs, order)[:, i]
            want = poly.deriv(order)(xs) if order else poly(xs)
            assert np.max(np.abs(got - want)) < 1e-9 * max(1.0, np.max(np.abs(want)))
