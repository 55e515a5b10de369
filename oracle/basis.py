"""1D tables for tensor-product Q_p elements (oracle; test infrastructure only).

Sec. 3.2 of the paper: shape functions are tensor products of 1D Lagrange polynomials; the 1D
number of DoFs and of Gauss points is k = p + 1 (written n here).  The DG experiments use nodal
Lagrange polynomials in the Gauss-Lobatto points (the delta property noted after Eq. sum_factorization_face, Sec. 3.2).

Everything here is written from the definitions:
  * Gauss-Legendre: roots of the Legendre polynomial P_n by Newton iteration on the three-term
    recurrence, weights 2 / ((1 - x^2) P_n'(x)^2), mapped from [-1, 1] to [0, 1].
  * Gauss-Lobatto: the end points plus the roots of P'_{n-1}.
  * Lagrange polynomials: product form prod_{m != i} (x - x_m) / (x_i - x_m), differentiated
    by the product rule.
"""
import itertools
import math

import numpy as np


def _legendre_and_derivs(n, x):
    """P_n(x), P_n'(x), P_n''(x) by the Bonnet recurrence and the Legendre ODE."""
    p0, p1 = 1.0, x
    if n == 0:
        return 1.0, 0.0, 0.0
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    # (1 - x^2) P_n' = n (P_{n-1} - x P_n)
    dp = n * (p0 - x * p1) / (1.0 - x * x)
    # (1 - x^2) P_n'' = 2 x P_n' - n (n + 1) P_n
    d2p = (2.0 * x * dp - n * (n + 1) * p1) / (1.0 - x * x)
    return p1, dp, d2p


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0, 1] (nodes ascending, weights)."""
    if n < 1:
        raise ValueError("n >= 1")
    xs = []
    ws = []
    for i in range(n):
        # Chebyshev-like initial guess for the i-th root (descending on [-1, 1])
        x = math.cos(math.pi * (i + 0.75) / (n + 0.5))
        for _ in range(100):
            p, dp, _ = _legendre_and_derivs(n, x)
            dx = p / dp
            x -= dx
            if abs(dx) < 1e-16:
                break
        _, dp, _ = _legendre_and_derivs(n, x)
        xs.append(x)
        ws.append(2.0 / ((1.0 - x * x) * dp * dp))
    xs = np.array(xs)
    ws = np.array(ws)
    order = np.argsort(xs)
    return 0.5 * (1.0 + xs[order]), 0.5 * ws[order]


def gauss_lobatto_nodes(n):
    """n Gauss-Lobatto points on [0, 1]: 0, 1 and the roots of P'_{n-1} (ascending)."""
    if n < 2:
        raise ValueError("Gauss-Lobatto needs n >= 2")
    m = n - 1
    interior = []
    for i in range(1, m):
        # initial guess: Chebyshev-Gauss-Lobatto point
        x = -math.cos(math.pi * i / m)
        for _ in range(100):
            _, dp, d2p = _legendre_and_derivs(m, x)
            dx = dp / d2p
            x -= dx
            if abs(dx) < 1e-16:
                break
        interior.append(x)
    xs = np.array([-1.0] + sorted(interior) + [1.0])
    return 0.5 * (1.0 + xs)


def lagrange_eval(nodes, xs, order=0):
    """Matrix V[q, i] = d^order/dx^order phi_i(xs[q]) for the Lagrange basis on `nodes`.

    phi_i(x) = prod_{m != i} (x - x_m) / (x_i - x_m).  Each factor is linear, so the j-th
    derivative is j! times the sum, over all ways to drop j of the factors, of the product of
    the remaining ones (product rule), divided by the same denominator.
    """
    xs = np.atleast_1d(np.asarray(xs, dtype=np.float64))
    n = len(nodes)
    V = np.zeros((len(xs), n))
    for i in range(n):
        others = [nodes[m] for m in range(n) if m != i]
        denom = 1.0
        for xm in others:
            denom *= nodes[i] - xm
        if order > len(others):
            continue
        total = np.zeros(len(xs))
        for dropped in itertools.combinations(range(len(others)), order):
            prod = np.ones(len(xs))
            for m, xm in enumerate(others):
                if m not in dropped:
                    prod = prod * (xs - xm)
            total += prod
        V[:, i] = math.factorial(order) * total / denom
    return V
