"""Chebyshev nodes of the first kind and Lagrange polynomials (§2.2).

Test infrastructure only (see ``oracle/__init__.py``).

Pins (tests/test_oracle_basics.py): node set equals NumPy's first-kind
Chebyshev points mapped to [a, b]; ell_k(eta_j) = delta_kj; sum_k ell_k = 1;
exact reproduction of polynomials of degree < p.  Derivatives: sum_k ell_k' = 0,
sum_k f(eta_k) ell_k'(x) = f'(x) for polynomials of degree < p (NumPy's polyder),
central differences of ``lagrange``.
"""
from __future__ import annotations

import numpy as np


def cheb_nodes(a: float, b: float, p: int) -> np.ndarray:
    """The p Chebyshev nodes of the first kind on [a, b], ascending (§2.2).

    eta_k = (a + b)/2 - (b - a)/2 * cos((2k - 1) pi / (2p)),  k = 1..p.
    """
    k = np.arange(1, p + 1, dtype=float)
    return 0.5 * (a + b) - 0.5 * (b - a) * np.cos((2.0 * k - 1.0) * np.pi / (2.0 * p))


def lagrange(nodes: np.ndarray, x) -> np.ndarray:
    """Values of the degree p-1 Lagrange polynomials, by the product formula of §2.2.

    Returns L with L[i, k] = ell_k(x_i) = prod_{j != k} (x_i - eta_j) / (eta_k - eta_j).
    At a node the result is an exact unit row.
    """
    x = np.atleast_1d(np.asarray(x, dtype=float)).ravel()
    p = len(nodes)
    L = np.ones((x.size, p))
    for k in range(p):
        for j in range(p):
            if j != k:
                L[:, k] *= (x - nodes[j]) / (nodes[k] - nodes[j])
    return L


def lagrange_derivative(nodes: np.ndarray, x) -> np.ndarray:
    """Derivatives of the Lagrange polynomials of ``lagrange``, by the product rule:

    ell_k'(x) = sum_{m != k} 1 / (eta_k - eta_m) * prod_{j != k, m} (x - eta_j) / (eta_k - eta_j).
    Returns Ld with Ld[i, k] = ell_k'(x_i); valid at the nodes too.
    """
    x = np.atleast_1d(np.asarray(x, dtype=float)).ravel()
    p = len(nodes)
    Ld = np.zeros((x.size, p))
    for k in range(p):
        for m in range(p):
            if m == k:
                continue
            term = np.full(x.size, 1.0 / (nodes[k] - nodes[m]))
            for j in range(p):
                if j != k and j != m:
                    term *= (x - nodes[j]) / (nodes[k] - nodes[j])
            Ld[:, k] += term
    return Ld


def parametric_vectors(theta, lo, hi, degree, deriv=None) -> list:
    """The parametric vectors v_i(theta_i) of App. A.4: [v_i]_k = ell_k on [lo_i, hi_i] at theta_i.

    degree[i] is the Chebyshev degree of parameter dimension i, so p_theta = degree + 1 nodes.
    With ``deriv = i`` dimension i carries d/dtheta_i of its Lagrange polynomials instead: the
    instantiated matrix is linear in each v_i, so this instantiates dK_hat/dtheta_i.
    """
    theta = np.atleast_1d(np.asarray(theta, float))
    out = []
    for i in range(theta.size):
        nodes = cheb_nodes(lo[i], hi[i], int(degree[i]) + 1)
        if deriv is not None and i == deriv:
            out.append(lagrange_derivative(nodes, theta[i])[0])
        else:
            out.append(lagrange(nodes, theta[i])[0])
    return out
