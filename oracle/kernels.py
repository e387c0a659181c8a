"""Parametric kernel functions kappa(x, y; theta) (§1, §6 kernel table).

Test infrastructure only (see ``oracle/__init__.py``).

All functions broadcast: x and y have a trailing axis of length d, theta a
trailing axis of length d_theta; the leading axes broadcast against each other.

* gauss       exp(-r^2 / (2 l^2)),                           theta = (l,)
* matern32    (1 + sqrt(3) r / l) exp(-sqrt(3) r / l),         theta = (l,)
* matern52    (1 + sqrt(5) r/l + 5 r^2/(3 l^2)) exp(-sqrt(5) r/l), theta = (l,)
* aniso_gauss exp(-sum_k (x_k - y_k)^2 / (2 l_k^2)),          theta = (l_1..l_d)
* se          exp(-(r / l)^2)            (the paper's SE kernel)
* exponential exp(-r / l)                (the paper's E kernel)
* mc          (1 + (r / l)^2)^(1/2)      (the paper's multiquadric)
* poly        1 + theta r^2 + theta^2 r^4 (test kernel: polynomial of degree 4 in
              each coordinate and 2 in theta, translation-invariant)
* polyxy      (1 + x.y)^2 (1 + theta)     (test kernel that is NOT
              translation-invariant)
* poly2       1 + theta_1 r^2 + theta_2^2 r^4 (two-parameter test kernel: degree 4 in each
              coordinate, 1 in theta_1 and 2 in theta_2, translation-invariant)

Pins (tests/test_oracle_basics.py): the Matern closed forms against the
general Matern formula with SciPy's Bessel K_nu at nu = 3/2 and 5/2; r = 0
values; symmetry in (x, y).
"""
from __future__ import annotations

import numpy as np

TRANSLATION_INVARIANT = {
    "gauss": True, "matern32": True, "matern52": True, "aniso_gauss": True,
    "se": True, "exponential": True, "mc": True, "poly": True, "polyxy": False, "poly2": True,
}


def _dist(x, y):
    diff = np.asarray(x, float) - np.asarray(y, float)
    return np.sqrt(np.sum(diff * diff, axis=-1)), diff


def kappa(name: str, x, y, theta):
    """Evaluate kernel ``name`` at (x, y; theta) with broadcasting."""
    theta = np.asarray(theta, float)
    r, diff = _dist(x, y)
    t0 = theta[..., 0]
    if name == "gauss":
        return np.exp(-(r * r) / (2.0 * t0 * t0))
    if name == "matern32":
        s = np.sqrt(3.0) * r / t0
        return (1.0 + s) * np.exp(-s)
    if name == "matern52":
        s = np.sqrt(5.0) * r / t0
        return (1.0 + s + s * s / 3.0) * np.exp(-s)
    if name == "aniso_gauss":
        q = np.sum(diff * diff / (2.0 * theta * theta), axis=-1)
        return np.exp(-q)
    if name == "se":
        return np.exp(-(r / t0) ** 2)
    if name == "exponential":
        return np.exp(-r / t0)
    if name == "mc":
        return np.sqrt(1.0 + (r / t0) ** 2)
    if name == "poly":
        r2 = r * r
        return 1.0 + t0 * r2 + t0 * t0 * r2 * r2
    if name == "poly2":
        r2 = r * r
        return 1.0 + theta[..., 0] * r2 + theta[..., 1] ** 2 * r2 * r2
    if name == "polyxy":
        dot = np.sum(np.asarray(x, float) * np.asarray(y, float), axis=-1)
        return (1.0 + dot) ** 2 * (1.0 + t0)
    raise ValueError(f"unknown kernel {name!r}")


def dense_matrix(name: str, points: np.ndarray, theta) -> np.ndarray:
    """K(X, X; theta) with [K]_ij = kappa(x_i, x_j; theta) (§1), formed entry by entry."""
    P = np.asarray(points, float)
    return kappa(name, P[:, None, :], P[None, :, :], np.asarray(theta, float))


def dense_apply(name: str, points: np.ndarray, theta, X: np.ndarray, rows=None,
                chunk: int = 512) -> np.ndarray:
    """Brute-force K(X, X; theta) @ X (the exact product the method approximates).

    ``rows`` restricts the output to those row indices (the paper's row-subset
    error estimator of §6 uses 200 random rows).  Evaluated in row chunks so
    that memory stays bounded.
    """
    P = np.asarray(points, float)
    X = np.asarray(X, float)
    rows = np.arange(P.shape[0]) if rows is None else np.asarray(rows)
    out = np.empty((rows.size,) + X.shape[1:])
    th = np.asarray(theta, float)
    for s in range(0, rows.size, chunk):
        rr = rows[s:s + chunk]
        K = kappa(name, P[rr][:, None, :], P[None, :, :], th)
        out[s:s + chunk] = K @ X
    return out
