"""Seeded synthetic workloads for the parametric H / H^2 online stage.

This module only draws random numbers and names workload shapes. It holds none
of the method's arithmetic (no kernel, no interpolation, no compression), so
both the CUDA path and the independent FP64 oracle can take their inputs from
it without sharing any computation.

Every generator uses NumPy's PCG64 (``numpy.random.default_rng(seed)``).  The
paper draws its point sets uniformly from the unit hypercube (§6, "Domain") and
its parameters uniformly from the parameter box (§6, "Error Calculation").
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def uniform_points(n: int, d: int, seed: int) -> np.ndarray:
    """n points drawn uniformly from [0, 1]^d, shape (n, d), float64, row-major."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.random((n, d)))


def gaussian_rhs(n: int, m: int, seed: int) -> np.ndarray:
    """m right-hand sides with i.i.d. N(0, 1) entries, shape (n, m), float64."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, m))


def uniform_rhs(n: int, m: int, seed: int) -> np.ndarray:
    """m right-hand sides with entries from U[0, 1] (the paper's error vector, §6)."""
    rng = np.random.default_rng(seed)
    return rng.random((n, m))


def uniform_thetas(lo, hi, count: int, seed: int) -> np.ndarray:
    """count parameters drawn uniformly from the box [lo, hi], shape (count, dtheta)."""
    lo = np.atleast_1d(np.asarray(lo, float))
    hi = np.atleast_1d(np.asarray(hi, float))
    rng = np.random.default_rng(seed)
    return lo + (hi - lo) * rng.random((count, lo.size))


def gaussian_mixture_points(n: int, d: int, components: int, seed: int) -> np.ndarray:
    """n points in [0,1]^d from an equal-weight mixture of anisotropic Gaussians: means uniform in
    [0.1, 0.9]^d, per-component axis standard deviations log-uniform in [0.005, 0.05], a random
    rotation per component (the Q factor of a Gaussian matrix, signs fixed by R's diagonal),
    points clipped to the unit cube."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(0.1, 0.9, (components, d))
    sds = np.exp(rng.uniform(np.log(0.005), np.log(0.05), (components, d)))
    rots = []
    for _ in range(components):
        Q, R = np.linalg.qr(rng.standard_normal((d, d)))
        rots.append(Q * np.sign(np.diag(R)))
    which = rng.integers(0, components, n)
    Z = rng.standard_normal((n, d))
    P = np.empty((n, d))
    for c in range(components):
        sel = which == c
        P[sel] = means[c] + (Z[sel] * sds[c]) @ rots[c].T
    return np.clip(P, 0.0, 1.0)


def sample_rows(n: int, count: int, seed: int) -> np.ndarray:
    """count distinct row indices drawn uniformly from 0..n-1, sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(count, n), replace=False))


@dataclass(frozen=True)
class Workload:
    """One synthetic configuration of the online stage.

    kernel     -- kernel name ("gauss", "matern32", "matern52", ...)
    theta_lo/hi -- the parameter box B_theta
    degree     -- Chebyshev degree in theta per parameter dimension (p_theta = degree + 1)
    p_s        -- spatial Chebyshev nodes per dimension
    l_max      -- depth of the uniform cluster tree
    eta        -- admissibility parameter
    tol        -- TT truncation tolerance
    rank_cap   -- cap on every far-field TT rank
    fmt        -- "h2" or "h"
    precision  -- "fp64" or "fp32"
    """

    name: str
    n: int
    d: int
    kernel: str
    theta_lo: tuple
    theta_hi: tuple
    degree: tuple
    p_s: int
    l_max: int
    eta: float
    tol: float
    rank_cap: int
    fmt: str
    precision: str
    m: int
    point_seed: int
    rhs_seed: int
    theta_seed: int
    theta: tuple = field(default=())
    near_degree: tuple = field(default=())  # the near field's own grid (empty: degree)

    def points(self) -> np.ndarray:
        return uniform_points(self.n, self.d, self.point_seed)

    def rhs(self) -> np.ndarray:
        return gaussian_rhs(self.n, self.m, self.rhs_seed)

    def thetas(self, count: int) -> np.ndarray:
        if self.theta and count == 1:
            return np.asarray([self.theta], float)
        return uniform_thetas(self.theta_lo, self.theta_hi, count, self.theta_seed)


# Plain method, small, FP64: n = 4096 uniform points in [0,1]^2, Gaussian
# exp(-r^2/(2 l^2)) with l in [0.1, 1], degree 16, eta = 1, leaf 64 (l_max = 3),
# far-field TT rank <= 32, theta = 0.37, one N(0,1) right-hand side.
SMALL_2D_GAUSS_H2 = Workload(
    name="n4096_d2_gauss_h2_fp64", n=4096, d=2, kernel="gauss",
    theta_lo=(0.1,), theta_hi=(1.0,), degree=(16,), p_s=8, l_max=3, eta=1.0,
    tol=1e-5, rank_cap=32, fmt="h2", precision="fp64", m=1,
    point_seed=1001, rhs_seed=2001, theta_seed=3001, theta=(0.37,))

SMALL_2D_GAUSS_H = Workload(
    name="n4096_d2_gauss_h_fp64", n=4096, d=2, kernel="gauss",
    theta_lo=(0.1,), theta_hi=(1.0,), degree=(16,), p_s=15, l_max=3, eta=1.0,
    tol=1e-5, rank_cap=32, fmt="h", precision="fp64", m=1,
    point_seed=1001, rhs_seed=2001, theta_seed=3001, theta=(0.37,))

# Plain method on the GPU, FP32, H^2: n = 65536 uniform points in [0,1]^3,
# Matern nu = 3/2 with l in [0.05, 0.5], degree 20, p_s = 8, rank <= 64,
# l_max = 3 (mean leaf 128), eta = sqrt(3), 16 N(0,1) right-hand sides.
LARGE_3D_MATERN_H2 = Workload(
    name="n65536_d3_matern32_h2_fp32_m16", n=65536, d=3, kernel="matern32",
    theta_lo=(0.05,), theta_hi=(0.5,), degree=(20,), p_s=8, l_max=3,
    eta=float(np.sqrt(3.0)), tol=1e-5, rank_cap=64, fmt="h2", precision="fp32",
    m=16, point_seed=1002, rhs_seed=2002, theta_seed=3002)

# Differentiation: n = 262144 uniform points in [0,1]^2, anisotropic Gaussian with
# (l_1, l_2) in [0.05, 0.5]^2, tensor Chebyshev degree 12 x 12, p_s = 8, l_max = 6 (mean
# leaf 64), eta = sqrt(2), rank <= 64, FP32, 8 N(0,1) right-hand sides.
DIFF_2D_ANISO = Workload(
    name="n262144_d2_aniso_gauss_h2_fp32_m8", n=262144, d=2, kernel="aniso_gauss",
    theta_lo=(0.05, 0.05), theta_hi=(0.5, 0.5), degree=(12, 12), p_s=8, l_max=6,
    eta=float(np.sqrt(2.0)), tol=1e-5, rank_cap=64, fmt="h2", precision="fp32",
    m=8, point_seed=1004, rhs_seed=2004, theta_seed=3004)

# Learned surrogate: n = 65536 uniform points in [0,1]^3, anisotropic Gaussian with
# (l_1, l_2, l_3) in [0.05, 0.5]^3, near-field degree 4 (125 grid points), far-field
# degree 8 (729 grid points, the polynomial path the network is compared with), p_s = 4
# (with p_s = 8 the offline TT-SVD of the 632 far tensors of 512 x 729 x 512 entries takes
# about ten minutes; network and polynomial share the spatial factors either way), l_max = 3,
# eta = sqrt(3), rank <= 64, FP32, 16 N(0,1) right-hand sides.
SURROGATE_3D_ANISO = Workload(
    name="n65536_d3_aniso_gauss_ps4_h2_fp32_m16", n=65536, d=3, kernel="aniso_gauss",
    theta_lo=(0.05, 0.05, 0.05), theta_hi=(0.5, 0.5, 0.5), degree=(8, 8, 8), p_s=4, l_max=3,
    eta=float(np.sqrt(3.0)), tol=1e-5, rank_cap=64, fmt="h2", precision="fp32",
    m=16, point_seed=1005, rhs_seed=2005, theta_seed=3005, near_degree=(4, 4, 4))

WORKLOADS = {w.name: w for w in (SMALL_2D_GAUSS_H2, SMALL_2D_GAUSS_H, LARGE_3D_MATERN_H2, DIFF_2D_ANISO,
                                 SURROGATE_3D_ANISO)}
