"""Pins for the oracle's surrogate pieces: the FP64 perceptron (oracle.mlp), the projected far-field
cores H*_b(theta) (ParametricMatrix.projected_cores) and a near field on its own theta grid.

Each pin compares with something outside the code it checks: SciPy's normal distribution,
printed values of Phi, central differences, the closed form of Adam's first step, the
non-parametric coupling matrix W_b of §3.6.2, the dense K(theta) X of the polynomial kernel."""
import math

import numpy as np
import pytest

from oracle import cheb, kernels, mlp, pmatrix
from paper_2511_03109_gb300 import inputs


def test_gelu_is_x_times_the_normal_distribution_function():
    scipy_stats = pytest.importorskip("scipy.stats")
    x = np.linspace(-6.0, 6.0, 121)
    np.testing.assert_allclose(mlp.gelu(x), x * scipy_stats.norm.cdf(x), rtol=1e-14, atol=1e-300)
    # Phi(1) = 0.8413447460685429, Phi(-1) = 0.15865525393145705, Phi(2) = 0.9772498680518208
    np.testing.assert_allclose(mlp.gelu([1.0, -1.0, 2.0]),
                               [0.8413447460685429, -0.15865525393145705, 2 * 0.9772498680518208], rtol=1e-15)
    assert mlp.gelu(0.0) == 0.0 and abs(mlp.gelu_grad(0.0) - 0.5) < 1e-16
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-9)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(5)
    p = mlp.init_params(3, 7, 5, seed=11)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.3 * rng.standard_normal(p[k].shape)
    U = rng.uniform(-1, 1, (4, 3))
    T = rng.standard_normal((4, 5))
    _, g = mlp.loss_and_grad(p, U, T)
    h = 1e-6
    for k in p:
        num = np.zeros_like(p[k])
        for idx in np.ndindex(p[k].shape):
            old = p[k][idx]
            p[k][idx] = old + h
            lp = mlp.loss(p, U, T)
            p[k][idx] = old - h
            lm = mlp.loss(p, U, T)
            p[k][idx] = old
            num[idx] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(g[k], num, rtol=1e-6, atol=1e-10, err_msg=k)


def test_zero_second_layer_returns_the_output_bias():
    p = mlp.init_params(2, 6, 4, seed=3)
    p["W2"][:] = 0.0
    p["b2"][:] = 0.0
    p["b3"] = np.array([0.5, -1.0, 2.0, 0.0])
    Y, _ = mlp.forward(p, np.random.default_rng(0).uniform(-1, 1, (3, 2)))
    np.testing.assert_array_equal(Y, np.tile(p["b3"], (3, 1)))  # gelu(0) = 0 exactly


def test_first_adam_step_moves_by_lr_times_the_sign():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -1e-3, 4.0])}
    mlp.adam_step(p, g, {}, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], rtol=1e-15)


def test_normalise_maps_the_box_to_the_unit_cube():
    U = mlp.normalise([[0.05, 0.5, 0.275]], [0.05, 0.05, 0.05], [0.5, 0.5, 0.5])
    np.testing.assert_allclose(U, [[-1.0, 1.0, 0.0]], atol=1e-15)


def _model(kernel, lo, hi, degree, tol, near_degree=None, n=260, d=2, seed=21, p_s=4):
    P = inputs.uniform_points(n, d, seed)
    return pmatrix.ParametricMatrix(P, kernel, lo, hi, degree, p_s, 2, 1.0, tol, fmt="h2", near_degree=near_degree)


def _W(b, kernel, theta, p_s):
    """W_b(theta)[i, j] = kappa(eta^s_i, eta^t_j; theta), little-endian multi-indices (§3.6.2)."""
    d = b.s.lo.size
    ps = np.empty((p_s ** d, d))
    pt = np.empty((p_s ** d, d))
    for flat in range(p_s ** d):
        idx = [(flat // p_s ** k) % p_s for k in range(d)]
        ps[flat] = [cheb.cheb_nodes(b.s.lo[k], b.s.hi[k], p_s)[idx[k]] for k in range(d)]
        pt[flat] = [cheb.cheb_nodes(b.t.lo[k], b.t.hi[k], p_s)[idx[k]] for k in range(d)]
    return kernels.kappa(kernel, ps[:, None], pt[None], theta)


def test_projected_cores_equal_the_interpolated_ones_at_a_node():
    """No truncation, theta at a Chebyshev node: M_b(theta) = L_b H_b(theta) R_b^T exactly, so the
    least-squares core is H_b(theta) itself.  The untruncated factors keep directions whose singular
    values are at rounding level, where H is not determined to rounding; so the gauge-invariant
    couplings L H* R^T, L H R^T and W_b are compared (to 1e-12)."""
    M = _model("gauss", [0.2], [1.0], [4], 0.0)
    M.offline()
    th = [cheb.cheb_nodes(0.2, 1.0, 5)[3]]
    inst = M.instantiate(th)
    Hs = M.projected_cores(th)
    for b in M.far[:10]:
        W = _W(b, "gauss", th, 4)
        Cs = b.L @ Hs[id(b)] @ b.R.T
        np.testing.assert_allclose(Cs, W, atol=1e-12 * np.abs(W).max())
        np.testing.assert_allclose(Cs, M.coupling(b, inst), atol=1e-12 * np.abs(W).max())


def test_projected_coupling_is_the_least_squares_fit():
    """Between nodes and with truncation, L_b H* R_b^T is the best fit to W_b(theta) in the spans of
    L_b and R_b: the residual is orthogonal to both (L^T (W - L H* R^T) R = 0), and it is no worse
    than the interpolated core's."""
    M = _model("matern32", [0.1], [0.6], [6], 1e-6)
    M.offline()
    th = [0.237]
    inst = M.instantiate(th)
    Hs = M.projected_cores(th)
    for b in M.far[:10]:
        W = _W(b, "matern32", th, 4)
        res = W - b.L @ Hs[id(b)] @ b.R.T
        assert np.abs(b.L.T @ res @ b.R).max() <= 1e-12 * np.abs(W).max()
        assert np.linalg.norm(res) <= np.linalg.norm(W - M.coupling(b, inst)) * (1 + 1e-12)


def test_polynomial_kernel_exact_with_projected_cores_and_its_own_near_grid():
    """kappa = 1 + theta r^2 + theta^2 r^4, no truncation: degree 4 per coordinate (p_s = 5 is exact)
    and 2 in theta, so a near grid of 3 nodes and a far grid of 5 are both exact, and the matrix
    with projected far cores reproduces the dense K(theta) X at any theta."""
    M = _model("poly", [0.5], [2.0], [4], 0.0, near_degree=[2], n=300, p_s=5)
    assert len(M.taxes_near[0]) == 3 and len(M.taxes[0]) == 5
    M.offline()
    X = np.random.default_rng(2).standard_normal((M.n, 2))
    for th in (0.61, 1.37):
        ref = kernels.dense_apply("poly", M.P, [th], X)
        for inst in (M.instantiate([th]), M.instantiate_projected([th])):
            Y = M.matvec(inst, X)
            assert np.linalg.norm(Y - ref) <= 1e-11 * np.linalg.norm(ref)


def test_near_grid_of_its_own_changes_only_the_near_field():
    """A coarser near grid leaves every far-field quantity unchanged and gives near blocks that
    interpolate on their own nodes: at a near-grid node D_b equals the kernel block."""
    A = _model("gauss", [0.2], [1.0], [6], 0.0)
    B = _model("gauss", [0.2], [1.0], [6], 0.0, near_degree=[3])
    A.offline()
    B.offline()
    th = [cheb.cheb_nodes(0.2, 1.0, 4)[1]]
    ia, ib = A.instantiate(th), B.instantiate(th)
    for ba, bb in zip(A.far[:5], B.far[:5]):
        np.testing.assert_allclose(ia["H"][id(ba)], ib["H"][id(bb)], rtol=0, atol=0)
    for b in B.near[:5]:
        K = kernels.kappa("gauss", B.P[b.s.idx][:, None], B.P[b.t.idx][None], th)
        np.testing.assert_allclose(ib["D"][id(b)], K, atol=1e-12)
    assert math.isclose(len(B.taxes_near[0]), 4)
