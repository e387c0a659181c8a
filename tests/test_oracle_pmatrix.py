"""Pins for the oracle's parametric H / H^2 construction and MVM (§3.6, §4, App. A.3, A.4).

Each pin compares the oracle with something that does not go through the same
code: the kernel evaluated directly, the non-parametric coupling matrix W_b of
§3.6.2, the dense product K(theta) X, or a mathematical identity.
"""
import numpy as np
import pytest

from oracle import cheb, kernels, pmatrix, tensor, tree
from paper_2511_03109_gb300 import inputs


def _model(n, d, kernel, lo, hi, degree, p_s, l_max, eta, tol, fmt, cap=None, seed=7):
    P = inputs.uniform_points(n, d, seed)
    return pmatrix.ParametricMatrix(P, kernel, lo, hi, degree, p_s, l_max, eta, tol,
                                    rank_cap=cap, fmt=fmt)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_nestedness_lemma(d):
    """Gamma_{s'} U_s = U_{s'} E_{s'} (App. A.3) to 1e-13."""
    P = inputs.uniform_points(200, d, 3)
    root = tree.build_cluster_tree(P, 2)
    for c in tree.all_nodes(root):
        for ch in c.children:
            Us = pmatrix.cluster_basis(pmatrix.basis_factors(P, c, 5))
            rows = np.searchsorted(c.idx, ch.idx)  # Gamma selects the child's rows of U_s
            Uc = pmatrix.cluster_basis(pmatrix.basis_factors(P, ch, 5))
            E = pmatrix.transfer_matrix(pmatrix.transfer_factors(ch, 5))
            np.testing.assert_allclose(Us[rows], Uc @ E, atol=1e-13, rtol=0)


def test_cluster_basis_is_tensor_lagrange():
    """Row x of U_s holds Lambda_i(x) = prod_k ell_{i_k}(x_k) at column i_1 + p i_2 + p^2 i_3 (§2.2, §3.3)."""
    P = inputs.uniform_points(50, 3, 9)
    c = tree.build_cluster_tree(P, 1).children[0]
    p = 4
    U = pmatrix.cluster_basis(pmatrix.basis_factors(P, c, p))
    x = P[c.idx[3]]
    nodes = [cheb.cheb_nodes(c.lo[k], c.hi[k], p) for k in range(3)]
    for i1 in range(p):
        for i2 in range(p):
            for i3 in range(p):
                ref = (cheb.lagrange(nodes[0], x[0])[0, i1] * cheb.lagrange(nodes[1], x[1])[0, i2]
                       * cheb.lagrange(nodes[2], x[2])[0, i3])
                assert abs(U[3, i1 + p * i2 + p * p * i3] - ref) < 1e-14


def test_near_block_exact_at_theta_node():
    """With tolerance 0, D_b(eta_k) is the kernel block K(X_s, X_t; eta_k) (§4.3)."""
    M = _model(300, 2, "matern32", [0.05], [0.5], [6], 5, 2, 1.0, 0.0, "h2")
    nodes = cheb.cheb_nodes(0.05, 0.5, 7)
    for b in M.near[:12]:
        M.compress_near(b)
        vs = M.parametric_vectors([nodes[3]])
        D = M.near_instance(b, vs)
        K = kernels.kappa("matern32", M.P[b.s.idx][:, None], M.P[b.t.idx][None], [nodes[3]])
        np.testing.assert_allclose(D, K, atol=1e-13)


@pytest.mark.parametrize("d,p_s", [(2, 5), (3, 3)])
def test_coupling_is_W_at_theta_node(d, p_s):
    """With tolerance 0 and theta = eta_k, C_b(theta) = W_b of §3.6.2 (evaluated directly)."""
    M = _model(300, d, "gauss", [0.2], [1.0], [4], p_s, 2, np.sqrt(d), 0.0, "h2")
    nodes = cheb.cheb_nodes(0.2, 1.0, 5)
    th = nodes[2]
    for b in M.far[:6]:
        M.compress_far(b)
        inst = {"H": {id(b): pmatrix.H_matrix(b.cores, d, M.parametric_vectors([th]))}}
        C = M.coupling(b, inst)
        # W_b[i, j] = kappa(eta^s_i, eta^t_j; theta) with little-endian multi-indices (§3.6.2)
        ps = np.empty((p_s ** d, d))
        pt = np.empty((p_s ** d, d))
        for flat in range(p_s ** d):
            idx = [(flat // p_s ** k) % p_s for k in range(d)]
            ps[flat] = [cheb.cheb_nodes(b.s.lo[k], b.s.hi[k], p_s)[idx[k]] for k in range(d)]
            pt[flat] = [cheb.cheb_nodes(b.t.lo[k], b.t.hi[k], p_s)[idx[k]] for k in range(d)]
        W = kernels.kappa("gauss", ps[:, None], pt[None], [th])
        np.testing.assert_allclose(C, W, atol=1e-12 * np.abs(W).max())


@pytest.mark.parametrize("fmt", ["h2", "h"])
@pytest.mark.parametrize("d,n,l_max,eta", [(2, 300, 3, 1.0), (3, 250, 2, np.sqrt(3.0))])
def test_polynomial_kernel_reproduced_exactly(fmt, d, n, l_max, eta):
    """kappa = 1 + theta r^2 + theta^2 r^4 has degree 4 per coordinate and 2 in theta, so with
    p_s = 5, p_theta = 3 and no truncation every interpolation is exact: K_hat(theta) X = K(theta) X."""
    M = _model(n, d, "poly", [0.5], [2.0], [2], 5, l_max, eta, 0.0, fmt)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((n, 2))
    targets = M.leaves[:: max(1, len(M.leaves) // 6)] if d == 3 else None
    M.offline(targets)
    for th in (0.5, 0.93, 1.71):
        inst = M.instantiate([th], targets)
        Y = M.matvec(inst, X, targets)
        ref = kernels.dense_apply("poly", M.P, [th], X)
        keep = ~np.isnan(Y[:, 0])
        assert keep.sum() > 0 and len(M.far) > 0
        err = np.linalg.norm(Y[keep] - ref[keep]) / np.linalg.norm(ref[keep])
        assert err < 1e-11


def test_non_translation_invariant_kernel_reproduced():
    """(1 + x.y)^2 (1 + theta) is exact as well; the oracle never reuses blocks across offsets."""
    M = _model(200, 2, "polyxy", [0.0], [1.0], [1], 3, 3, 1.0, 0.0, "h2")
    X = np.random.default_rng(2).standard_normal((200, 1))
    M.offline()
    inst = M.instantiate([0.37])
    np.testing.assert_allclose(M.matvec(inst, X), kernels.dense_apply("polyxy", M.P, [0.37], X),
                               rtol=1e-11, atol=1e-11)


def test_theta_outside_box_rejected():
    M = _model(100, 2, "gauss", [0.1], [1.0], [4], 4, 2, 1.0, 1e-6, "h2")
    with pytest.raises(ValueError):
        M.instantiate([1.5])


def test_near_part_symmetric_mirror():
    """A_{ts} is a row permutation of A_{st}, so the truncated TT gives D_ts = D_st^T (§4.3)."""
    M = _model(400, 2, "matern32", [0.05], [0.5], [20], 8, 3, 1.0, 1e-5, "h2")
    vs = M.parametric_vectors([0.21])
    blocks = {(b.s.id, b.t.id): b for b in M.near}
    checked = 0
    for (i, j), b in blocks.items():
        if i < j and (j, i) in blocks:
            D1 = M.near_instance(M.compress_near(b), vs)
            D2 = M.near_instance(M.compress_near(blocks[(j, i)]), vs)
            np.testing.assert_allclose(D1, D2.T, atol=1e-12)
            checked += 1
            if checked == 10:
                break
    assert checked == 10


def test_interpolation_error_decays_with_degree():
    """Near-field-only case (l_max = 1: every block is near), so the error against the exact
    K(theta) X is the theta-interpolation error alone; it must fall as p_theta grows."""
    P = inputs.uniform_points(256, 2, 21)
    X = inputs.gaussian_rhs(256, 1, 22)
    errs = []
    for deg in (4, 8, 16, 24, 32):
        M = pmatrix.ParametricMatrix(P, "gauss", [0.1], [1.0], [deg], 4, 1, 1.0, 1e-13, fmt="h2")
        assert len(M.far) == 0
        M.offline()
        e = 0.0
        for th in (0.13, 0.42, 0.77):
            ref = kernels.dense_apply("gauss", P, [th], X)
            e = max(e, pmatrix.relative_error(ref, M.matvec(M.instantiate([th]), X))[0])
        errs.append(e)
    # geometric (Chebyshev) convergence for the analytic dependence on l: each step of 8 in
    # the degree gains well over a factor of 10
    assert all(errs[i + 1] < 0.3 * errs[i] for i in range(4)), errs
    assert errs[-1] < 1e-6


@pytest.mark.parametrize("fmt", ["h2", "h"])
def test_whole_method_close_to_dense_for_gaussian(fmt):
    """Whole method against the exact product for a small 2-D Gaussian case: the error is the
    approximation's own (spatial + theta interpolation + TT truncation) and must shrink when the
    theta degree grows (degree 16 -> 32 on l in [0.1, 1])."""
    X = np.random.default_rng(3).standard_normal((500, 1))
    errs = {}
    for deg in (16, 32):
        M = _model(500, 2, "gauss", [0.1], [1.0], [deg], 8, 2, 1.0, 1e-9, fmt, cap=32)
        assert len(M.far) > 0
        M.offline()
        errs[deg] = max(pmatrix.relative_error(kernels.dense_apply("gauss", M.P, [th], X),
                                               M.matvec(M.instantiate([th]), X))[0]
                        for th in (0.37, 0.9))
    assert errs[16] < 1e-4 and errs[32] < 1e-6 and errs[32] < 0.05 * errs[16], errs


def test_target_rows_match_full():
    M = _model(300, 2, "matern52", [0.1], [0.6], [8], 6, 3, 1.0, 1e-8, "h2")
    X = np.random.default_rng(4).standard_normal((300, 3))
    M.offline()
    inst = M.instantiate([0.33])
    full = M.matvec(inst, X)
    targets = M.leaves[5:9]
    part = M.matvec(M.instantiate([0.33], targets), X, targets)
    keep = ~np.isnan(part[:, 0])
    np.testing.assert_allclose(part[keep], full[keep], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("fmt", ["h2", "h"])
def test_theta_derivative_against_differences_and_exact_derivative(fmt):
    """dK_hat/dtheta X (v replaced by its derivative) equals the central difference of the
    method in theta (K_hat is a polynomial of degree q in theta), and approximates the exact
    derivative of the Gaussian, d/dl exp(-r^2 / (2 l^2)) = r^2 / l^3 exp(-r^2 / (2 l^2))."""
    X = np.random.default_rng(21).standard_normal((400, 2))
    M = _model(400, 2, "gauss", [0.2], [0.6], [24], 8, 2, 1.0, 1e-10, fmt, cap=48)
    M.offline()
    th, h = 0.37, 1e-5
    dY = M.matvec(M.instantiate([th], deriv=0), X)
    fd = (M.matvec(M.instantiate([th + h]), X) - M.matvec(M.instantiate([th - h]), X)) / (2 * h)
    assert np.all(pmatrix.relative_error(fd, dY) < 1e-8)
    P = M.P
    r2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    dK = r2 / th ** 3 * np.exp(-r2 / (2 * th * th))
    assert np.all(pmatrix.relative_error(dK @ X, dY) < 1e-6)
    with pytest.raises(ValueError):
        M.instantiate([th], deriv=1)


@pytest.mark.parametrize("fmt", ["h2", "h"])
def test_instance_is_lagrange_combination_of_node_instances(fmt):
    """K_hat(theta) X = sum_q ell_q(theta) K_hat(eta_q) X (and the same with ell_q' for the
    theta-derivative): the identity the batched product relies on, checked on the oracle."""
    X = np.random.default_rng(33).standard_normal((350, 2))
    M = _model(350, 2, "matern52", [0.1], [0.6], [9], 6, 2, 1.0, 1e-9, fmt)
    M.offline()
    nodes = cheb.cheb_nodes(0.1, 0.6, 10)
    Yq = np.stack([M.matvec(M.instantiate([eta]), X) for eta in nodes])
    for th in (0.1, 0.2345, float(nodes[4]), 0.6):
        direct = M.matvec(M.instantiate([th]), X)
        comb = np.tensordot(cheb.lagrange(nodes, th)[0], Yq, axes=1)
        assert np.all(pmatrix.relative_error(direct, comb) < 1e-12)
        d_direct = M.matvec(M.instantiate([th], deriv=0), X)
        d_comb = np.tensordot(cheb.lagrange_derivative(nodes, th)[0], Yq, axes=1)
        assert np.all(pmatrix.relative_error(d_direct, d_comb) < 1e-11)


@pytest.mark.parametrize("fmt", ["h2", "h"])
def test_adjoint_inner_products_and_dense_transpose(fmt):
    """matvec_transpose is the adjoint of matvec: <K_hat x, y> = <x, K_hat^T y> for random x, y
    (matrix and theta-derivative), and on a tiny problem it applies the transpose of the dense
    matrix that matvec applies (both formed column by column)."""
    rng = np.random.default_rng(44)
    M = _model(400, 2, "matern52", [0.1], [0.6], [8], 6, 3, 1.0, 1e-9, fmt)
    M.offline()
    x = rng.standard_normal((400, 3))
    y = rng.standard_normal((400, 3))
    for deriv in (None, 0):
        inst = M.instantiate([0.29], deriv=deriv)
        lhs = np.sum(M.matvec(inst, x) * y, axis=0)
        rhs = np.sum(x * M.matvec_transpose(inst, y), axis=0)
        scale = np.linalg.norm(M.matvec(inst, x), axis=0) * np.linalg.norm(y, axis=0)
        assert np.all(np.abs(lhs - rhs) <= 1e-13 * scale)
    T = _model(90, 2, "gauss", [0.2], [0.9], [6], 4, 2, 1.0, 1e-10, fmt)
    T.offline()
    assert len(T.far) > 0
    inst = T.instantiate([0.55])
    eye = np.eye(90)
    K = T.matvec(inst, eye)
    Kt = T.matvec_transpose(inst, eye)
    np.testing.assert_allclose(Kt, K.T, rtol=0, atol=1e-13 * np.abs(K).max())


def test_adjoint_close_to_matrix_for_symmetric_kernel():
    """For a symmetric kernel K_hat^T differs from K_hat only by the truncations of the blocks
    (each block and its mirror are compressed on their own)."""
    M = _model(500, 2, "gauss", [0.1], [1.0], [16], 8, 2, 1.0, 1e-9, "h2", cap=32)
    M.offline()
    y = np.random.default_rng(45).standard_normal((500, 2))
    inst = M.instantiate([0.37])
    assert np.all(pmatrix.relative_error(M.matvec(inst, y), M.matvec_transpose(inst, y)) < 1e-8)


def test_error_follows_the_truncation_tolerance():
    """With a fine spatial and theta grid the error against the exact product is set by the
    TT-SVD tolerance (§2.1): it stays within 2 eps and falls with eps (1e-2 ... 1e-8)."""
    X = np.random.default_rng(61).standard_normal((500, 1))
    errs = []
    for tol in (1e-2, 1e-4, 1e-6, 1e-8):
        M = _model(500, 2, "gauss", [0.2], [0.9], [24], 10, 2, 1.0, tol, "h2")
        M.offline()
        e = max(pmatrix.relative_error(kernels.dense_apply("gauss", M.P, [th], X),
                                       M.matvec(M.instantiate([th]), X))[0] for th in (0.27, 0.81))
        assert e <= 2 * tol, (tol, e)
        errs.append(e)
    assert all(errs[i + 1] < errs[i] / 30 for i in range(3)), errs


@pytest.mark.parametrize("fmt", ["h2", "h"])
def test_two_parameter_method_exact_on_polynomial_kernel(fmt):
    """d_theta = 2 (§4.3 product over the parameter cores, App. A.4 H_b as a product of the
    parameter-core matrices): with the two-parameter polynomial kernel, no truncation and enough
    nodes (degree 1 in theta_1, 2 in theta_2; spatial degree 4 < p_s), the method reproduces the
    dense K(theta) X to rounding for any theta, and its theta-derivatives reproduce the exact ones."""
    from paper_2511_03109_gb300 import inputs
    n = 180
    P = inputs.uniform_points(n, 2, 77)
    X = inputs.gaussian_rhs(n, 2, 78)
    M = pmatrix.ParametricMatrix(P, "poly2", [0.5, 0.2], [2.0, 1.5], [1, 2], 5, 2, 1.0, 0.0, fmt=fmt)
    M.offline()
    for th in ([0.5, 0.2], [1.3, 0.77], [2.0, 1.5]):
        ref = kernels.dense_apply("poly2", P, th, X)
        got = M.matvec(M.instantiate(th), X)
        assert np.max(pmatrix.relative_error(ref, got)) < 1e-11
    # d/dtheta_1 = r^2, d/dtheta_2 = 2 theta_2 r^4
    th = [1.1, 0.9]
    D = np.sum((P[:, None, :] - P[None, :, :]) ** 2, axis=-1)
    for dim, Kd in ((0, D), (1, 2 * th[1] * D * D)):
        got = M.matvec(M.instantiate(th, deriv=dim), X)
        assert np.max(pmatrix.relative_error(Kd @ X, got)) < 1e-10
