"""Pins for the oracle's primitives (Chebyshev/Lagrange, kernels, tensor algebra, TT-SVD).

Each check is against something other than the oracle's own formula: NumPy's
Chebyshev points, polynomial reproduction, SciPy's Bessel K_nu, Eckart-Young,
tensors of known TT rank, the vec-kron identity.
"""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from numpy.polynomial import polynomial as nppoly

from oracle import cheb, kernels, tensor


@pytest.mark.parametrize("p", [1, 2, 5, 8, 17, 27])
def test_cheb_nodes_are_first_kind_points(p):
    a, b = 0.05, 0.5
    ref = a + (b - a) * (npcheb.chebpts1(p) + 1.0) / 2.0  # ascending first-kind points
    got = cheb.cheb_nodes(a, b, p)
    assert np.all(np.diff(got) > 0)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15)
    # they are the roots of T_p mapped to [a, b]
    t = 2.0 * (got - a) / (b - a) - 1.0
    np.testing.assert_allclose(npcheb.chebval(t, [0] * p + [1]), 0.0, atol=1e-12)


@pytest.mark.parametrize("p", [3, 8, 15, 21])
def test_lagrange_kronecker_unity_and_reproduction(p):
    rng = np.random.default_rng(5)
    nodes = cheb.cheb_nodes(-0.3, 1.7, p)
    L = cheb.lagrange(nodes, nodes)
    assert np.array_equal(L, np.eye(p))  # exact unit rows at the nodes
    x = rng.uniform(-0.3, 1.7, 50)
    Lx = cheb.lagrange(nodes, x)
    np.testing.assert_allclose(Lx.sum(axis=1), 1.0, atol=1e-12)
    coef = rng.standard_normal(p)  # degree p-1 polynomial is reproduced exactly
    np.testing.assert_allclose(Lx @ nppoly.polyval(nodes, coef), nppoly.polyval(x, coef),
                               rtol=1e-9, atol=1e-9)


def test_parametric_vectors_unit_at_node():
    lo, hi, deg = [0.1], [1.0], [16]
    nodes = cheb.cheb_nodes(0.1, 1.0, 17)
    v = cheb.parametric_vectors([nodes[4]], lo, hi, deg)[0]
    assert np.array_equal(v, np.eye(17)[4])


def _matern_general(r, ell, nu):
    from scipy.special import gamma, kv
    s = np.sqrt(2 * nu) * r / ell
    return 2 ** (1 - nu) / gamma(nu) * s ** nu * kv(nu, s)


@pytest.mark.parametrize("name,nu", [("matern32", 1.5), ("matern52", 2.5)])
def test_matern_closed_forms_match_bessel(name, nu):
    pytest.importorskip("scipy")
    rng = np.random.default_rng(1)
    x = rng.random((40, 3))
    y = rng.random((40, 3))
    ell = np.array([0.07])
    r = np.linalg.norm(x - y, axis=1)
    np.testing.assert_allclose(kernels.kappa(name, x, y, ell), _matern_general(r, 0.07, nu),
                               rtol=1e-12)
    assert kernels.kappa(name, x[0], x[0], ell) == 1.0


def test_kernels_symmetric_and_gauss_scale():
    rng = np.random.default_rng(2)
    x, y = rng.random((10, 2)), rng.random((10, 2))
    for name in ("gauss", "matern32", "matern52", "se", "exponential", "mc", "poly", "polyxy"):
        np.testing.assert_allclose(kernels.kappa(name, x, y, [0.3]), kernels.kappa(name, y, x, [0.3]))
    r2 = np.sum((x - y) ** 2, axis=1)
    np.testing.assert_allclose(kernels.kappa("gauss", x, y, [0.3]), np.exp(-r2 / 0.18), rtol=1e-14)
    # anisotropic Gaussian with equal lengths is the isotropic one
    np.testing.assert_allclose(kernels.kappa("aniso_gauss", x, y, [0.3, 0.3]),
                               kernels.kappa("gauss", x, y, [0.3]), rtol=1e-14)


def test_reshape_unfoldings_index_rules():
    rng = np.random.default_rng(3)
    G = rng.standard_normal((3, 4, 5))
    G1, G2 = tensor.unfold1(G), tensor.unfold2(G)
    for a in range(3):
        for m in range(4):
            for b in range(5):
                assert G1[a, m + 4 * b] == G[a, m, b]
                assert G2[a + 3 * m, b] == G[a, m, b]


def test_vec_kron_identity_and_face_split():
    rng = np.random.default_rng(4)
    A, X, B = rng.standard_normal((3, 4)), rng.standard_normal((4, 5)), rng.standard_normal((5, 2))
    vec = lambda M: tensor.freshape(M, (-1,))
    np.testing.assert_allclose(vec(A @ X @ B), tensor.kron_chain([B.T, A]) @ vec(X), atol=1e-13)
    P, Q = rng.standard_normal((6, 2)), rng.standard_normal((6, 3))
    F = tensor.face_split(P, Q)
    for i in range(6):
        np.testing.assert_array_equal(F[i], np.kron(P[i], Q[i]))


def _random_tt(dims, ranks, rng):
    return [rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(len(dims))]


def test_tt_svd_recovers_known_low_rank():
    rng = np.random.default_rng(6)
    dims, ranks = (4, 5, 3, 6), (1, 2, 3, 2, 1)
    A = tensor.tt_full(_random_tt(dims, ranks, rng))
    # the entry formula of the TT format, written out for one entry
    cores = _random_tt(dims, ranks, rng)
    B = tensor.tt_full(cores)
    e = cores[0][:, 1, :] @ cores[1][:, 2, :] @ cores[2][:, 0, :] @ cores[3][:, 4, :]
    assert abs(B[1, 2, 0, 4] - e[0, 0]) < 1e-12
    got, r = tensor.tt_svd(A, 1e-12)
    assert r == [1, 2, 3, 2, 1]
    np.testing.assert_allclose(tensor.tt_full(got), A, atol=1e-11 * np.abs(A).max())


@pytest.mark.parametrize("eps", [1e-2, 1e-5])
def test_tt_svd_error_bound_random(eps):
    rng = np.random.default_rng(7)
    # smooth tensor with decaying spectrum
    g = np.linspace(0, 1, 9)
    A = 1.0 / (1.0 + g[:, None, None, None] + 2 * g[None, :, None, None] + 3 * g[None, None, :, None]
               + 4 * g[None, None, None, :])
    A = A + 1e-9 * rng.standard_normal(A.shape)
    cores, ranks = tensor.tt_svd(A, eps)
    assert np.linalg.norm(tensor.tt_full(cores) - A) <= eps * np.linalg.norm(A) * (1 + 1e-10)
    cores2, ranks2 = tensor.tt_svd(A, eps, rank_cap=2)
    assert max(ranks2) <= 2


def test_tt_svd_two_way_is_eckart_young():
    rng = np.random.default_rng(8)
    U, _ = np.linalg.qr(rng.standard_normal((30, 10)))
    V, _ = np.linalg.qr(rng.standard_normal((12, 10)))
    s = 10.0 ** -np.arange(10)
    A = (U * s) @ V.T
    eps = 2e-4
    cores, ranks = tensor.tt_svd(A, eps)
    # delta = eps ||A|| (q = 2); smallest rank whose tail is below delta
    tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])
    expect = int(np.argmax(np.append(tail[1:], 0.0) <= eps * np.linalg.norm(s))) + 1
    assert ranks[1] == expect
    approx = tensor.tt_full(cores)
    np.testing.assert_allclose(np.linalg.norm(approx - A), tail[expect] if expect < 10 else 0.0,
                               rtol=1e-8, atol=1e-15)


def test_truncation_rank_keeps_ties_whole():
    s = np.array([1.0, 0.5, 1e-3, 1e-3, 1e-7])
    # the tail rule alone would stop inside the tied pair; the tie rule keeps both
    assert tensor.truncation_rank(s, delta=1.0001e-3) == 4
    assert tensor.truncation_rank(s, delta=1.0, rank_cap=3) == 1
    assert tensor.truncation_rank(s, delta=0.0) == 5


@pytest.mark.parametrize("p", [2, 5, 11, 21])
def test_lagrange_derivative_against_polyder_and_differences(p):
    """ell_k' from the product rule: sums to zero, differentiates polynomials of degree < p
    exactly (NumPy's polyder), and matches central differences of the Lagrange values."""
    rng = np.random.default_rng(9)
    a, b = 0.05, 0.5
    nodes = cheb.cheb_nodes(a, b, p)
    x = np.concatenate([rng.uniform(a, b, 40), nodes])  # includes the nodes themselves
    Ld = cheb.lagrange_derivative(nodes, x)
    scale = np.abs(Ld).max()
    np.testing.assert_allclose(Ld.sum(axis=1), 0.0, atol=1e-12 * scale)
    coef = rng.standard_normal(p)
    ref = nppoly.polyval(x, nppoly.polyder(coef))
    np.testing.assert_allclose(Ld @ nppoly.polyval(nodes, coef), ref, rtol=1e-9,
                               atol=1e-10 * scale * np.abs(coef).sum())
    h = 1e-6
    fd = (cheb.lagrange(nodes, x + h) - cheb.lagrange(nodes, x - h)) / (2 * h)
    np.testing.assert_allclose(Ld, fd, rtol=0, atol=1e-6 * scale)


def test_parametric_vectors_derivative_dimension_only():
    lo, hi, deg = [0.1, 1.0], [1.0, 3.0], [6, 9]
    th = [0.43, 2.2]
    v = cheb.parametric_vectors(th, lo, hi, deg)
    dv = cheb.parametric_vectors(th, lo, hi, deg, deriv=1)
    assert np.array_equal(dv[0], v[0])  # other dimensions keep their values
    nodes = cheb.cheb_nodes(1.0, 3.0, 10)
    np.testing.assert_allclose(dv[1], cheb.lagrange_derivative(nodes, 2.2)[0], rtol=0, atol=0)


def test_aniso_gauss_per_axis_lengths():
    """exp(-sum_k (x_k - y_k)^2 / (2 l_k^2)) evaluated by hand with three different lengths: a
    swapped pair of axes or lengths changes the value, and the kernel is the product of the
    1-D Gaussians of each axis."""
    x = np.array([0.1, 0.2, 0.3])
    y = np.array([0.4, 0.0, 0.35])
    ell = np.array([0.5, 0.1, 0.2])
    # 0.3^2 / (2 * 0.25) + 0.2^2 / (2 * 0.01) + 0.05^2 / (2 * 0.04) = 0.18 + 2 + 0.03125
    expect = np.exp(-2.21125)
    np.testing.assert_allclose(kernels.kappa("aniso_gauss", x, y, ell), expect, rtol=1e-14)
    assert abs(kernels.kappa("aniso_gauss", x, y, ell[[1, 0, 2]]) - expect) > 1e-3
    assert abs(kernels.kappa("aniso_gauss", x[[1, 0, 2]], y, ell) - expect) > 1e-3
    rng = np.random.default_rng(5)
    xs, ys = rng.random((20, 2)), rng.random((20, 2))
    l2 = np.array([0.07, 0.31])
    prod = (kernels.kappa("gauss", xs[:, :1], ys[:, :1], [l2[0]]) *
            kernels.kappa("gauss", xs[:, 1:], ys[:, 1:], [l2[1]]))
    np.testing.assert_allclose(kernels.kappa("aniso_gauss", xs, ys, l2), prod, rtol=1e-13)


def test_poly2_closed_form():
    """The two-parameter test kernel 1 + t1 r^2 + t2^2 r^4, evaluated by hand."""
    x, y = np.array([0.1, 0.4]), np.array([0.4, 0.0])  # r^2 = 0.09 + 0.16 = 0.25
    np.testing.assert_allclose(kernels.kappa("poly2", x, y, [0.7, 1.5]), 1 + 0.7 * 0.25 + 2.25 * 0.0625, rtol=1e-15)
    assert kernels.kappa("poly2", x, x, [0.7, 1.5]) == 1.0


def test_truncation_rank_cap_never_splits_a_tied_group():
    """A cap that falls inside a group of equal singular values drops the whole group (a cut inside
    it would keep an arbitrary subspace); a cap between distinct values is applied as is."""
    s = np.array([5.0, 3.0, 2.0, 2.0, 2.0, 1.0, 0.5])
    assert tensor.truncation_rank(s, 0.0, rank_cap=3) == 2  # 2.0 x 3 would be split: keep 5, 3
    assert tensor.truncation_rank(s, 0.0, rank_cap=5) == 5  # the group fits
    assert tensor.truncation_rank(s, 0.0, rank_cap=6) == 6
    assert tensor.truncation_rank(s, 0.0, rank_cap=None) == 7
    # the exact factorisation of a Kronecker-structured matrix (repeated products of singular
    # values) truncated at a cap inside a repeated value: unique whatever the SVD's basis
    a = np.diag([1.0, 0.5])
    K = np.kron(np.kron(a, a), a)  # singular values 1, .5 x3, .25 x3, .125
    sv = np.linalg.svd(K, compute_uv=False)
    assert tensor.truncation_rank(sv, 0.0, rank_cap=2) == 1
    assert tensor.truncation_rank(sv, 0.0, rank_cap=4) == 4
