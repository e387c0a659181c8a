"""Pins for the oracle's TT-cross and TT-rounding (oracle.cross), the paper's compressor (§2.1).

They compare with things outside the code they check: tensors built from known TT cores, the
kernel evaluated on the grid, and the TT-SVD of the same tensor (oracle.tensor, itself pinned
against Eckart-Young and known low-rank tensors)."""
import numpy as np
import pytest

from oracle import cross, pmatrix, tensor, tree


def _random_tt(dims, ranks, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(len(dims))]


def _far(kern, d, ps, lo, hi, deg):
    s = tree.Cluster([], np.zeros(d), np.full(d, 0.25), 0)
    t = tree.Cluster([], np.full(d, 0.5), np.full(d, 0.75), 0)
    return pmatrix.far_tensor(kern, s, t, pmatrix.theta_grid(lo, hi, deg), ps)


@pytest.mark.parametrize("dims,ranks", [((5, 6, 4, 7), (1, 3, 3, 2, 1)), ((4, 4, 4, 4, 4), (1, 2, 4, 4, 2, 1))])
def test_exact_on_tensors_of_known_tt_rank(dims, ranks):
    A = tensor.tt_full(_random_tt(dims, ranks, seed=sum(dims)))
    cores, got, T = cross.tt_cross(lambda idx: A[tuple(idx.T)], dims, 1e-12)
    assert np.linalg.norm(tensor.tt_full(cores) - A) <= 1e-10 * np.linalg.norm(A)
    assert all(g >= r for g, r in zip(got, ranks))
    c2, r2 = cross.tt_round(cores, 1e-10)
    assert list(r2) == list(ranks)
    assert np.linalg.norm(tensor.tt_full(c2) - A) <= 1e-9 * np.linalg.norm(A)


def test_interpolates_the_tensor_on_its_crosses():
    M = _far("gauss", 2, 5, [0.1], [1.0], [6])
    cores, _, T = cross.tt_cross(lambda idx: M[tuple(idx.T)], M.shape, 1e-6)
    A = tensor.tt_full(cores)
    q = M.ndim
    for k in range(q - 1):
        for a in T.I[k + 1]:
            for b in T.J[k + 1]:
                x = tuple(a) + tuple(b)
                assert abs(A[x] - M[x]) <= 1e-10 * np.abs(M).max(), (k, x)


@pytest.mark.parametrize("kern,d,ps,lo,hi,deg", [
    ("gauss", 2, 5, [0.1], [1.0], [6]),
    ("matern32", 3, 4, [0.05], [0.5], [8]),
    ("aniso_gauss", 2, 5, [0.1, 0.1], [0.5, 0.5], [4, 4]),
])
@pytest.mark.parametrize("eps", [1e-4, 1e-7])
def test_rounded_cross_matches_tt_svd_on_kernel_tensors(kern, d, ps, lo, hi, deg, eps):
    M = _far(kern, d, ps, lo, hi, deg)
    cores, _, T = cross.tt_cross(lambda idx: M[tuple(idx.T)], M.shape, eps)
    c2, r2 = cross.tt_round(cores, eps)
    err = np.linalg.norm(tensor.tt_full(c2) - M) / np.linalg.norm(M)
    _, rs = tensor.tt_svd(M, eps)
    assert err <= 3 * eps, err
    assert all(abs(a - b) <= 1 for a, b in zip(r2, rs)), (r2, rs)


def test_evaluates_a_small_part_of_a_large_tensor():
    M = _far("matern32", 3, 6, [0.05], [0.5], [8])  # 6^3 x 9 x 6^3 = 419 904 entries
    cores, _, T = cross.tt_cross(lambda idx: M[tuple(idx.T)], M.shape, 1e-5)
    c2, _ = cross.tt_round(cores, 1e-5)
    assert np.linalg.norm(tensor.tt_full(c2) - M) <= 3e-5 * np.linalg.norm(M)
    assert T.count < 0.25 * M.size, T.count
