"""The library's TT-cross + TT-rounding (host code, ph_tt_cross_check; no GPU) against the
oracle: exact recovery of tensors of known TT rank, and on kernel tensors the TT-SVD ranks of
the oracle with an error within a small multiple of the tolerance, from a fraction of the
entries."""
import numpy as np
import pytest

from oracle import pmatrix, tensor, tree


def _far(kern, d, ps, lo, hi, deg):
    s = tree.Cluster([], np.zeros(d), np.full(d, 0.25), 0)
    t = tree.Cluster([], np.full(d, 0.5), np.full(d, 0.75), 0)
    return pmatrix.far_tensor(kern, s, t, pmatrix.theta_grid(lo, hi, deg), ps)


@pytest.mark.parametrize("dims,ranks", [((5, 6, 4, 7), (1, 3, 3, 2, 1)), ((4, 4, 4, 4, 4), (1, 2, 4, 4, 2, 1))])
def test_exact_on_tensors_of_known_tt_rank(dims, ranks):
    from paper_2511_03109_gb300 import ph

    rng = np.random.default_rng(sum(dims))
    A = tensor.tt_full([rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(len(dims))])
    r, B, ev = ph.tt_cross_check(A, 1e-12)
    assert list(r) == list(ranks)
    assert np.linalg.norm(B - A) <= 1e-9 * np.linalg.norm(A)


@pytest.mark.parametrize("kern,d,ps,lo,hi,deg", [
    ("gauss", 2, 5, [0.1], [1.0], [6]),
    ("matern32", 3, 4, [0.05], [0.5], [8]),
    ("aniso_gauss", 2, 5, [0.1, 0.1], [0.5, 0.5], [4, 4]),
])
@pytest.mark.parametrize("eps", [1e-4, 1e-7])
def test_matches_tt_svd_on_kernel_tensors(kern, d, ps, lo, hi, deg, eps):
    from paper_2511_03109_gb300 import ph

    M = _far(kern, d, ps, lo, hi, deg)
    r, B, ev = ph.tt_cross_check(M, eps)
    _, rs = tensor.tt_svd(M, eps)
    assert all(abs(a - b) <= 1 for a, b in zip(r, rs)), (r, rs)
    assert np.linalg.norm(B - M) <= 3 * eps * np.linalg.norm(M)
    assert ev <= M.size


def test_evaluates_a_small_part_of_a_large_tensor():
    from paper_2511_03109_gb300 import ph

    M = _far("matern32", 3, 6, [0.05], [0.5], [8])  # 419 904 entries
    r, B, ev = ph.tt_cross_check(M, 1e-5, cap=64)
    assert np.linalg.norm(B - M) <= 3e-5 * np.linalg.norm(M)
    assert ev < 0.25 * M.size, ev


def test_rank_cap_is_respected():
    from paper_2511_03109_gb300 import ph

    M = _far("matern32", 3, 4, [0.05], [0.5], [8])
    r, B, ev = ph.tt_cross_check(M, 1e-9, cap=8)
    assert max(r) <= 8


@pytest.mark.parametrize("kern,d,lo,hi,deg,ps,bound", [
    ("gauss", 2, [0.1], [1.0], [10], 6, 3),
    ("matern32", 3, [0.05], [0.5], [8], 4, 3),
    ("aniso_gauss", 3, [0.05] * 3, [0.5] * 3, [3, 3, 3], 4, 100),  # ranks near the cap: a looser bound
])
def test_offline_far_cross_reproduces_the_far_tensor(kern, d, lo, hi, deg, ps, bound):
    """The offline build's route (ph_far_cross_check: kernel entries on the boxes' Chebyshev grids
    and the theta grid, then TT-cross) against the oracle's far tensor M_b of the same boxes."""
    from paper_2511_03109_gb300 import ph

    s = tree.Cluster([], np.zeros(d), np.full(d, 0.25), 0)
    t = tree.Cluster([], np.full(d, 0.5), np.r_[np.full(d - 1, 0.75), 0.25], 0)
    M = pmatrix.far_tensor(kern, s, t, pmatrix.theta_grid(lo, hi, deg), ps)
    r, A = ph.far_cross_check(kern, (s.lo, s.hi), (t.lo, t.hi), lo, hi, deg, ps, 1e-7, 64)
    assert A.shape == M.shape
    assert np.linalg.norm(A - M) <= bound * 1e-7 * np.linalg.norm(M)
    _, rs = tensor.tt_svd(M, 1e-7, 64)
    assert all(abs(a - b) <= 3 for a, b in zip(r, rs)), (r, rs)
