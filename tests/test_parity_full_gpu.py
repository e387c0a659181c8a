"""Parity at the workloads' full sizes.

* the small 2-D FP64 configuration (n = 4096, Gaussian, degree 16, eta = 1, leaf 64, rank <= 32,
  theta = 0.37, one RHS) for both formats: every row against the oracle, <= 1e-10;
* the 3-D FP32 configuration that bench.py times (n = 65536, Matern 3/2, degree 20, rank <= 64,
  16 RHS), built and launched exactly as bench.py does: the rows of at least eight sampled target
  leaves (corners, edges, faces, interior, the largest leaf) against the oracle (which compresses
  those leaves' blocks in a spawn-started pool), <= 1e-5;
* edge cases: n = 0 is refused; the maximum m = 1024 right-hand sides.
"""
import os

import numpy as np
import pytest

from oracle import pmatrix
from paper_2511_03109_gb300 import inputs

from helpers import TOL, build_pair, device_apply, rel_err_rows, target_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pool():
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        return mp.get_context("spawn").Pool(max(1, os.cpu_count() or 2))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("wl", [inputs.SMALL_2D_GAUSS_H2, inputs.SMALL_2D_GAUSS_H], ids=lambda w: w.name)
def test_small_2d_fp64_all_rows(wl):
    P, X = wl.points(), wl.rhs()
    with _pool() as pool:
        A, M, _ = build_pair(P, wl.kernel, wl.theta_lo, wl.theta_hi, wl.degree, wl.p_s, wl.l_max, wl.eta,
                             wl.tol, wl.rank_cap, wl.fmt, wl.precision, pool=pool)
    ref = M.matvec(M.instantiate(wl.theta), X)
    got = device_apply(A, wl.theta, X, wl.precision)
    assert np.all(rel_err_rows(ref, got) <= TOL["fp64"])
    A.close()


def test_bench_workload_sampled_rows():
    from paper_2511_03109_gb300 import ph

    wl = inputs.LARGE_3D_MATERN_H2
    P, X = wl.points(), wl.rhs()
    opts = ph.make_opts(wl.d, wl.theta_lo, wl.theta_hi, wl.degree, wl.p_s, wl.l_max, wl.eta, wl.tol,
                        rank_cap=wl.rank_cap, fmt=wl.fmt, prec=wl.precision)
    A = ph.ParametricMatrix(P, wl.kernel, opts)
    M = pmatrix.ParametricMatrix(P, wl.kernel, wl.theta_lo, wl.theta_hi, wl.degree, wl.p_s, wl.l_max,
                                 wl.eta, wl.tol, rank_cap=wl.rank_cap, fmt=wl.fmt)
    # leaves of every far-field structure of the 8 x 8 x 8 leaf grid: two corners, two edges, two
    # faces, two interior boxes (random, seeded), and the largest leaf
    rng = np.random.default_rng(11)
    side = 2 ** wl.l_max
    by_kind = {k: [] for k in range(4)}
    for i, c in enumerate(M.leaves):
        box = np.rint(c.lo * side).astype(int)
        by_kind[int(np.sum((box == 0) | (box == side - 1)))].append(i)
    idx = set()
    for kind in (3, 2, 1, 0):
        idx.update(int(i) for i in rng.choice(by_kind[kind], size=2, replace=False))
    idx.add(int(np.argmax([c.n for c in M.leaves])))
    targets = [M.leaves[i] for i in sorted(idx)]
    assert len(targets) >= 8
    with _pool() as pool:
        M.offline(targets, pool=pool)
    rows = target_rows(targets)
    theta = list(inputs.uniform_thetas(wl.theta_lo, wl.theta_hi, 1, wl.theta_seed)[0])
    ref = M.matvec(M.instantiate(theta, targets), X, targets)
    got = device_apply(A, theta, X, wl.precision)
    err = rel_err_rows(ref, got, rows)
    assert np.all(err <= TOL["fp32"]), err
    A.close()


def test_empty_input_refused():
    from paper_2511_03109_gb300 import ph

    opts = ph.make_opts(2, [0.1], [1.0], [8], 4, 2, 1.0, 1e-6)
    with pytest.raises(ph.PHError) as e:
        ph.ParametricMatrix(np.zeros((0, 2)), "gauss", opts)
    assert e.value.status == ph.PH_ERR_INVALID_ARG


def test_maximum_rhs_count():
    n, m = 300, 1024
    P = inputs.uniform_points(n, 2, 91)
    X = inputs.gaussian_rhs(n, m, 92)
    A, M, _ = build_pair(P, "matern32", [0.1], [0.5], [10], 6, 2, 1.0, 1e-6, 32, "h2", "fp32")
    ref = M.matvec(M.instantiate([0.2]), X)
    assert np.all(rel_err_rows(ref, device_apply(A, [0.2], X, "fp32")) <= TOL["fp32"])
    A.close()
