"""The offline build with the paper's compressor (compressor = 1: greedy TT-cross and TT-rounding
of the far-field tensors on the host, §2.1) against the TT-SVD build and the exact product.
TT-cross and TT-SVD give different (equally valid) approximations, so the check is accuracy:
the product with the cross-built far field is as close to the exact K(theta) X as the
TT-SVD-built one, with the largest far rank within three of TT-SVD's."""
import numpy as np
import pytest

from oracle import kernels
from paper_2511_03109_gb300 import inputs

from helpers import device_apply, rel_err_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("d,n,kern,lo,hi,deg,ps,lmax,eta,tol,prec", [
    (2, 1500, "gauss", [0.1], [1.0], [10], 6, 3, 1.0, 1e-8, "fp64"),
    (3, 3000, "matern32", [0.05], [0.5], [12], 4, 2, np.sqrt(3.0), 1e-6, "fp32"),
])
def test_cross_build_is_as_accurate_as_tt_svd(d, n, kern, lo, hi, deg, ps, lmax, eta, tol, prec):
    from paper_2511_03109_gb300 import ph

    P = inputs.uniform_points(n, d, 2100 + n)
    X = inputs.gaussian_rhs(n, 2, 2101 + n)
    built = {}
    for comp in ("svd", "cross"):
        opts = ph.make_opts(d, lo, hi, deg, ps, lmax, eta, tol, rank_cap=64, fmt="h2", prec=prec, compressor=comp)
        built[comp] = ph.ParametricMatrix(P, kern, opts)
    ia, ib = built["svd"].info(), built["cross"].info()
    assert ia["n_far_keys"] == ib["n_far_keys"] > 0
    # the cross is a heuristic: its rounded ranks match TT-SVD's on these tensors up to a few
    assert abs(ia["far_rank_max"] - ib["far_rank_max"]) <= 3, (ia["far_rank_max"], ib["far_rank_max"])
    rows = inputs.sample_rows(n, 300, 2102 + n)
    for th in (lo[0] + 0.3 * (hi[0] - lo[0]), lo[0] + 0.85 * (hi[0] - lo[0])):
        exact = kernels.dense_apply(kern, P, [th], X, rows=rows)
        ea = rel_err_rows(exact, device_apply(built["svd"], [th], X, prec)[rows])
        eb = rel_err_rows(exact, device_apply(built["cross"], [th], X, prec)[rows])
        assert np.all(eb <= 3 * ea + (1e-9 if prec == "fp64" else 1e-5)), (th, ea, eb)
    for A in built.values():
        A.close()
