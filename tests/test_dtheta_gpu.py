"""Parameter dimension d_theta > 1 on the GPU against the FP64 oracle (§4.3: near weights as the
product over the parameter cores; App. A.4: H_b(theta) as the product of the parameter-core
matrices).  Covers the first near-field TT cut by QR + Jacobi SVD (at most 32 theta-grid points)
and by the Gram eigendecomposition (more points), both formats, FP64 and FP32, theta inside the
box, at a corner and at a grid node, the value and each theta-derivative; and exact reproduction
of a two-parameter polynomial kernel.  Bars: 1e-10 (FP64), 1e-5 (FP32)."""
import numpy as np
import pytest

from oracle import cheb, kernels
from paper_2511_03109_gb300 import inputs

from helpers import TOL, build_pair, device_apply, rel_err_rows, target_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [
    # name, d, degrees, fmt, prec, m, n, p_s, l_max, tol
    ("d2_p30_h2_fp64", 2, [4, 5], "h2", "fp64", 2, 1100, 6, 3, 1e-8),   # 30 grid points: QR + Jacobi SVD
    ("d2_p56_h2_fp64", 2, [6, 7], "h2", "fp64", 1, 1100, 6, 3, 1e-8),   # 56 grid points: Gram path
    ("d2_p56_h_fp64", 2, [6, 7], "h", "fp64", 2, 1000, 6, 3, 1e-8),
    ("d2_p56_h2_fp32", 2, [6, 7], "h2", "fp32", 16, 1500, 8, 3, 1e-6),
    ("d3_p36_h2_fp32", 3, [2, 2, 3], "h2", "fp32", 16, 2500, 4, 2, 1e-6),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_aniso_gauss_parity(case):
    name, d, deg, fmt, prec, m, n, ps, lmax, tol = case
    lo, hi = [0.1] * d, [0.5] * d
    P = inputs.uniform_points(n, d, 500 + n + d)
    X = inputs.gaussian_rhs(n, m, 600 + n)
    eta = float(np.sqrt(d))
    A, M, targets = build_pair(P, "aniso_gauss", lo, hi, deg, ps, lmax, eta, tol, 64, fmt, prec,
                               targets_every=None if d == 2 else 9)
    rows = None if targets is None else target_rows(targets)
    node = [float(cheb.cheb_nodes(lo[i], hi[i], deg[i] + 1)[1]) for i in range(d)]
    inside = [lo[i] + (0.31 + 0.17 * i) * (hi[i] - lo[i]) for i in range(d)]
    for theta in (inside, list(lo), list(hi[:1]) + list(lo[1:]), node):
        ref = M.matvec(M.instantiate(theta, targets), X, targets)
        got = device_apply(A, theta, X, prec)
        err = rel_err_rows(ref, got, rows)
        assert np.all(err <= TOL[prec]), (name, theta, err)
    for dim in range(d):
        ref = M.matvec(M.instantiate(inside, targets, deriv=dim), X, targets)
        got = device_apply(A, inside, X, prec, deriv=dim)
        err = rel_err_rows(ref, got, rows)
        assert np.all(err <= TOL[prec]), (name, "d/dtheta", dim, err)
    A.close()


@pytest.mark.parametrize("fmt", ["h2", "h"])
def test_two_parameter_polynomial_kernel_exact(fmt):
    """No truncation: K_hat(theta) X = K(theta) X to rounding for any theta in the box."""
    n = 500
    P = inputs.uniform_points(n, 2, 71)
    X = inputs.gaussian_rhs(n, 2, 72)
    A, _, _ = build_pair(P, "poly2", [0.5, 0.2], [2.0, 1.5], [1, 2], 5, 3, 1.0, 0.0, 0, fmt, "fp64")
    for theta in ([0.5, 0.2], [1.234, 0.77], [2.0, 1.5]):
        exact = kernels.dense_apply("poly2", P, theta, X)
        assert np.all(rel_err_rows(exact, device_apply(A, theta, X, "fp64")) <= 1e-11)
    A.close()


def test_dtheta_options_checked():
    from paper_2511_03109_gb300 import ph

    P = inputs.uniform_points(100, 2, 3)
    with pytest.raises(ph.PHError) as e:  # one-parameter kernel with two parameters
        ph.ParametricMatrix(P, "gauss", ph.make_opts(2, [0.1, 0.1], [1.0, 1.0], [3, 3], 4, 2, 1.0, 1e-6))
    assert e.value.status == ph.PH_ERR_INVALID_ARG
    P3 = inputs.uniform_points(100, 3, 4)
    with pytest.raises(ph.PHError) as e:  # 16^3 > 1024 theta-grid points
        ph.ParametricMatrix(P3, "aniso_gauss", ph.make_opts(3, [0.1] * 3, [1.0] * 3, [15] * 3, 4, 1, 1.8, 1e-6))
    assert e.value.status == ph.PH_ERR_UNSUPPORTED
