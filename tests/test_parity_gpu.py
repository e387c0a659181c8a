"""GPU parity of the whole online stage (instantiate + matvec) against the FP64 oracle.

Bar: relative 2-norm error per right-hand side <= 1e-10 on the FP64 path and <= 1e-5 on the
FP32 path, on inputs that span several leaves, ragged leaf sizes, both formats and several m.
"""
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
    # name, n, d, kernel, lo, hi, degree, p_s, l_max, eta, tol, cap, fmt, prec, m
    ("h2_fp64_d2", 1000, 2, "gauss", [0.1], [1.0], [12], 6, 3, 1.0, 1e-8, 32, "h2", "fp64", 3),
    ("h_fp64_d2", 1000, 2, "gauss", [0.1], [1.0], [12], 6, 3, 1.0, 1e-8, 32, "h", "fp64", 1),
    ("h2_fp32_d2_m16", 1500, 2, "matern32", [0.05], [0.5], [20], 8, 3, 1.0, 1e-5, 64, "h2", "fp32", 16),
    ("h_fp32_d2_m5", 1500, 2, "matern52", [0.05], [0.5], [16], 8, 3, np.sqrt(2.0), 1e-5, 64, "h", "fp32", 5),
    ("h2_fp64_d1", 400, 1, "exponential", [0.2], [1.0], [10], 6, 4, 1.0, 1e-9, 0, "h2", "fp64", 2),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_parity_small(case):
    name, n, d, kern, lo, hi, deg, ps, lmax, eta, tol, cap, fmt, prec, m = case
    P = inputs.uniform_points(n, d, 1000 + n)
    X = inputs.gaussian_rhs(n, m, 2000 + n)
    A, M, _ = build_pair(P, kern, lo, hi, deg, ps, lmax, eta, tol, cap, fmt, prec)
    for theta in ([lo[0] + 0.37 * (hi[0] - lo[0])], [lo[0]], [hi[0]]):
        ref = M.matvec(M.instantiate(theta), X)
        got = device_apply(A, theta, X, prec)
        err = rel_err_rows(ref, got)
        assert np.all(err <= TOL[prec]), (name, theta, err)
    A.close()


@pytest.mark.parametrize("coupling", ["explicit", "chain"])
@pytest.mark.parametrize("d,prec,m", [(2, "fp64", 2), (3, "fp32", 16)])
def test_coupling_modes(coupling, d, prec, m):
    """Both H^2 coupling stages: explicit L_k / R_k products and the TT chain (§4.5)."""
    n = 1200 if d == 2 else 2500
    P = inputs.uniform_points(n, d, 55 + d)
    X = inputs.gaussian_rhs(n, m, 56 + d)
    lmax, eta, ps = (3, 1.0, 6) if d == 2 else (2, np.sqrt(3.0), 4)
    A, M, targets = build_pair(P, "matern52", [0.1], [0.6], [12], ps, lmax, eta, 1e-7, 0, "h2", prec,
                               coupling=coupling, targets_every=None if d == 2 else 9)
    rows = None if targets is None else target_rows(targets)
    ref = M.matvec(M.instantiate([0.31], targets), X, targets)
    got = device_apply(A, [0.31], X, prec)
    assert np.all(rel_err_rows(ref, got, rows) <= TOL[prec])
    A.close()


@pytest.mark.parametrize("ps,theta", [(4, 0.13), (8, 0.47)])
def test_tensor_core_phase1_against_cuda_core_and_oracle(ps, theta):
    """FP32, 16 right-hand sides, p_s^d a multiple of 32: phase 1 of the explicit coupling runs on
    the tensor cores (3xTF32) when enabled; the CUDA-core kernel and the oracle must agree with it."""
    n = 2500 if ps == 4 else 6000
    P = inputs.uniform_points(n, 3, 90 + ps)
    X = inputs.gaussian_rhs(n, 16, 91 + ps)
    A, M, targets = build_pair(P, "matern32", [0.05], [0.5], [16], ps, 2, np.sqrt(3.0), 1e-5, 64, "h2", "fp32",
                               targets_every=11 if ps == 4 else 23)
    rows = target_rows(targets)
    ref = M.matvec(M.instantiate([theta], targets), X, targets)
    assert A.info()["tensor_core_phase1"] == 0  # off by default
    y_cc = device_apply(A, [theta], X, "fp32")
    assert not A.info()["kernel_variants"] & 4
    A.set_tensor_cores(True)
    assert A.info()["tensor_core_phase1"] == 1
    y_tc = device_apply(A, [theta], X, "fp32")
    assert A.info()["kernel_variants"] & 4
    assert np.all(rel_err_rows(ref, y_tc, rows) <= TOL["fp32"])
    assert np.all(rel_err_rows(ref, y_cc, rows) <= TOL["fp32"])
    # two FP32 evaluations in different summation orders, each within the FP32 bar of the oracle
    assert np.all(rel_err_rows(y_cc, y_tc) <= TOL["fp32"])
    A.close()


def test_bulk_copy_kernels_match_fallback_kernels():
    """m = 16 takes the bulk-copy near field and phase 2 (one chunk of right-hand sides); m = 17
    takes the register-staged kernels for the same first 16 columns.  Both meet the oracle."""
    n = 2500
    P = inputs.uniform_points(n, 3, 123)
    X = inputs.gaussian_rhs(n, 17, 124)
    A, M, targets = build_pair(P, "matern52", [0.1], [0.6], [12], 4, 2, np.sqrt(3.0), 1e-7, 0, "h2", "fp32",
                               targets_every=9)
    rows = target_rows(targets)
    ref = M.matvec(M.instantiate([0.27], targets), X, targets)
    y16 = device_apply(A, [0.27], X[:, :16], "fp32")
    assert A.info()["kernel_variants"] & 3 == 3
    y17 = device_apply(A, [0.27], X, "fp32")
    assert A.info()["kernel_variants"] & 3 == 0
    assert np.all(rel_err_rows(ref[:, :16], y16, rows) <= TOL["fp32"])
    assert np.all(rel_err_rows(ref, y17, rows) <= TOL["fp32"])
    assert np.all(rel_err_rows(y17[:, :16], y16) <= 2 * TOL["fp32"])
    A.close()


def test_parity_3d_h2_fp32_sampled_rows():
    """3-D Matern 3/2, eta = sqrt(3), 16 right-hand sides; oracle on a sample of target leaves."""
    n = 3000
    P = inputs.uniform_points(n, 3, 77)
    X = inputs.gaussian_rhs(n, 16, 78)
    A, M, targets = build_pair(P, "matern32", [0.05], [0.5], [20], 5, 2, np.sqrt(3.0), 1e-5, 64,
                               "h2", "fp32", targets_every=13)
    rows = target_rows(targets)
    theta = [0.211]
    ref = M.matvec(M.instantiate(theta, targets), X, targets)
    got = device_apply(A, theta, X, "fp32")
    assert np.all(rel_err_rows(ref, got, rows) <= TOL["fp32"])
    A.close()


def test_theta_at_chebyshev_node_and_ragged_ld():
    n = 800
    P = inputs.uniform_points(n, 2, 31)
    X = inputs.gaussian_rhs(n, 17, 32)  # 17 = one full chunk of 16 plus a ragged one
    A, M, _ = build_pair(P, "gauss", [0.1], [1.0], [16], 8, 3, 1.0, 1e-7, 32, "h2", "fp64")
    node = float(cheb.cheb_nodes(0.1, 1.0, 17)[5])
    ref = M.matvec(M.instantiate([node]), X)
    got = device_apply(A, [node], X, "fp64", ldx_pad=13)
    assert np.all(rel_err_rows(ref, got) <= TOL["fp64"])
    A.close()


@pytest.mark.parametrize("fmt", ["h2", "h"])
def test_polynomial_kernel_exact_against_dense(fmt):
    """No truncation and a polynomial kernel of low degree: K_hat(theta) X = K(theta) X to rounding."""
    n = 700
    P = inputs.uniform_points(n, 2, 41)
    X = inputs.gaussian_rhs(n, 2, 42)
    A, _, _ = build_pair(P, "poly", [0.5], [2.0], [2], 5, 3, 1.0, 0.0, 0, fmt, "fp64")
    for theta in ([0.5], [1.234], [2.0]):
        exact = kernels.dense_apply("poly", P, theta, X)
        assert np.all(rel_err_rows(exact, device_apply(A, theta, X, "fp64")) <= 1e-11)
    A.close()


def test_no_far_field_and_single_leaf():
    P = inputs.uniform_points(300, 2, 51)
    X = inputs.gaussian_rhs(300, 1, 52)
    for lmax in (0, 1):
        A, M, _ = build_pair(P, "gauss", [0.1], [1.0], [10], 4, lmax, 1.0, 1e-9, 0, "h2", "fp64")
        assert A.info()["n_far"] == 0
        ref = M.matvec(M.instantiate([0.3]), X)
        assert np.all(rel_err_rows(ref, device_apply(A, [0.3], X, "fp64")) <= TOL["fp64"])
        A.close()


def test_dedup_matches_per_block_compression():
    P = inputs.uniform_points(900, 2, 61)
    X = inputs.gaussian_rhs(900, 2, 62)
    A1, M, _ = build_pair(P, "matern52", [0.1], [0.6], [10], 6, 3, 1.0, 1e-9, 0, "h2", "fp64", dedup=True)
    A2, _, _ = build_pair(P, "matern52", [0.1], [0.6], [10], 6, 3, 1.0, 1e-9, 0, "h2", "fp64", dedup=False)
    assert A1.info()["n_far_keys"] < A2.info()["n_far_keys"] == A2.info()["n_far"]
    y1 = device_apply(A1, [0.44], X, "fp64")
    y2 = device_apply(A2, [0.44], X, "fp64")
    assert np.all(rel_err_rows(y2, y1) <= 1e-11)
    A1.close()
    A2.close()


def test_errors_are_status_codes():
    from paper_2511_03109_gb300 import ph

    P = inputs.uniform_points(200, 2, 71)
    opts = ph.make_opts(2, [0.1], [1.0], [8], 4, 2, 1.0, 1e-6, prec="fp64", check_finite=True)
    A = ph.ParametricMatrix(P, "gauss", opts)
    X = torch.zeros((1, 200), dtype=torch.float64, device="cuda:0")
    Y = torch.zeros_like(X)
    with pytest.raises(ph.PHError) as e:
        A.matvec_ptr(X.data_ptr(), 200, 1, Y.data_ptr(), 200)
    assert e.value.status == ph.PH_ERR_NOT_INSTANTIATED
    with pytest.raises(ph.PHError) as e:
        A.instantiate([1.5])
    assert e.value.status == ph.PH_ERR_THETA_OUT_OF_BOX
    with pytest.raises(ph.PHError) as e:
        A.instantiate([float("nan")])
    assert e.value.status == ph.PH_ERR_NONFINITE
    A.instantiate([0.5])
    X[0, 17] = float("inf")
    with pytest.raises(ph.PHError) as e:
        A.matvec_ptr(X.data_ptr(), 200, 1, Y.data_ptr(), 200)
    assert e.value.status == ph.PH_ERR_NONFINITE
    with pytest.raises(ph.PHError) as e:
        A.matvec_ptr(X.data_ptr(), 100, 1, Y.data_ptr(), 200)  # ldx < n
    assert e.value.status == ph.PH_ERR_INVALID_ARG
    A.close()


DERIV_CASES = [
    # name, n, d, kernel, lo, hi, degree, p_s, l_max, eta, tol, fmt, prec, m, targets_every
    ("h2_fp64_d2", 1200, 2, "matern52", [0.1], [0.6], [12], 6, 3, 1.0, 1e-9, "h2", "fp64", 2, None),
    ("h_fp64_d2", 1000, 2, "gauss", [0.2], [0.9], [14], 6, 3, 1.0, 1e-9, "h", "fp64", 3, None),
    ("h2_fp32_d3_m16", 2500, 3, "matern32", [0.05], [0.5], [20], 4, 2, np.sqrt(3.0), 1e-6, "h2", "fp32", 16, 9),
]


@pytest.mark.parametrize("case", DERIV_CASES, ids=[c[0] for c in DERIV_CASES])
def test_theta_derivative_parity(case):
    """dK_hat/dtheta X (ph_instantiate_derivative + ph_matvec) against the oracle's derivative
    instantiation, inside the box, at both ends and at a Chebyshev node (the node branch of the
    barycentric derivative)."""
    name, n, d, kern, lo, hi, deg, ps, lmax, eta, tol, fmt, prec, m, every = case
    P = inputs.uniform_points(n, d, 300 + n)
    X = inputs.gaussian_rhs(n, m, 301 + n)
    A, M, targets = build_pair(P, kern, lo, hi, deg, ps, lmax, eta, tol, 0, fmt, prec, targets_every=every)
    rows = None if targets is None else target_rows(targets)
    node = float(cheb.cheb_nodes(lo[0], hi[0], deg[0] + 1)[3])
    for theta in ([lo[0] + 0.43 * (hi[0] - lo[0])], [lo[0]], [hi[0]], [node]):
        ref = M.matvec(M.instantiate(theta, targets, deriv=0), X, targets)
        got = device_apply(A, theta, X, prec, deriv=0)
        err = rel_err_rows(ref, got, rows)
        assert np.all(err <= TOL[prec]), (name, theta, err)
    from paper_2511_03109_gb300 import ph
    with pytest.raises(ph.PHError) as e:
        A.instantiate_derivative([lo[0]], 1)
    assert e.value.status == ph.PH_ERR_INVALID_ARG
    A.close()


def _batched(A, thetas, X, prec, deriv=-1, ldy_pad=3):
    """ph_matvec_batched on cuda:0: returns (len(thetas), n, m)."""
    dt = torch.float64 if prec == "fp64" else torch.float32
    n, m = X.shape
    ldy = n + ldy_pad
    Xd = torch.tensor(X.T, dtype=dt, device="cuda:0").contiguous()
    Yd = torch.full((len(thetas), m, ldy), float("nan"), dtype=dt, device="cuda:0")
    A.matvec_batched_ptr(list(thetas), Xd.data_ptr(), n, m, Yd.data_ptr(), ldy, m * ldy, deriv)
    torch.cuda.synchronize()
    return Yd[:, :, :n].double().cpu().numpy().transpose(0, 2, 1)


@pytest.mark.parametrize("prec,d,m", [("fp64", 2, 3), ("fp32", 3, 16)])
def test_batched_theta_products(prec, d, m):
    """ph_matvec_batched: with at least p_theta values of theta it combines the products at the
    theta nodes, with fewer it applies each theta; both against the oracle per theta, for the
    matrix and its theta-derivative, and the two routes against each other."""
    from paper_2511_03109_gb300 import ph

    n = 1200 if d == 2 else 2500
    P = inputs.uniform_points(n, d, 410 + d)
    X = inputs.gaussian_rhs(n, m, 411 + d)
    lmax, eta, ps = (3, 1.0, 6) if d == 2 else (2, np.sqrt(3.0), 4)
    lo, hi, deg = [0.1], [0.6], [12]
    A, M, targets = build_pair(P, "matern52", lo, hi, deg, ps, lmax, eta, 1e-7, 0, "h2", prec,
                               targets_every=None if d == 2 else 9)
    rows = None if targets is None else target_rows(targets)
    node = float(cheb.cheb_nodes(lo[0], hi[0], deg[0] + 1)[2])
    many = [0.1, 0.6, node] + list(np.linspace(0.13, 0.57, 14))  # 17 >= p_theta = 13
    few = many[:5]
    for deriv in (-1, 0):
        Ym = _batched(A, many, X, prec, deriv)
        Yf = _batched(A, few, X, prec, deriv)
        for t in (0, 1, 2, 3, 4):
            ref = M.matvec(M.instantiate([many[t]], targets, deriv=None if deriv < 0 else 0), X, targets)
            assert np.all(rel_err_rows(ref, Ym[t], rows) <= TOL[prec]), (deriv, t, "nodes")
            assert np.all(rel_err_rows(ref, Yf[t], rows) <= TOL[prec]), (deriv, t, "direct")
            assert np.all(rel_err_rows(Yf[t], Ym[t], rows) <= 2 * TOL[prec])
        t = 11
        ref = M.matvec(M.instantiate([many[t]], targets, deriv=None if deriv < 0 else 0), X, targets)
        assert np.all(rel_err_rows(ref, Ym[t], rows) <= TOL[prec])
    dt = torch.float64 if prec == "fp64" else torch.float32
    Xd = torch.zeros((m, n), dtype=dt, device="cuda:0")
    Yd = torch.zeros((2, m, n), dtype=dt, device="cuda:0")
    with pytest.raises(ph.PHError) as e:  # blocks would overlap
        A.matvec_batched_ptr([0.2, 0.3], Xd.data_ptr(), n, m, Yd.data_ptr(), n, n * m - 1)
    assert e.value.status == ph.PH_ERR_INVALID_ARG
    with pytest.raises(ph.PHError) as e:
        A.matvec_batched_ptr([0.2, 0.7], Xd.data_ptr(), n, m, Yd.data_ptr(), n, n * m)
    assert e.value.status == ph.PH_ERR_THETA_OUT_OF_BOX
    A.close()


def test_bounded_device_wait_returns_timeout_and_context_survives():
    """The device-side wait bound: a wait on an mbarrier nothing arrives on gives up after about
    a second and reports PH_ERR_TIMEOUT; the context keeps working afterwards."""
    from paper_2511_03109_gb300 import ph

    st, waited = ph.selftest_wait_bound(0)
    assert st == ph.PH_ERR_TIMEOUT
    assert 0.9 <= waited <= 5.0, waited
    n = 500
    P = inputs.uniform_points(n, 2, 131)
    X = inputs.gaussian_rhs(n, 2, 132)
    A, M, _ = build_pair(P, "gauss", [0.1], [1.0], [10], 5, 3, 1.0, 1e-9, 0, "h2", "fp64")
    ref = M.matvec(M.instantiate([0.4]), X)
    assert np.all(rel_err_rows(ref, device_apply(A, [0.4], X, "fp64")) <= TOL["fp64"])
    A.close()


def test_host_entry_point_and_save_load(tmp_path):
    from paper_2511_03109_gb300 import ph

    n = 600
    P = inputs.uniform_points(n, 2, 81)
    X = inputs.gaussian_rhs(n, 4, 82)
    opts = ph.make_opts(2, [0.1], [1.0], [10], 6, 3, 1.0, 1e-7, rank_cap=32, prec="fp32")
    A = ph.ParametricMatrix(P, "gauss", opts)
    ref = device_apply(A, [0.6], X, "fp32")
    Xh = np.asfortranarray(X, dtype=np.float32)
    Yh = np.zeros_like(Xh)
    A.matvec_host_ptr(Xh.ctypes.data, n, 4, Yh.ctypes.data, n)
    # far-field partial sums meet through atomic adds, so runs agree to rounding, not bitwise
    assert np.all(rel_err_rows(ref, Yh.astype(np.float64)) <= 1e-6)
    path = str(tmp_path / "a.ph")
    A.save(path)
    B = ph.ParametricMatrix.load(path)
    assert B.info()["near_bytes"] == A.info()["near_bytes"]
    assert np.all(rel_err_rows(ref, device_apply(B, [0.6], X, "fp32")) <= 1e-6)
    A.close()
    B.close()
