"""The adjoint X = K_hat(theta)^T Y (ph_matvec_transpose) and the autograd wrapper on the GPU.

* parity with the oracle's matvec_transpose (every block transposed) for both formats, FP64
  (<= 1e-10) and FP32 (<= 1e-5), d = 2 and 3, for the matrix and for its theta-derivative;
* <K_hat x, y> = <x, K_hat^T y> on the device;
* ph.khat_apply under torch.autograd: dX against the oracle's adjoint, d theta against the
  oracle's exact derivative product <dY, dK_hat/dtheta X> and against central finite differences
  of the loss with step 1e-4 (d_theta = 1 and 2)."""
import numpy as np
import pytest

from paper_2511_03109_gb300 import inputs

from helpers import TOL, build_pair, rel_err_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _transpose(A, theta, Y, prec, deriv=None):
    dt = torch.float64 if prec == "fp64" else torch.float32
    n, m = Y.shape
    Yd = torch.tensor(Y.T, dtype=dt, device="cuda:0").contiguous()
    Xd = torch.full_like(Yd, float("nan"))
    if deriv is None:
        A.instantiate(theta)
    else:
        A.instantiate_derivative(theta, deriv)
    A.matvec_transpose_ptr(Yd.data_ptr(), n, m, Xd.data_ptr(), n)
    torch.cuda.synchronize()
    return Xd.double().cpu().numpy().T


CASES = [
    # name, n, d, kernel, lo, hi, degree, p_s, l_max, eta, tol, cap, fmt, prec, m
    ("h2_fp64_d2", 900, 2, "matern52", [0.1], [0.6], [12], 6, 3, 1.0, 1e-9, 32, "h2", "fp64", 3),
    ("h_fp64_d2", 800, 2, "gauss", [0.1], [1.0], [12], 6, 3, 1.0, 1e-9, 32, "h", "fp64", 2),
    ("h2_fp32_d3_m16", 1500, 3, "matern32", [0.05], [0.5], [16], 4, 2, np.sqrt(3.0), 1e-6, 64, "h2", "fp32", 16),
    ("h2_fp64_aniso_d2", 700, 2, "aniso_gauss", [0.1, 0.1], [0.5, 0.5], [4, 5], 6, 3, np.sqrt(2.0), 1e-9, 64, "h2",
     "fp64", 2),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_adjoint_parity(case):
    name, n, d, kern, lo, hi, deg, ps, lmax, eta, tol, cap, fmt, prec, m = case
    P = inputs.uniform_points(n, d, 800 + n)
    Y = inputs.gaussian_rhs(n, m, 801 + n)
    A, M, _ = build_pair(P, kern, lo, hi, deg, ps, lmax, eta, tol, cap, fmt, prec)
    theta = [lo[i] + (0.37 + 0.2 * i) * (hi[i] - lo[i]) for i in range(len(lo))]
    ref = M.matvec_transpose(M.instantiate(theta), Y)
    got = _transpose(A, theta, Y, prec)
    assert np.all(rel_err_rows(ref, got) <= TOL[prec]), (name, rel_err_rows(ref, got))
    for dim in range(len(lo)):
        ref = M.matvec_transpose(M.instantiate(theta, deriv=dim), Y)
        got = _transpose(A, theta, Y, prec, deriv=dim)
        assert np.all(rel_err_rows(ref, got) <= TOL[prec]), (name, "d/dtheta", dim, rel_err_rows(ref, got))
    A.close()


def test_inner_product_identity_on_device():
    n = 1000
    P = inputs.uniform_points(n, 2, 901)
    x = inputs.gaussian_rhs(n, 1, 902)
    y = inputs.gaussian_rhs(n, 1, 903)
    A, _, _ = build_pair(P, "matern32", [0.05], [0.5], [16], 6, 3, 1.0, 1e-7, 32, "h2", "fp64")
    A.instantiate([0.23])
    xd = torch.tensor(x.T, dtype=torch.float64, device="cuda:0").contiguous()
    yd = torch.tensor(y.T, dtype=torch.float64, device="cuda:0").contiguous()
    kx, kty = torch.empty_like(xd), torch.empty_like(yd)
    A.matvec_ptr(xd.data_ptr(), n, 1, kx.data_ptr(), n)
    A.matvec_transpose_ptr(yd.data_ptr(), n, 1, kty.data_ptr(), n)
    torch.cuda.synchronize()
    lhs, rhs = float(torch.dot(kx[0], yd[0])), float(torch.dot(xd[0], kty[0]))
    assert abs(lhs - rhs) <= 1e-12 * float(kx.norm() * yd.norm())
    A.close()


@pytest.mark.parametrize("kern,lo,hi,deg", [("matern52", [0.1], [0.6], [14]),
                                            ("aniso_gauss", [0.1, 0.15], [0.5, 0.6], [6, 5])])
def test_autograd_gradients(kern, lo, hi, deg):
    from paper_2511_03109_gb300 import ph

    n, m = 700, 3
    P = inputs.uniform_points(n, 2, 911)
    X0 = inputs.gaussian_rhs(n, m, 912)
    W = inputs.gaussian_rhs(n, m, 913)
    A, M, _ = build_pair(P, kern, lo, hi, deg, 6, 3, np.sqrt(2.0), 1e-10, 64, "h2", "fp64")
    theta0 = [lo[i] + (0.41 + 0.13 * i) * (hi[i] - lo[i]) for i in range(len(lo))]
    X = torch.tensor(X0, dtype=torch.float64, device="cuda:0", requires_grad=True)
    th = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    Wd = torch.tensor(W, dtype=torch.float64, device="cuda:0")
    loss = torch.sum(ph.khat_apply(A, X, th) * Wd)
    loss.backward()
    # dX = K_hat^T W (oracle adjoint), d theta_i = <W, dK_hat/dtheta_i X> (oracle derivative)
    ref_dx = M.matvec_transpose(M.instantiate(theta0), W)
    assert np.all(rel_err_rows(ref_dx, X.grad.cpu().numpy()) <= 1e-10)
    for i in range(len(lo)):
        exact = float(np.sum(W * M.matvec(M.instantiate(theta0, deriv=i), X0)))
        assert abs(th.grad[i].item() - exact) <= 1e-10 * abs(exact) + 1e-12
        # central finite difference of the loss with step 1e-4 (through the library's forward)
        h = 1e-4
        vals = []
        for sgn in (1.0, -1.0):
            t = list(theta0)
            t[i] += sgn * h
            with torch.no_grad():
                vals.append(float(torch.sum(ph.khat_apply(A, X.detach(), torch.tensor(t, dtype=torch.float64)) * Wd)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - th.grad[i].item()) <= 1e-6 * abs(th.grad[i].item()), (i, fd, th.grad[i].item())
    A.close()
