"""Mirror sharing of near blocks on the GPU (§4.3 with a symmetric kernel): each unordered near
pair {s, t} is compressed and stored once and the block (t, s) is applied as D_st(theta)^T.

* the near part alone (eta = 1e-3: no box pair is admissible, every block is near) is exactly symmetric with sharing:
  <x, K_hat y> = <y, K_hat x> to rounding, on the bulk-copy kernel (m = 4 in FP64, 16 in FP32)
  and on the register-staged kernel with its separate mirror kernel (m = 17: two chunks of 16);
* shared and unshared handles both match the oracle, which compresses and stores every block
  (both mirrors) separately: <= 1e-10 (FP64) and <= 1e-5 (FP32), both near kernels, the
  forward product, the theta-derivative and the adjoint;
* the shared handle stores about half the near cores, and survives save / load."""
import numpy as np
import pytest

from paper_2511_03109_gb300 import inputs

from helpers import TOL, build_pair, device_apply, rel_err_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _transpose(A, theta, Y, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    n, m = Y.shape
    Yd = torch.tensor(Y.T, dtype=dt, device="cuda:0").contiguous()
    Xd = torch.full_like(Yd, float("nan"))
    A.instantiate(theta)
    A.matvec_transpose_ptr(Yd.data_ptr(), n, m, Xd.data_ptr(), n)
    torch.cuda.synchronize()
    return Xd.double().cpu().numpy().T


@pytest.mark.parametrize("prec,m", [("fp64", 4), ("fp64", 17), ("fp32", 16), ("fp32", 17)])
def test_near_part_is_symmetric(prec, m):
    from paper_2511_03109_gb300 import ph

    n, d = 1200, 2
    P = inputs.uniform_points(n, d, 1201)
    opts = ph.make_opts(d, [0.1], [0.6], [10], 6, 2, 1e-3, 1e-9 if prec == "fp64" else 1e-6, rank_cap=32,
                        fmt="h2", prec=prec)
    A = ph.ParametricMatrix(P, "matern52", opts)
    info = A.info()
    assert info["n_far"] == 0 and info["n_near"] == 16 * 16
    X = inputs.gaussian_rhs(n, m, 1202)
    Yr = inputs.gaussian_rhs(n, m, 1203)
    KX = device_apply(A, [0.27], X, prec)
    KY = device_apply(A, [0.27], Yr, prec)
    lhs = np.einsum("ic,ic->c", Yr, KX)
    rhs = np.einsum("ic,ic->c", X, KY)
    scale = np.linalg.norm(Yr, axis=0) * np.linalg.norm(KX, axis=0)
    bar = 1e-13 if prec == "fp64" else 1e-5
    assert np.all(np.abs(lhs - rhs) <= bar * scale), (prec, m, np.abs(lhs - rhs) / scale)
    bulk = A.info()["kernel_variants"] & 1  # bit 0: the bulk-copy near kernel ran
    assert bulk == (1 if m in (4, 16) else 0), (m, A.info()["kernel_variants"])
    A.close()


CASES = [
    # name, n, d, kernel, lo, hi, degree, p_s, l_max, eta, tol, cap, fmt, prec, m
    ("h2_fp64_d2_m4", 1500, 2, "matern52", [0.1], [0.6], [12], 6, 3, 1.0, 1e-9, 32, "h2", "fp64", 4),
    ("h_fp64_d2_m3", 1000, 2, "gauss", [0.1], [1.0], [12], 6, 3, 1.0, 1e-9, 32, "h", "fp64", 3),
    ("h2_fp32_d3_m16", 3000, 3, "matern32", [0.05], [0.5], [16], 4, 2, np.sqrt(3.0), 1e-6, 64, "h2", "fp32", 16),
    ("h2_fp32_d3_m17", 3000, 3, "matern32", [0.05], [0.5], [16], 4, 2, np.sqrt(3.0), 1e-6, 64, "h2", "fp32", 17),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_shared_and_unshared_match_the_oracle(case, tmp_path):
    from paper_2511_03109_gb300 import ph

    name, n, d, kern, lo, hi, deg, ps, lmax, eta, tol, cap, fmt, prec, m = case
    P = inputs.uniform_points(n, d, 1300 + n)
    X = inputs.gaussian_rhs(n, m, 1301 + n)
    A, M, _ = build_pair(P, kern, lo, hi, deg, ps, lmax, eta, tol, cap, fmt, prec)
    B, _, _ = build_pair(P, kern, lo, hi, deg, ps, lmax, eta, tol, cap, fmt, prec, near_shared=False)
    ia, ib = A.info(), B.info()
    assert ia["n_near"] == ib["n_near"] and ia["near_entries"] == ib["near_entries"]
    # the stored pairs: every off-diagonal pair once plus the diagonal blocks
    assert ia["near_bytes"] < 0.6 * ib["near_bytes"], (ia["near_bytes"], ib["near_bytes"])
    theta = [0.33 * (lo[0] + hi[0])]
    inst = M.instantiate(theta)
    ref = M.matvec(inst, X)
    for H in (A, B):
        got = device_apply(H, theta, X, prec)
        assert np.all(rel_err_rows(ref, got) <= TOL[prec]), (name, rel_err_rows(ref, got))
    ref_d = M.matvec(M.instantiate(theta, deriv=0), X)
    got_d = device_apply(A, theta, X, prec, deriv=0)
    assert np.all(rel_err_rows(ref_d, got_d) <= TOL[prec]), (name, "d/dtheta", rel_err_rows(ref_d, got_d))
    ref_t = M.matvec_transpose(inst, X)
    for H in (A, B):
        got_t = _transpose(H, theta, X, prec)
        assert np.all(rel_err_rows(ref_t, got_t) <= TOL[prec]), (name, "adjoint", rel_err_rows(ref_t, got_t))
    # save / load keeps the sharing
    path = str(tmp_path / "shared.ph")
    A.save(path)
    C = ph.ParametricMatrix.load(path)
    assert C.info()["near_bytes"] == ia["near_bytes"]
    got = device_apply(C, theta, X, prec)
    assert np.all(rel_err_rows(ref, got) <= TOL[prec]), (name, "loaded", rel_err_rows(ref, got))
    for H in (A, B, C):
        H.close()
