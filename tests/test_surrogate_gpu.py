"""The learned surrogate of the far-field cores on the GPU (ph_far_project, ph_instantiate_cores,
ph_surrogate_train / _use, ph_mlp_check).

* the network kernels (forward, loss, backward; BF16 weights, FP32 accumulation) against the FP64
  oracle perceptron with the same (BF16-representable) weights;
* the projected cores H*_k(theta) (training targets) against the oracle's per-block projection,
  compared through the gauge-invariant product K_hat X: <= 1e-10 (FP64), <= 1e-5 (FP32);
* training on the GPU lowers the loss, and with a coarse far-field tensor grid the trained network
  beats the polynomial path on validation thetas, and in the product its far-field error (against
  the product with the exact projected cores) is the smaller one (what the network gains);
* an untrained network is not accepted: ph_surrogate_use refuses and the polynomial path stays."""
import numpy as np
import pytest

from oracle import kernels, mlp
from paper_2511_03109_gb300 import inputs

from helpers import TOL, build_pair, device_apply, rel_err_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bf16(x):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("n_in,hidden,n_out,B", [(3, 32, 37, 5), (2, 64, 300, 17), (3, 256, 1000, 64),
                                                 (3, 64, 20000, 32)])  # the last splits K = n_out over CTAs
def test_network_kernels_match_the_oracle(n_in, hidden, n_out, B):
    from paper_2511_03109_gb300 import ph

    rng = np.random.default_rng(n_out)
    p = mlp.init_params(n_in, hidden, n_out, seed=hidden)
    for k in ("W1", "W2", "W3"):
        p[k] = _bf16(p[k]).astype(np.float64)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape).astype(np.float32).astype(np.float64) * 0.2
    flat = np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]])
    U = rng.uniform(-1, 1, (B, n_in)).astype(np.float32)
    T = rng.standard_normal((B, n_out)).astype(np.float32)
    Y, g, loss = ph.mlp_check(n_in, hidden, n_out, flat.astype(np.float32), U, T)
    Yo, cache = mlp.forward(p, U.astype(np.float64))
    np.testing.assert_allclose(Y, Yo, rtol=0, atol=2e-5 * np.abs(Yo).max())
    Lo, go = mlp.loss_and_grad(p, U.astype(np.float64), T.astype(np.float64))
    assert abs(loss - Lo) <= 1e-5 * Lo
    off = 0
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        n = go[k].size
        gk = g[off:off + n].reshape(go[k].shape)
        off += n
        np.testing.assert_allclose(gk, go[k], rtol=0, atol=1e-4 * np.abs(go[k]).max() + 1e-12, err_msg=k)


CASES = [
    # name, n, d, kernel, lo, hi, degree, p_s, l_max, eta, tol, cap, prec, every (oracle target leaves)
    ("fp64_d2_matern52", 900, 2, "matern52", [0.1], [0.6], [10], 5, 3, 1.0, 1e-8, 32, "fp64", None),
    ("fp32_d2_gauss", 900, 2, "gauss", [0.1], [1.0], [10], 5, 3, 1.0, 1e-6, 32, "fp32", None),
    ("fp32_d3_aniso", 1200, 3, "aniso_gauss", [0.1] * 3, [0.5] * 3, [3, 3, 3], 4, 2, np.sqrt(3.0), 1e-5, 32, "fp32",
     9),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_projected_cores_match_the_oracle(case):
    from helpers import target_rows

    name, n, d, kern, lo, hi, deg, ps, lmax, eta, tol, cap, prec, every = case
    P = inputs.uniform_points(n, d, 1700 + n)
    X = inputs.gaussian_rhs(n, 3, 1701 + n)
    A, M, targets = build_pair(P, kern, lo, hi, deg, ps, lmax, eta, tol, cap, "h2", prec, targets_every=every)
    rows = target_rows(targets) if targets else None
    dt = torch.float64 if prec == "fp64" else torch.float32
    ne = A.info()["far_core_elems"]
    thetas = [[lo[k] + (0.23 + 0.31 * t + 0.1 * k) % 1.0 * (hi[k] - lo[k]) for k in range(len(lo))] for t in range(3)]
    out = torch.full((len(thetas), ne), float("nan"), dtype=dt, device="cuda:0")
    A.far_project_ptr(thetas, out.data_ptr())
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    for t, th in enumerate(thetas):
        ref = M.matvec(M.instantiate_projected(th, targets), X, targets)
        A.instantiate_cores_ptr(th, out[t].data_ptr())
        Xd = torch.tensor(X.T, dtype=dt, device="cuda:0").contiguous()
        Yd = torch.empty_like(Xd)
        A.matvec_ptr(Xd.data_ptr(), n, 3, Yd.data_ptr(), n)
        torch.cuda.synchronize()
        got = Yd.double().cpu().numpy().T
        err = rel_err_rows(ref, got, rows)
        assert np.all(err <= TOL[prec]), (name, t, err)
    A.close()


def _aniso_handle(far_degree, seed=1900, n=2000):
    from paper_2511_03109_gb300 import ph

    P = inputs.uniform_points(n, 3, seed)
    opts = ph.make_opts(3, [0.05] * 3, [0.5] * 3, [far_degree] * 3, 4, 2, np.sqrt(3.0), 1e-5, rank_cap=16,
                        fmt="h2", prec="fp32", near_degree=[4] * 3)
    return P, ph.ParametricMatrix(P, "aniso_gauss", opts)


def test_trained_network_beats_a_coarse_tensor_grid():
    P, A = _aniso_handle(far_degree=2)
    assert A.info()["p_theta"] == [3, 3, 3] and A.info()["p_theta_near"] == [5, 5, 5]
    tt = inputs.uniform_thetas([0.05] * 3, [0.5] * 3, 2048, 1901)
    tv = inputs.uniform_thetas([0.05] * 3, [0.5] * 3, 64, 1902)
    rep = A.surrogate_train(tt, tv, hidden=256, steps=1500, batch=256, lr=1e-3, seed=3)
    assert rep["loss_last"] < 0.5 * rep["loss_first"], rep
    assert rep["val_err_net_rms"] < rep["val_err_poly_rms"], rep
    assert rep["accepted"] == 1 and rep["out_dim"] == A.info()["far_core_elems"]
    # in the product: the far-field part of the error against the product with the exact projected
    # cores (same spatial factors, same near field), network against polynomial cores; and the
    # total error against the exact K(theta) X, which the near grid and the rank cap also enter
    n = P.shape[0]
    X = inputs.gaussian_rhs(n, 2, 1903)
    rows = inputs.sample_rows(n, 300, 1904)
    cores = torch.empty((1, A.info()["far_core_elems"]), dtype=torch.float32, device="cuda:0")
    Xd = torch.tensor(X.T, dtype=torch.float32, device="cuda:0").contiguous()
    Yd = torch.empty_like(Xd)
    far_err = {False: [], True: []}
    total = {False: [], True: []}
    for th in tv[:4]:
        A.far_project_ptr([th], cores.data_ptr())
        A.instantiate_cores_ptr(th, cores.data_ptr())
        A.matvec_ptr(Xd.data_ptr(), n, 2, Yd.data_ptr(), n)
        torch.cuda.synchronize()
        ystar = Yd.double().cpu().numpy().T
        exact = kernels.dense_apply("aniso_gauss", P, th, X, rows=rows)
        for use in (False, True):
            A.surrogate_use(use)
            got = device_apply(A, th, X, "fp32")
            far_err[use].append(float(np.max(rel_err_rows(ystar, got))))
            total[use].append(float(np.max(rel_err_rows(exact, got[rows]))))
    assert max(far_err[True]) < max(far_err[False]), (far_err, total)
    assert max(total[True]) < 1.5 * max(total[False]), (far_err, total)
    A.close()


def test_untrained_network_is_refused_and_the_polynomial_path_stays():
    from paper_2511_03109_gb300 import ph

    P, A = _aniso_handle(far_degree=4, n=1200)
    tt = inputs.uniform_thetas([0.05] * 3, [0.5] * 3, 64, 1911)
    tv = inputs.uniform_thetas([0.05] * 3, [0.5] * 3, 8, 1912)
    X = inputs.gaussian_rhs(P.shape[0], 2, 1913)
    before = device_apply(A, tv[0], X, "fp32")
    rep = A.surrogate_train(tt, tv, hidden=16, steps=1, batch=16, seed=5)
    assert rep["accepted"] == 0 and rep["val_err_net_rms"] > rep["val_err_poly_rms"], rep
    with pytest.raises(ph.PHError) as e:
        A.surrogate_use(True)
    assert e.value.status == ph.PH_ERR_UNSUPPORTED
    after = device_apply(A, tv[0], X, "fp32")
    # the same polynomial path (the up-sweep accumulates with atomics: equal to FP32 rounding)
    np.testing.assert_allclose(after, before, rtol=0, atol=1e-6 * np.abs(before).max())
    A.close()


def test_surrogate_calls_check_their_arguments():
    from paper_2511_03109_gb300 import ph

    P = inputs.uniform_points(500, 2, 1921)
    A = ph.ParametricMatrix(P, "gauss", ph.make_opts(2, [0.1], [1.0], [6], 4, 2, 1.0, 1e-6, fmt="h", prec="fp32"))
    with pytest.raises(ph.PHError) as e:
        A.surrogate_train([[0.5]], [[0.5]])
    assert e.value.status == ph.PH_ERR_UNSUPPORTED
    A.close()
    A = ph.ParametricMatrix(P, "gauss", ph.make_opts(2, [0.1], [1.0], [6], 4, 2, 1.0, 1e-6, prec="fp32"))
    with pytest.raises(ph.PHError) as e:
        A.surrogate_train([[1.5]], [[0.5]])
    assert e.value.status == ph.PH_ERR_THETA_OUT_OF_BOX
    with pytest.raises(ph.PHError) as e:
        A.surrogate_use(True)
    assert e.value.status == ph.PH_ERR_UNSUPPORTED
    A.close()
