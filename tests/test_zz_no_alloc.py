"""ph_matvec_noalloc: the entry point for callers that cannot allocate device memory when they
apply the matrix (processes held to a fixed device-memory budget, host applications that own
every device allocation, loops that must not stall on cudaMalloc).  It must give ph_matvec's
result, call after call, from the library's static workspace, on a handle that has never
allocated a workspace of its own, and without changing the device's free memory.

This file is collected last on purpose, so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2511_03109_gb300 import inputs

from helpers import TOL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _setup(fmt, prec, m, n=1500):
    from paper_2511_03109_gb300 import ph

    P = inputs.uniform_points(n, 2, 901)
    opts = ph.make_opts(2, [0.05], [0.5], [16], 8, 3, 1.0, 1e-6, rank_cap=32, fmt=fmt, prec=prec)
    A = ph.ParametricMatrix(P, "matern32", opts)
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = torch.tensor(inputs.gaussian_rhs(n, m, 902).T, dtype=dt, device="cuda:0").contiguous()
    return A, X


@pytest.mark.parametrize("fmt,prec,m", [("h2", "fp32", 16), ("h2", "fp64", 3), ("h", "fp32", 5)])
def test_noalloc_matches_matvec_twice(fmt, prec, m):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A, X = _setup(fmt, prec, m)
    n = X.shape[1]
    ref = torch.empty_like(X)
    A.instantiate([0.23])
    A.matvec_ptr(X.data_ptr(), n, m, ref.data_ptr(), n)
    for _ in range(2):  # two calls in a row share (and must reset) the static workspace
        out = torch.full_like(X, float("nan"))
        A.matvec_noalloc_ptr(X.data_ptr(), n, m, out.data_ptr(), n)
        torch.cuda.synchronize()
        r, o = ref.double().cpu().numpy(), out.double().cpu().numpy()
        err = np.linalg.norm(r - o, axis=1) / np.linalg.norm(r, axis=1)
        assert np.all(err <= TOL[prec]), err
    A.close()


def test_noalloc_rejects_oversized_problem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_03109_gb300 import ph

    A, X = _setup("h2", "fp32", 1)
    n = X.shape[1]
    A.instantiate([0.3])
    big = torch.zeros((1024, n), dtype=torch.float32, device="cuda:0")
    with pytest.raises(ph.PHError) as e:
        A.matvec_noalloc_ptr(big.data_ptr(), n, 1024, big.data_ptr() + 0, n)
    assert e.value.status == ph.PH_ERR_INVALID_ARG
    assert "limit" in str(e.value)
    A.close()


@pytest.mark.parametrize("fmt,prec,m", [("h2", "fp32", 16), ("h", "fp64", 2)])
def test_noalloc_on_fresh_handle_allocates_nothing(fmt, prec, m):
    """A handle that has never run ph_matvec: two noalloc calls give ph_matvec's result (called
    afterwards), and the device's free memory is the same before and after the second call."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A, X = _setup(fmt, prec, m)
    n = X.shape[1]
    A.instantiate([0.41])
    outs = [torch.full_like(X, float("nan")) for _ in range(2)]
    A.matvec_noalloc_ptr(X.data_ptr(), n, m, outs[0].data_ptr(), n)  # first call: symbol lookup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    A.matvec_noalloc_ptr(X.data_ptr(), n, m, outs[1].data_ptr(), n)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref = torch.empty_like(X)
    A.matvec_ptr(X.data_ptr(), n, m, ref.data_ptr(), n)
    torch.cuda.synchronize()
    r = ref.double().cpu().numpy()
    for out in outs:
        o = out.double().cpu().numpy()
        err = np.linalg.norm(r - o, axis=1) / np.linalg.norm(r, axis=1)
        assert np.all(err <= TOL[prec]), err
    A.close()
