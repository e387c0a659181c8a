"""Failure handling on the GPU without faulting it (the device is shared):

* a bounded device wait that runs out is counted in the handle's device flag and reported as
  PH_ERR_TIMEOUT by ph_check and by the next call after the stream passed it, without
  check_finite; the handle then works normally;
* an injected host-side allocation failure (ph_inject_alloc_failure) surfaces as PH_ERR_OOM
  from ph_offline_build and from ph_matvec; the handle stays valid and destroyable.
"""
import ctypes as C

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


def test_timeout_reported_by_check_and_next_call():
    from paper_2511_03109_gb300 import ph

    n = 500
    P = inputs.uniform_points(n, 2, 141)
    X = inputs.gaussian_rhs(n, 2, 142)
    A, M, _ = build_pair(P, "gauss", [0.1], [1.0], [10], 5, 3, 1.0, 1e-9, 0, "h2", "fp64")
    ref = M.matvec(M.instantiate([0.4]), X)
    assert np.all(rel_err_rows(ref, device_apply(A, [0.4], X, "fp64")) <= TOL["fp64"])
    # ph_check reports an expired wait once
    assert ph.ph_selftest_timeout(A.h, None) == ph.PH_OK
    assert ph.ph_check(A.h, None) == ph.PH_ERR_TIMEOUT
    assert b"ran out" in ph.ph_last_error(A.h)
    assert ph.ph_check(A.h, None) == ph.PH_OK
    # without ph_check, the first call after the stream passed the wait reports it and does no work
    assert ph.ph_selftest_timeout(A.h, None) == ph.PH_OK
    torch.cuda.synchronize()
    with pytest.raises(ph.PHError) as e:
        A.instantiate([0.4])
    assert e.value.status == ph.PH_ERR_TIMEOUT
    assert np.all(rel_err_rows(ref, device_apply(A, [0.4], X, "fp64")) <= TOL["fp64"])
    A.close()


def test_injected_allocation_failure_in_build_and_matvec():
    from paper_2511_03109_gb300 import ph

    n = 600
    P = inputs.uniform_points(n, 2, 151)
    X = inputs.gaussian_rhs(n, 3, 152)
    opts = ph.make_opts(2, [0.1], [1.0], [10], 5, 3, 1.0, 1e-8, rank_cap=32, prec="fp64")
    try:
        for after in (0, 3, 12):  # fail at the first, the fourth, the thirteenth allocation
            assert ph.ph_inject_alloc_failure(after) == ph.PH_OK
            with pytest.raises(ph.PHError) as e:
                ph.ParametricMatrix(P, "gauss", opts)
            assert e.value.status == ph.PH_ERR_OOM
            assert b"injected" in ph.ph_last_error(None)
        ph.ph_inject_alloc_failure(-1)
        A, M, _ = build_pair(P, "gauss", [0.1], [1.0], [10], 5, 3, 1.0, 1e-8, 32, "h2", "fp64")
        A.instantiate([0.5])
        Xd = torch.tensor(X.T, dtype=torch.float64, device="cuda:0").contiguous()
        Yd = torch.zeros_like(Xd)
        ph.ph_inject_alloc_failure(0)  # the workspace of the first matvec cannot be allocated
        with pytest.raises(ph.PHError) as e:
            A.matvec_ptr(Xd.data_ptr(), n, 3, Yd.data_ptr(), n)
        assert e.value.status == ph.PH_ERR_OOM
        ph.ph_inject_alloc_failure(-1)
        ref = M.matvec(M.instantiate([0.5]), X)
        assert np.all(rel_err_rows(ref, device_apply(A, [0.5], X, "fp64")) <= TOL["fp64"])
        A.close()
    finally:
        ph.ph_inject_alloc_failure(-1)
