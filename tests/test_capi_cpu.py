"""CPU-side checks of the C ABI: the library loads, exports every declared symbol, and its
host-only planning (cluster tree and block cluster tree) agrees with the oracle's."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import tree
from paper_2511_03109_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

ph = pytest.importorskip("paper_2511_03109_gb300.ph", reason="libph not built")


def _declared():
    text = open(os.path.join(ROOT, "include", "ph.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ph_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 10
    lib = C.CDLL(ph.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
        assert name in ph.EXPORTED, name


def test_version_string():
    assert b"sm_103a" in ph.ph_version()


@pytest.mark.parametrize("n,d,l_max,eta", [(4096, 2, 3, 1.0), (3000, 3, 2, np.sqrt(3.0)),
                                           (777, 2, 4, np.sqrt(2.0)), (300, 1, 5, 1.0)])
def test_plan_matches_oracle_tree(n, d, l_max, eta):
    P = inputs.uniform_points(n, d, 99 + n)
    counts, perm = ph.plan(P, l_max, eta)
    root = tree.build_cluster_tree(P, l_max)
    near, far = tree.build_block_tree(root, eta)
    lv = tree.leaves(root)
    assert counts["nodes"] == len(tree.all_nodes(root))
    assert counts["leaves"] == len(lv)
    assert counts["near"] == len(near)
    assert counts["far"] == len(far)
    assert counts["near_entries"] == sum(s.n * t.n for s, t in near)
    # cluster order: leaves in depth-first order, original order inside each leaf
    assert np.array_equal(perm, np.concatenate([c.idx for c in lv]))
    # translation classes: (level, offset in box units)
    keys = {(s.level,) + tuple(np.round((t.lo - s.lo) / (s.hi - s.lo)).astype(int)) for s, t in far}
    assert counts["far_keys"] == len(keys)


def test_plan_rejects_points_outside_box():
    P = np.array([[0.5, 1.5]])
    with pytest.raises(ph.PHError) as e:
        ph.plan(P, 2, 1.0)
    assert e.value.status == ph.PH_ERR_INVALID_ARG


def test_build_argument_checks_without_gpu():
    P = inputs.uniform_points(64, 2, 1)
    bad = ph.make_opts(2, [0.1], [1.0], [8], 0, 2, 1.0, 1e-6)  # p_s = 0
    with pytest.raises(ph.PHError) as e:
        ph.ParametricMatrix(P, "gauss", bad)
    assert e.value.status == ph.PH_ERR_INVALID_ARG
    swapped = ph.make_opts(2, [1.0], [0.1], [8], 4, 2, 1.0, 1e-6)  # empty parameter box
    with pytest.raises(ph.PHError):
        ph.ParametricMatrix(P, "gauss", swapped)


def test_null_handle_calls_fail_cleanly():
    th = (C.c_double * 3)(0.5, 0, 0)
    assert ph.ph_instantiate(None, th, None) == ph.PH_ERR_INVALID_ARG
    assert ph.ph_matvec(None, None, 1, 1, None, 1, None) == ph.PH_ERR_INVALID_ARG
    assert ph.ph_last_error(None)
    ph.ph_destroy(None)
    assert ph.ph_instantiate_derivative(None, th, 0, None) == ph.PH_ERR_INVALID_ARG
    assert ph.ph_matvec_batched(None, th, 1, None, 1, 1, None, 1, 1, -1, None) == ph.PH_ERR_INVALID_ARG
    assert ph.ph_set_tensor_cores(None, 1) == ph.PH_ERR_INVALID_ARG
    assert ph.ph_set_overlap(None, 1) == ph.PH_ERR_INVALID_ARG
    assert ph.ph_profile_enable(None, 1) == ph.PH_ERR_INVALID_ARG


def test_wait_bound_selftest_rejects_missing_device():
    waited = C.c_double(-1.0)
    assert ph.ph_selftest_wait_bound(-1, C.byref(waited)) == ph.PH_ERR_INVALID_ARG
    assert waited.value == -1.0  # untouched on error


def test_load_rejects_missing_foreign_old_and_corrupt_files(tmp_path):
    """ph_load refuses files it cannot trust before it touches a device: a missing path, a
    foreign file, the previous format's magic, a truncated file, and a vector length the file
    cannot hold (refused without allocating it)."""
    import struct

    def load(path):
        h = C.c_void_p()
        return ph.ph_load(str(path).encode(), 0, C.byref(h))

    assert load(tmp_path / "missing.ph") == ph.PH_ERR_IO
    (tmp_path / "foreign.ph").write_bytes(b"not a handle at all" * 10)
    assert load(tmp_path / "foreign.ph") == ph.PH_ERR_IO
    (tmp_path / "old.ph").write_bytes(b"PHLIB002" + bytes(4096))
    assert load(tmp_path / "old.ph") == ph.PH_ERR_IO
    (tmp_path / "short.ph").write_bytes(b"PHLIB003" + bytes(3))
    assert load(tmp_path / "short.ph") == ph.PH_ERR_IO
    # the right magic followed by 8-byte words of 2^40: whichever field reads a length first
    # gets an impossible one
    (tmp_path / "huge.ph").write_bytes(b"PHLIB003" + struct.pack("<Q", 1 << 40) * 4096)
    assert load(tmp_path / "huge.ph") == ph.PH_ERR_IO
