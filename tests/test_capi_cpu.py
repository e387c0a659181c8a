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
    for field, value in (("compressor", 2), ("near_unshared", 3)):  # options outside their sets
        o = ph.make_opts(2, [0.1], [1.0], [8], 4, 2, 1.0, 1e-6)
        setattr(o, field, value)
        with pytest.raises(ph.PHError) as e:
            ph.ParametricMatrix(P, "gauss", o)
        assert e.value.status == ph.PH_ERR_INVALID_ARG, field


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
    (tmp_path / "old.ph").write_bytes(b"PHLIB004" + bytes(4096))
    assert load(tmp_path / "old.ph") == ph.PH_ERR_IO
    (tmp_path / "short.ph").write_bytes(b"PHLIB005" + bytes(3))
    assert load(tmp_path / "short.ph") == ph.PH_ERR_IO
    # the right magic followed by 8-byte words of 2^40: whichever field reads a length first
    # gets an impossible one
    (tmp_path / "huge.ph").write_bytes(b"PHLIB005" + struct.pack("<Q", 1 << 40) * 4096)
    assert load(tmp_path / "huge.ph") == ph.PH_ERR_IO


def _handle_file(mutate=None):
    """Bytes of a small, consistent handle file in the library's format (one leaf of 4 points in
    1-D, one near block of rank 1, no far field, FP64), with `mutate(fields)` applied to the
    fields first.  Built here from the format's definition, not by the library."""
    import struct

    f = {
        "opts": ph.make_opts(1, [0.1], [1.0], [1], 2, 0, 1.0, 1e-6, fmt="h2", prec="fp64"),
        "PD": 2, "Delta": 3, "P": 2, "scalar": 8,
        "nb_rank": [1], "nb_off": [0], "nb_toff": [0], "nb_woff": [0, 1],
        "near_elems": 16, "near_theta_elems": 2, "w_elems": 1,
        "perm": [0, 1, 2, 3], "leaves": [0], "near_s": [0], "near_t": [0], "near_by_leaf": [0, 1],
        "far_by_target": [0],
        "node": {"level": 0, "parent": -1, "halves": 0, "begin": 0, "end": 4, "leaf": 0},
        "arenas": [16 * 8, 2 * 8, 0, 0, 0, 4 * 1 * 2 * 8, 2 * 2 * 2 * 8, 0, 0],
    }
    if mutate:
        mutate(f)
    out = bytearray(b"PHLIB005")
    vec = lambda fmt, xs: struct.pack("<Q", len(xs)) + struct.pack("<%d%s" % (len(xs), fmt), *xs)
    out += struct.pack("<i", 0)  # kernel: Gaussian
    out += bytes(f["opts"])
    out += struct.pack("<iiii", f["PD"], f["Delta"], f["P"], f["P"])  # far and near theta-grid sizes
    out += struct.pack("<Qd", f["scalar"], 0.0)
    out += vec("i", f["nb_rank"]) + vec("q", f["nb_off"]) + vec("q", f["nb_toff"]) + vec("i", f["nb_woff"])
    out += vec("i", []) + vec("q", []) + vec("q", [])          # key ranks, core offsets, H offsets
    out += vec("q", []) + vec("q", [])                           # S_b, T_b offsets
    out += vec("q", []) + struct.pack("<q", 0)                   # L/R offsets, L/R elements
    out += vec("q", []) + struct.pack("<q", 0)                   # tensor-core offsets, elements
    out += struct.pack("<7q", f["near_elems"], f["near_theta_elems"], 0, 0, 0, 0, f["w_elems"])
    out += vec("d", [0.0] * 192) + vec("d", [0.0] * 192) + vec("d", [0.0] * 8)  # nodes, weights (2 grids), E
    out += struct.pack("<iqi", 1, 4, 0)                          # plan: d, n, depth
    for key in ("perm", "leaves", "near_s", "near_t"):
        out += vec("i", f[key])
    out += vec("i", []) * 4                                      # far_s, far_t, far_key, key_rep
    out += vec("i", f["near_by_leaf"]) + vec("i", []) + vec("i", f["far_by_target"])
    nd = f["node"]
    out += struct.pack("<Q6i", 1, nd["level"], nd["parent"], nd["halves"], nd["begin"], nd["end"], nd["leaf"])
    out += struct.pack("<6d", 0, 0, 0, 1, 0, 0) + vec("i", [])
    for nbytes in f["arenas"]:
        out += vec("B", [0] * nbytes)
    return bytes(out)


def _set(key, value, index=None):
    def mutate(f):
        if index is None:
            f[key] = value
        else:
            f[key][index] = value
    return mutate


def _node_end(f):
    f["node"]["end"] = 5


def _short_near_arena(f):
    f["arenas"][0] -= 8


def _other_p_s(f):
    f["opts"].p_s = 3


def _bad_sharing_option(f):
    f["opts"].near_unshared = 2


def _bad_compressor(f):
    f["opts"].compressor = 7


@pytest.mark.parametrize("mutate", [
    _set("nb_off", [1]),            # the block's cores would end one entry past the arena
    _set("perm", 4, 0),             # a permutation entry outside 0..n-1
    _set("near_t", 5, 0),           # a near source that is not a node
    _set("nb_woff", [0, 2]),        # weight offsets that disagree with the rank
    _set("nb_rank", [40]),          # a rank above the kernels' limit
    _set("leaves", 1, 0),           # a leaf id that is not a node
    _node_end,                      # a node range past n
    _short_near_arena,              # an arena shorter than its element count (length still consistent)
    _other_p_s,                     # options from another build (p_s^d no longer the stored PD)
    _bad_sharing_option,            # a near-sharing option that is neither 0 nor 1
    _bad_compressor,                # a compressor that is neither TT-SVD nor TT-cross
], ids=["nb_off", "perm", "near_t", "nb_woff", "rank", "leaves", "node_end", "arena", "p_s", "sharing",
        "compressor"])
def test_load_refuses_corrupt_contents(tmp_path, mutate):
    """ph_load checks every stored offset, index and size on the host before it touches a
    device: one flipped value in an otherwise consistent file is refused with PH_ERR_IO."""
    good = tmp_path / "good.ph"
    good.write_bytes(_handle_file())
    h = C.c_void_p()
    st = ph.ph_load(str(good).encode(), 0, C.byref(h))
    # without a GPU the good file passes every check and fails only at the device
    assert st in (ph.PH_OK, ph.PH_ERR_CUDA), ph.ph_last_error(None)
    if st == ph.PH_OK:
        ph.ph_destroy(h)
    bad = tmp_path / "bad.ph"
    bad.write_bytes(_handle_file(mutate))
    h = C.c_void_p()
    assert ph.ph_load(str(bad).encode(), 0, C.byref(h)) == ph.PH_ERR_IO
    assert b"inconsistent handle data" in ph.ph_last_error(None)
    assert not h.value


def _two_leaf_file(mutate=None):
    """A consistent handle file with two leaves of 2 points in 1-D and mirror sharing: near
    blocks (1,1), (1,2), (2,1), (2,2) of rank 1, the block (2,1) reading the cores of (1,2)."""
    import struct

    f = {
        "opts": ph.make_opts(1, [0.1], [1.0], [1], 2, 1, 1.0, 1e-6, fmt="h2", prec="fp64"),
        "nb_rank": [1, 1, 1, 1], "nb_off": [0, 4, 4, 8], "nb_toff": [0, 2, 2, 4], "nb_woff": [0, 1, 2, 3, 4],
        "near_elems": 12, "near_theta_elems": 6, "w_elems": 4,
    }
    if mutate:
        mutate(f)
    out = bytearray(b"PHLIB005")
    vec = lambda fmt, xs: struct.pack("<Q", len(xs)) + struct.pack("<%d%s" % (len(xs), fmt), *xs)
    out += struct.pack("<i", 0) + bytes(f["opts"]) + struct.pack("<iiii", 2, 3, 2, 2) + struct.pack("<Qd", 8, 0.0)
    out += vec("i", f["nb_rank"]) + vec("q", f["nb_off"]) + vec("q", f["nb_toff"]) + vec("i", f["nb_woff"])
    out += vec("i", []) + vec("q", []) + vec("q", []) + vec("q", []) + vec("q", [])
    out += vec("q", []) + struct.pack("<q", 0) + vec("q", []) + struct.pack("<q", 0)
    out += struct.pack("<7q", f["near_elems"], f["near_theta_elems"], 0, 0, 0, 0, f["w_elems"])
    out += vec("d", [0.0] * 192) + vec("d", [0.0] * 192) + vec("d", [0.0] * 8)
    out += struct.pack("<iqi", 1, 4, 1)                          # plan: d, n, depth
    out += vec("i", [0, 1, 2, 3]) + vec("i", [1, 2])             # perm, leaves
    out += vec("i", [1, 1, 2, 2]) + vec("i", [1, 2, 1, 2])       # near_s, near_t
    out += vec("i", []) * 4
    out += vec("i", [0, 2, 4]) + vec("i", []) + vec("i", [0])
    nodes = [(0, -1, 0, 0, 4, -1, 0.0, 1.0, [1, 2]), (1, 0, 0, 0, 2, 0, 0.0, 0.5, []), (1, 0, 1, 2, 4, 1, 0.5, 1.0, [])]
    out += struct.pack("<Q", len(nodes))
    for level, parent, halves, begin, end, leaf, lo, hi, children in nodes:
        out += struct.pack("<6i", level, parent, halves, begin, end, leaf)
        out += struct.pack("<6d", lo, 0, 0, hi, 0, 0) + vec("i", children)
    for nbytes in (12 * 8, 6 * 8, 0, 0, 0, 4 * 1 * 2 * 8, 2 * 2 * 2 * 8, 0, 0):
        out += vec("B", [0] * nbytes)
    return bytes(out)


def test_load_checks_the_mirror_blocks(tmp_path):
    """With mirror sharing the block (t, s) must read exactly the cores of its stored partner
    (s, t): a file where it points elsewhere is refused before anything reaches a device."""
    good = tmp_path / "good.ph"
    good.write_bytes(_two_leaf_file())
    h = C.c_void_p()
    st = ph.ph_load(str(good).encode(), 0, C.byref(h))
    assert st in (ph.PH_OK, ph.PH_ERR_CUDA), ph.ph_last_error(None)
    if st == ph.PH_OK:
        ph.ph_destroy(h)
    for key, value in (("nb_off", [0, 4, 8, 8]), ("nb_toff", [0, 2, 4, 4])):
        bad = tmp_path / f"bad_{key}.ph"
        bad.write_bytes(_two_leaf_file(_set(key, value)))
        h = C.c_void_p()
        assert ph.ph_load(str(bad).encode(), 0, C.byref(h)) == ph.PH_ERR_IO, key
        assert b"mirrored near block" in ph.ph_last_error(None), ph.ph_last_error(None)


def test_alloc_failure_hook_and_check_without_gpu():
    assert ph.ph_inject_alloc_failure(3) == ph.PH_OK
    assert ph.ph_inject_alloc_failure(-1) == ph.PH_OK
    assert ph.ph_check(None, None) == ph.PH_ERR_INVALID_ARG
