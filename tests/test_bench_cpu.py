"""Host-side checks of bench.py's bookkeeping (no GPU): every kernel it can name exists in the
CUDA source, every DRAM-traffic record matches the current source of its kernel, and the
workload it reports is the 65536-point 3-D Matern 3/2 problem."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_named_kernel_exists(bench):
    names = set(bench.KERNEL_OF_KIND.values())
    for kind in ("near", "coupling", "coupling_b"):
        for var in (0, 1, 2, 4, 7):
            names.add(bench.kernel_of(kind, {"kernel_variants": var}))
    for name in names:
        assert bench.kernel_source_hash(name), name


def test_variant_bits_pick_the_launched_kernels(bench):
    assert bench.kernel_of("near", {"kernel_variants": 1}) == "near_tma_kernel"
    assert bench.kernel_of("near", {"kernel_variants": 0}) == "near_kernel"
    assert bench.kernel_of("coupling_b", {"kernel_variants": 2}) == "coupling_b_tma_kernel"
    assert bench.kernel_of("coupling", {"kernel_variants": 4}) == "coupling_a_umma_kernel"
    assert bench.kernel_of("coupling", {"kernel_variants": 3}) == "coupling_a_staged_kernel"


def test_traffic_records_follow_the_kernel_sources(bench):
    """A record reaches the bench line only while its kernel's source is the one captured."""
    with open(os.path.join(ROOT, "profiles", "kernel_traffic.json")) as f:
        rec = json.load(f)
    kernels = [k for k in rec if not k.startswith("_")]
    assert kernels
    kind_of = {"near_tma_kernel": ("near", 1), "near_kernel": ("near", 0),
               "coupling_a_staged_kernel": ("coupling", 0), "coupling_a_umma_kernel": ("coupling", 4),
               "coupling_b_tma_kernel": ("coupling_b", 2), "coupling_b_kernel": ("coupling_b", 0)}
    for name in kernels:
        assert rec[name]["bytes_per_launch"] > 0
        kind, var = kind_of[name]
        got = bench.measured_traffic(kind, {"kernel_variants": var})
        if rec[name]["source_sha256"] == bench.kernel_source_hash(name):
            assert got == rec[name]["bytes_per_launch"], name
        else:
            assert got is None, name


def test_workload_is_the_3d_matern_problem(bench):
    cfg = bench.workload_config()
    assert cfg["n"] == 65536 and cfg["d"] == 3 and cfg["kernel"] == "matern32" and cfg["m"] == 16
    assert cfg["workload"] == "n65536_d3_matern32_h2_fp32_m16"
