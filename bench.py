"""Throughput of the online stage (instantiate + H^2 matvec) on the GB300.

Workload (the FP32 GPU configuration of the parametric H^2 matrix): n = 65536
points uniform in [0,1]^3 (seed 1002), Matern nu = 3/2 with l in [0.05, 0.5],
Chebyshev degree 20 in l, p_s = 8, uniform tree of depth 3 (mean leaf 128),
eta = sqrt(3), TT tolerance 1e-5, far-field rank cap 64, 16 right-hand sides
~N(0, 1) (seed 2002), one theta per step drawn from U(B_theta) (seed 3002).

A step is one ph_instantiate(theta) + one ph_matvec(X) through the C ABI.
Metric: (theta * RHS)/s = steps * m / time, summed over ranks (each rank owns
its own replica and its own thetas: theta-sharded, no collective on the data
path).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2511_03109_gb300 import inputs, sharding  # noqa: E402

WL = inputs.LARGE_3D_MATERN_H2
METRIC = "online instantiate+H-MVM (theta*RHS)/s and % HBM roofline at rel.err vs FP64 oracle"
UNIT = "(theta*RHS)/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
ORACLE_SAMPLE_LEAVES = 2


def workload_config():
    return {
        "workload": WL.name, "n": WL.n, "d": WL.d, "kernel": WL.kernel,
        "theta_box": [WL.theta_lo[0], WL.theta_hi[0]], "degree": WL.degree[0], "p_s": WL.p_s,
        "l_max": WL.l_max, "eta": WL.eta, "tol": WL.tol, "rank_cap": WL.rank_cap,
        "format": WL.fmt, "m": WL.m, "thetas": "one per step, U(B_theta), seed %d" % WL.theta_seed,
        "l2": "no flush: the near-field cores streamed every step (> 4 GB) exceed the 129 MB L2",
        "parallelism": "theta-sharded replicas, one process per GPU",
    }


KERNEL_OF_KIND = {"near": "near_kernel", "coupling": "coupling_a_staged_kernel", "coupling_b": "coupling_b_kernel",
                  "combine": "combine_kernel", "upsweep_leaf": "upsweep_leaf_kernel"}


def kernel_source_hash(name):
    """sha256 (16 hex digits) of a kernel's template definition in csrc/online.cu."""
    import hashlib
    import re
    src = open(os.path.join(ROOT, "paper_2511_03109_gb300", "csrc", "online.cu")).read()
    m = re.search(r"__global__[^\n]*\n?[^\n]*\b" + re.escape(name) + r"\(", src)
    if not m:
        return None
    line0 = src.rfind("\n", 0, m.start()) + 1
    tmpl = src.rfind("template", 0, m.start())
    # the template line directly above the definition, else the definition itself
    start = tmpl if tmpl >= 0 and src.count("\n", tmpl, line0) <= 1 and "}" not in src[tmpl:line0] else line0
    end = src.index("\n}\n", m.end()) + 3
    return hashlib.sha256(src[start:end].encode()).hexdigest()[:16]


def kernel_of(kind, info):
    """The kernel behind a profiling kind, from the variants the last call reported."""
    var = info.get("kernel_variants", 0)
    if kind == "coupling" and var & 4:
        return "coupling_a_umma_kernel"
    if kind == "near" and var & 1:
        return "near_tma_kernel"
    if kind == "coupling_b" and var & 2:
        return "coupling_b_tma_kernel"
    return KERNEL_OF_KIND.get(kind, kind)


def measured_traffic(kind, info):
    """ncu DRAM bytes per launch of the kernel, or None if it changed since the capture."""
    name = kernel_of(kind, info)
    try:
        with open(os.path.join(ROOT, "profiles", "kernel_traffic.json")) as f:
            rec = json.load(f).get(name)
    except Exception:
        return None
    if not rec or rec.get("source_sha256") != kernel_source_hash(name):
        return None
    return rec["bytes_per_launch"]


def alu_peak_tflops(peaks, sms):
    """FP32 FMA peak derived from unit counts: SMs x 128 FP32 lanes x 2 flops x max SM clock."""
    return sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) / 1e6


def step_binding(step_bytes, step_flops, step_ms, peaks, sms):
    """max(B_alg / BW, F / P_simt) / T for one step, with the term that binds: the step's
    algorithmic bytes against the measured copy bandwidth, its flops against the FP32 FMA
    peak derived from the device's SM count (alu_peak_tflops)."""
    t = step_ms / 1e3
    hbm = step_bytes / peaks["hbm_gbs"] / 1e9
    alu = step_flops / (alu_peak_tflops(peaks, sms) * 1e12)
    return {"term": "hbm" if hbm >= alu else "alu", "fraction": max(hbm, alu) / t,
            "hbm_seconds": hbm, "alu_seconds": alu}


def tensor_roofline(flops, ms, peaks):
    """Roofline of a 3xTF32 tensor-core contraction.  `achieved` counts the algorithmic FP32
    flops; the peak is the dense TF32 rate (measured bf16 x the nominal TF32 / bf16 ratio
    1.1 / 2.25) divided by 3, since every FP32 product is issued as three TF32 MMAs."""
    tf32 = peaks["bf16_tflops"] * 1.1 / 2.25
    ach = flops / (ms / 1e3) / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": tf32 / 3.0, "unit": "TFLOP/s", "per_launch_flops": flops,
            "peak_source": "derived", "tf32_issue_frac": 3.0 * ach / tf32,
            "peak_note": "3xTF32 ceiling: dense TF32 (measured bf16 x nominal 1.1/2.25) / 3 MMAs per FP32 product"}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------- oracle (CPU) baseline
ORACLE_RUNS = 5


def oracle_model(P, n_leaves=ORACLE_SAMPLE_LEAVES, seed=7):
    """The oracle's model of the workload with the offline work of a bounded sample done: the
    near blocks of `n_leaves` target leaves (a corner leaf and random others) and the far
    blocks of their ancestors, compressed in a spawn-started pool (offline, not timed)."""
    from oracle import pmatrix

    M = pmatrix.ParametricMatrix(P, WL.kernel, WL.theta_lo, WL.theta_hi, WL.degree, WL.p_s,
                                 WL.l_max, WL.eta, WL.tol, rank_cap=WL.rank_cap, fmt=WL.fmt)
    rng = np.random.default_rng(seed)
    rest = [int(i) for i in rng.choice(np.arange(1, len(M.leaves)), size=max(0, n_leaves - 1), replace=False)]
    targets = [M.leaves[i] for i in sorted([0] + rest)]
    with _oracle_pool() as pool:
        M.offline(targets, pool=pool)
    return M, targets


def oracle_step_seconds(M, targets, X, theta):
    """Seconds of one online step (instantiate + H^2 matvec) of the FP64 oracle for the WHOLE
    matrix, composed from timed samples: every part of the oracle's step (near-block
    instantiation and product, far-block core instantiation and coupling, leaf sweeps, transfers)
    is timed on the sample's units and scaled by that part's own count of units in the full
    matrix (near blocks by stored entries, far blocks, leaves and transfer nodes by number), so
    no unit is counted more often than the full step holds it.  Returns (seconds, parts)."""
    from oracle import pmatrix

    near, far = M.blocks_for(targets)
    anc = {}
    for c in targets:
        a = c
        while a.parent is not None:
            anc[a.id] = a
            a = a.parent
    tnodes = list(anc.values())
    m = X.shape[1]
    pd = M.p_s ** M.d
    rng = np.random.default_rng(5)
    xh = {c.id: rng.standard_normal((pd, m)) for c in M.nodes}
    parts = {}
    t = time.perf_counter
    vs = M.parametric_vectors(np.atleast_1d(theta))
    t0 = t()
    D = {id(b): M.near_instance(b, vs) for b in near}
    parts["near_instantiate"] = t() - t0
    t0 = t()
    H = {id(b): pmatrix.H_matrix(b.cores, M.d, vs) for b in far}
    parts["far_instantiate"] = t() - t0
    inst = {"H": H}
    t0 = t()
    for c in targets:
        M.basis(c).T @ X[c.idx]
    parts["leaf_up"] = t() - t0
    t0 = t()
    for c in tnodes:
        M.transfer(c).T @ xh[c.id]
    parts["transfer_up"] = t() - t0
    t0 = t()
    for b in far:
        M.coupling(b, inst) @ xh[b.t.id]
    parts["coupling"] = t() - t0
    t0 = t()
    for b in near:
        D[id(b)] @ X[b.t.idx]
    parts["near_product"] = t() - t0
    t0 = t()
    for c in tnodes:
        M.transfer(c) @ xh[c.parent.id]
    parts["transfer_down"] = t() - t0
    t0 = t()
    for c in targets:
        M.basis(c) @ xh[c.id]
    parts["leaf_down"] = t() - t0
    ent = lambda bs: sum(b.s.n * b.t.n for b in bs)
    scale = {"near_instantiate": ent(M.near) / ent(near), "near_product": ent(M.near) / ent(near),
             "far_instantiate": len(M.far) / max(1, len(far)), "coupling": len(M.far) / max(1, len(far)),
             "leaf_up": len(M.leaves) / len(targets), "leaf_down": len(M.leaves) / len(targets),
             "transfer_up": (len(M.nodes) - 1) / max(1, len(tnodes)),
             "transfer_down": (len(M.nodes) - 1) / max(1, len(tnodes))}
    total = sum(parts[k] * scale[k] for k in parts)
    return total, {k: parts[k] * scale[k] for k in parts}


def oracle_baseline_runs(M, targets, X, thetas, runs=ORACLE_RUNS):
    """Warm-up (builds the oracle's cached bases, offline work), then `runs` timed steps:
    (median seconds, all per-step seconds, median parts, sample wall seconds per step)."""
    oracle_step_seconds(M, targets, X, thetas[0])
    totals, parts, walls = [], [], []
    for k in range(runs):
        w0 = time.perf_counter()
        tot, pr = oracle_step_seconds(M, targets, X, thetas[(k + 1) % len(thetas)])
        walls.append(time.perf_counter() - w0)
        totals.append(tot)
        parts.append(pr)
    med = float(statistics.median(totals))
    i = totals.index(sorted(totals)[len(totals) // 2])
    return med, totals, parts[i], float(statistics.median(walls))


def _single_thread_child(args):
    M, targets, X, thetas = args
    return oracle_baseline_runs(M, targets, X, thetas)


def oracle_baseline(M, targets, X, thetas):
    """The oracle's step time on this host with BLAS on one thread (a spawned process started
    with OMP/OPENBLAS/MKL_NUM_THREADS=1) and with NumPy's default threads (all cores)."""
    import multiprocessing as mp
    nproc = os.cpu_count() or 1
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(1) as pool:
            single = pool.apply(_single_thread_child, ((M, targets, X, list(thetas)),))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    multi = oracle_baseline_runs(M, targets, X, thetas)
    return {"single": single, "all": multi, "nproc": nproc}


def oracle_rows(M, targets, X, theta, deriv=None):
    """The oracle's Y (or dK_hat/dtheta X) on the rows of the sampled target leaves (untimed)."""
    rows = np.sort(np.concatenate([c.idx for c in targets]))
    Y = M.matvec(M.instantiate(theta, targets, deriv=deriv), X, targets)
    return rows, Y[rows]


def _oracle_pool():
    """Spawn-started pool for the oracle's per-block TT-SVDs, one single-threaded BLAS per worker."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        return mp.get_context("spawn").Pool(max(1, os.cpu_count() or 2))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def log(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


# ------------------------------------------------------------------------ clock sampling
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")

    def _lines(self):
        try:
            with open(self.path) as f:
                return f.read().splitlines()
        except OSError:
            return []

    def start(self):
        """Starts sampling every 50 ms and returns once the first sample is in, so that the
        samples counted (from `mark()` to `stop()`) fall inside the timed region."""
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        self.first = 0
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5 and not self._lines() and self.proc.poll() is None:
            time.sleep(0.01)

    def mark(self):
        self.first = len(self._lines())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        lines = self._lines()[self.first:]
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        if True:
            for line in lines:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# -------------------------------------------------------------------------------- our arm
def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_2511_03109_gb300 import ph

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    P = WL.points()
    Xh = WL.rhs()
    m, n = WL.m, WL.n
    opts = ph.make_opts(WL.d, WL.theta_lo, WL.theta_hi, WL.degree, WL.p_s, WL.l_max, WL.eta, WL.tol,
                        rank_cap=WL.rank_cap, fmt=WL.fmt, prec=WL.precision, device=local_rank)
    if args.load:
        A = ph.ParametricMatrix.load(args.load, device=local_rank)
    else:
        log(f"offline build n={n} on cuda:{local_rank}")
        A = ph.ParametricMatrix(P, WL.kernel, opts)
        if args.save:
            A.save(args.save)
    if args.tensor_cores is not None:
        A.set_tensor_cores(args.tensor_cores == 1)
    info = A.info()
    log(f"offline done in {info['offline_seconds']:.1f} s")
    total_steps = args.warmup + args.steps
    thetas_all = inputs.uniform_thetas(WL.theta_lo, WL.theta_hi, max(30, world * total_steps), WL.theta_seed)
    thetas = sharding.shard(thetas_all, rank, world)[:total_steps]
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    X = torch.tensor(Xh.T, dtype=torch.float32, device=dev).contiguous()  # column-major n x m
    Y = torch.empty((m, n), dtype=torch.float32, device=dev)

    def step(th):
        A.instantiate(th, sp)
        A.matvec_ptr(X.data_ptr(), n, m, Y.data_ptr(), n, sp)

    for k in range(args.warmup):
        step(thetas[k])
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    A.profile(True)
    A.profile_read()  # reset counters
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    sampler.mark()
    ev0.record(stream)
    for k in range(args.steps):
        step(thetas[args.warmup + k])
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    prof = A.profile_read()
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    A.profile(False)
    ms = sharding.max_over_ranks(ms, dist)

    # end to end through the host entry point: pinned host X in, Y out every step
    Xp = torch.tensor(Xh.T, dtype=torch.float32).contiguous().pin_memory()
    Yp = torch.empty((m, n), dtype=torch.float32).pin_memory()

    def step_host(th):
        A.instantiate(th, sp)
        A.matvec_host_ptr(Xp.data_ptr(), n, m, Yp.data_ptr(), n, sp)

    for k in range(min(args.warmup, 3)):
        step_host(thetas[k])
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        step_host(thetas[args.warmup + k])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = sharding.max_over_ranks(e2e_s, dist)

    # theta-derivative products dK_hat/dtheta X (ph_instantiate_derivative + ph_matvec), device
    # inputs as in the timed region
    def step_d(th):
        A.instantiate_derivative(th, 0, sp)
        A.matvec_ptr(X.data_ptr(), n, m, Y.data_ptr(), n, sp)

    nd = min(args.steps, 50)
    for k in range(min(args.warmup, 3)):
        step_d(thetas[k])
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(nd):
        step_d(thetas[args.warmup + k])
    ev1.record(stream)
    torch.cuda.synchronize()
    d_ms = sharding.max_over_ranks(ev0.elapsed_time(ev1), dist)

    # many theta, one X (ph_matvec_batched): BATCH_THETAS values per call, the first being the
    # oracle's theta below; a failure here is reported in the line instead of ending the bench
    b_local, b_err, Ybs = -1.0, None, None
    tb = [thetas[args.warmup]] + list(inputs.uniform_thetas(WL.theta_lo, WL.theta_hi, BATCH_THETAS - 1,
                                                             WL.theta_seed + 17))
    try:
        Yb = torch.empty((len(tb), m, n), dtype=torch.float32, device=f"cuda:{local_rank}")
        A.matvec_batched_ptr(tb, X.data_ptr(), n, m, Yb.data_ptr(), n, m * n, -1, sp)  # warm-up
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(BATCH_CALLS):
            A.matvec_batched_ptr(tb, X.data_ptr(), n, m, Yb.data_ptr(), n, m * n, -1, sp)
        ev1.record(stream)
        torch.cuda.synchronize()
        b_local = ev0.elapsed_time(ev1) / BATCH_CALLS
        Ybs = [(t, Yb[t].double().cpu().numpy().T) for t in (0, len(tb) // 2, len(tb) - 1)]
        del Yb
    except Exception as exc:  # noqa: BLE001 - reported in the line, not hidden
        b_err = f"{type(exc).__name__}: {exc}"
    # every rank takes part in both reductions, whatever happened above
    b_ms = sharding.max_over_ranks(b_local, dist)
    b_fail = sharding.max_over_ranks(1.0 if b_err else 0.0, dist)
    if b_fail > 0 or b_ms <= 0:
        batched = {"error": b_err or "failed on another rank"}
        Ybs = None
    else:
        batched = {"what": f"ph_matvec_batched: {len(tb)} theta x {m} RHS per call, one X",
                   "value": world * len(tb) * m / (b_ms / 1e3), "unit": UNIT, "ms_per_call": b_ms,
                   "calls": BATCH_CALLS}

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        A.close()
        return

    value = world * args.steps * m / (ms / 1e3)
    peaks, peak_kind = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # roofline pass: the same steps with the far and near paths serialised on one stream, so that
    # each kernel's CUDA-event time is its own (in the timed region they overlap)
    A.set_overlap(False)
    A.profile(True)
    for k in range(2):
        step(thetas[k])
    A.profile_read()
    nprof = min(args.steps, 10)
    for k in range(nprof):
        step(thetas[args.warmup + k % args.steps])
    torch.cuda.synchronize()
    alone = {k: v for k, v in A.profile_read().items() if v[1] > 0}
    A.profile(False)
    A.set_overlap(True)
    info = A.info()  # now with the kernel variants of the last call
    dom = max(alone, key=lambda k: alone[k][0])
    dom_ms, dom_launches = alone[dom]
    avg_ms = dom_ms / dom_launches
    sc = 4
    if dom == "near":
        alg = info["near_bytes"] + 2.0 * n * m * sc + info["near_rank_sum"] * sc
        roof = {"bound": "hbm", "achieved": alg / (avg_ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "per_launch_bytes": alg}
    else:
        # FP32 CUDA-core flops of the kernel (flop counts of the built structure, per launch)
        per_rhs = {"coupling": info["coupling_a_flops_per_rhs"], "coupling_b": info["coupling_b_flops_per_rhs"]}
        fl = per_rhs.get(dom, info["flops_per_rhs"] - 2.0 * info["near_entries"]) * m
        if kernel_of(dom, info) == "coupling_a_umma_kernel":
            roof = tensor_roofline(fl, avg_ms, peaks)
        else:
            alu_peak = alu_peak_tflops(peaks, sms)
            roof = {"bound": "alu", "achieved": fl / (avg_ms / 1e3) / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                    "per_launch_flops": fl, "peak_source": "derived",
                    "peak_note": f"FP32 FMA lanes: {sms} SMs (device count) x 128 x 2 flops x max SM clock"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = kernel_of(dom, info)
    roof.setdefault("peak_source", peak_kind)
    roof["traffic"] = measured_traffic(dom, info)
    roof["timing"] = "CUDA events around each launch, far and near paths serialised (roofline pass)"
    # the three large kernels against their own bounds, same pass
    others = {}
    alu_peak = alu_peak_tflops(peaks, sms)
    if "near" in alone:
        t = alone["near"][0] / alone["near"][1] / 1e3
        b = info["near_bytes"] + 2.0 * n * m * sc + info["near_rank_sum"] * sc
        others["near"] = {"kernel": kernel_of("near", info), "bound": "hbm", "ms": t * 1e3,
                          "achieved": b / t / 1e9, "unit": "GB/s", "frac": b / t / 1e9 / peaks["hbm_gbs"],
                          "traffic": measured_traffic("near", info)}
    for kind, key in (("coupling", "coupling_a_flops_per_rhs"), ("coupling_b", "coupling_b_flops_per_rhs")):
        if kind in alone and info[key] > 0:
            t = alone[kind][0] / alone[kind][1] / 1e3
            f = info[key] * m
            if kernel_of(kind, info) == "coupling_a_umma_kernel":
                rt = tensor_roofline(f, t * 1e3, peaks)
                others[kind] = {"kernel": kernel_of(kind, info), "bound": "tensor", "ms": t * 1e3,
                                "achieved": rt["achieved"], "unit": "TFLOP/s", "frac": rt["achieved"] / rt["peak"],
                                "tf32_issue_frac": rt["tf32_issue_frac"], "traffic": measured_traffic(kind, info)}
            else:
                others[kind] = {"kernel": kernel_of(kind, info), "bound": "alu", "ms": t * 1e3,
                                "achieved": f / t / 1e12, "unit": "TFLOP/s", "frac": f / t / 1e12 / alu_peak,
                                "traffic": measured_traffic(kind, info)}
    gpu_launches = int(sum(v[1] for v in prof.values()))
    # whole-step bytes over the step time, for context
    step_bytes = info["alg_bytes_per_call"] + 2.0 * n * m * sc
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(), "roofline": roof, "rooflines_by_kernel": others,
        "step_hbm_fraction": step_bytes / (ms / args.steps / 1e3) / 1e9 / peaks["hbm_gbs"],
        "step_binding": step_binding(step_bytes, info["flops_per_rhs"] * m, ms / args.steps, peaks, sms),
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in kinds.items()},
        "kernels_ms_alone": {k: v[0] / v[1] for k, v in alone.items()},
        "gpu_launches": gpu_launches, "clocks": clocks,
        "e2e": {"value": world * args.steps * m / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": n * m * sc + 8 * WL.d, "d2h_bytes_per_step": n * m * sc},
        "derivative": {"what": "dK_hat/dtheta X: ph_instantiate_derivative + ph_matvec, one theta per step",
                       "value": world * nd * m / (d_ms / 1e3), "unit": UNIT, "steps": nd,
                       "ms_per_step": d_ms / nd},
        "batched": batched,
        "offline_seconds": info["offline_seconds"],
        "structure": {k: info[k] for k in ("n_near", "n_far", "n_far_keys", "near_entries", "near_rank_max",
                                           "far_rank_max", "far_rank_mean", "near_bytes", "far_bytes")},
    }
    if not args.no_cpu_baseline:
        th0 = thetas[args.warmup]
        A.instantiate(th0, sp)
        A.matvec_ptr(X.data_ptr(), n, m, Y.data_ptr(), n, sp)
        torch.cuda.synchronize()
        Ygpu = Y.double().cpu().numpy().T
        A.instantiate_derivative(th0, 0, sp)
        A.matvec_ptr(X.data_ptr(), n, m, Y.data_ptr(), n, sp)
        torch.cuda.synchronize()
        Ygpu_d = Y.double().cpu().numpy().T
        log("oracle sample: offline work of the sample")
        M, targets = oracle_model(P)
        rows, Yo = oracle_rows(M, targets, Xh, th0)
        _, Yod = oracle_rows(M, targets, Xh, th0, deriv=0)
        rel = lambda ref, got: float((np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)).max())
        out["rel_err_vs_oracle"] = rel(Yo, Ygpu[rows])
        out["derivative"]["rel_err_vs_oracle"] = rel(Yod, Ygpu_d[rows])
        out["oracle_rows"] = {"leaves": [int(c.id) for c in targets], "rows": int(len(rows))}
        if Ybs is not None:
            errs = []
            for t, Yt in Ybs:
                _, Yot = oracle_rows(M, targets, Xh, tb[t])
                errs.append(rel(Yot, Yt[rows]))
            out["batched"]["rel_err_vs_oracle"] = max(errs)
            out["batched"]["thetas_checked"] = [int(t) for t, _ in Ybs]
        log("oracle step timing (single thread and all cores)")
        base = oracle_baseline(M, targets, Xh, thetas[args.warmup:args.warmup + ORACLE_RUNS + 1])
        s1, s_all, parts, wall = base["single"][0], base["all"][0], base["all"][2], base["all"][3]
        sample = (f"one full online step (instantiate + H^2 matvec, {m} RHS, every block) composed from timed "
                  f"parts of {len(targets)} of {len(M.leaves)} target leaves (their near blocks, the far blocks "
                  f"of their ancestors, their sweeps), each part scaled by its own unit count in the full matrix; "
                  f"median of {ORACLE_RUNS} warm runs")
        out["cpu_baseline"] = {"value": m / s_all, "unit": UNIT, "cores": base["nproc"], "kind": "oracle",
                               "sample": sample, "seconds_per_step": s_all,
                               "single_thread": {"value": m / s1, "cores": 1, "seconds_per_step": s1},
                               "parts_seconds": parts, "sample_wall_seconds_per_step": wall}
        from oracle import kernels
        t_dense = time.perf_counter()
        exact = kernels.dense_apply(WL.kernel, P, th0, Xh, rows=rows)
        t_dense = time.perf_counter() - t_dense
        frac = len(rows) / n
        out["cpu_dense"] = {"value": m / (t_dense / frac), "unit": UNIT, "cores": base["nproc"],
                            "kind": "brute-force K(theta) X (NumPy FP64), the product the method avoids",
                            "sample": f"the same {len(rows)} rows; time scaled by n / rows (every row costs the same)"}
        out["rel_err_vs_exact"] = rel(exact, Ygpu[rows])
    print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    A.close()


# -------------------------------------------------------------------- reference (oracle) arm
REF_TIME_LIMIT = 120.0
BATCH_THETAS = 256
BATCH_CALLS = 3


def run_reference(args, rank, world):
    """The FP64 oracle on this host's cores: each step is one full online step composed from
    timed parts of a bounded sample (oracle_step_seconds), all cores (NumPy's default threads)."""
    if rank != 0:
        return
    P = WL.points()
    Xh = WL.rhs()
    m = WL.m
    thetas = inputs.uniform_thetas(WL.theta_lo, WL.theta_hi, max(30, args.warmup + args.steps), WL.theta_seed)
    M, targets = oracle_model(P)
    for k in range(min(max(args.warmup, 1), 3)):
        oracle_step_seconds(M, targets, Xh, thetas[k])
    # every composed step takes about a second of host work: stop after REF_TIME_LIMIT s so that
    # any --steps finishes within a few minutes, and report the steps actually timed
    t0 = time.perf_counter()
    secs = []
    for k in range(args.steps):
        secs.append(oracle_step_seconds(M, targets, Xh, thetas[(args.warmup + k) % len(thetas)])[0])
        if time.perf_counter() - t0 > REF_TIME_LIMIT:
            break
    wall = (time.perf_counter() - t0) / len(secs)
    step_s = float(statistics.median(secs))
    value = m / step_s
    cores = os.cpu_count() or 1
    sample = (f"one full online step (instantiate + H^2 matvec, {m} RHS, every block) composed from timed parts "
              f"of {len(targets)} of {len(M.leaves)} target leaves, each part scaled by its own unit count in the "
              f"full matrix; median over the steps timed")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "steps_timed": len(secs), "warmup": args.warmup, "ms_per_step": step_s * 1e3,
           "sample_wall_ms_per_step": wall * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------- the differentiated and learned forms


def _make(wl, ph):
    opts = ph.make_opts(wl.d, wl.theta_lo, wl.theta_hi, wl.degree, wl.p_s, wl.l_max, wl.eta, wl.tol,
                        rank_cap=wl.rank_cap, fmt=wl.fmt, prec=wl.precision,
                        near_degree=list(wl.near_degree) if wl.near_degree else None)
    return ph.ParametricMatrix(wl.points(), wl.kernel, opts)


def _timed(fn, count, stream):
    import torch

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(count):
        fn(k)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / count


def run_differentiation(args):
    """y = K_hat(theta) x, its adjoint K_hat^T ybar (d/dx) and the d_theta derivative products
    dK_hat/dtheta_i x (d/dtheta through the derivatives of the Lagrange weights), each timed against
    the forward product; checked by central differences (step 1e-4), the adjoint identity and the
    oracle's exact dK/dtheta x on sampled rows."""
    import torch

    from paper_2511_03109_gb300 import ph

    wl = inputs.DIFF_2D_ANISO
    log(f"offline build {wl.name}")
    A = _make(wl, ph)
    info = A.info()
    n, m, dt = wl.n, wl.m, wl.d
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    X = torch.tensor(wl.rhs().T, dtype=torch.float32, device="cuda").contiguous()
    Y = torch.empty_like(X)
    Z = torch.empty_like(X)
    K, W = args.steps, args.warmup
    th = wl.thetas(K + W)

    def fwd(k):
        A.instantiate(th[k % len(th)], sp)
        A.matvec_ptr(X.data_ptr(), n, m, Y.data_ptr(), n, sp)

    def adj(k):
        A.instantiate(th[k % len(th)], sp)
        A.matvec_transpose_ptr(X.data_ptr(), n, m, Z.data_ptr(), n, sp)

    def der(k):
        for i in range(dt):
            A.instantiate_derivative(th[k % len(th)], i, sp)
            A.matvec_ptr(X.data_ptr(), n, m, Z.data_ptr(), n, sp)

    def grad(k):  # one loss gradient: forward, adjoint, every theta derivative
        fwd(k)
        adj(k)
        der(k)

    res = {}
    for name, fn in (("forward", fwd), ("adjoint", adj), ("dtheta_products", der), ("gradient_step", grad)):
        for k in range(W):
            fn(k)
        ms = _timed(fn, K, stream)
        res[name] = {"ms_per_step": ms, "value": m / (ms / 1e3), "unit": UNIT}
    for name in ("adjoint", "dtheta_products", "gradient_step"):
        res[name]["vs_forward"] = res[name]["ms_per_step"] / res["forward"]["ms_per_step"]
    # checks at one theta
    t0 = np.asarray(th[0], float)
    h = 1e-4
    A.instantiate(t0, sp)
    A.matvec_ptr(X.data_ptr(), n, m, Y.data_ptr(), n, sp)
    A.matvec_transpose_ptr(X.data_ptr(), n, m, Z.data_ptr(), n, sp)
    torch.cuda.synchronize()
    Xh = X.double().cpu().numpy()
    ident = abs(float(np.sum(Xh * Y.double().cpu().numpy()) - np.sum(Z.double().cpu().numpy() * Xh)))
    ident /= float(np.linalg.norm(Xh) * np.linalg.norm(Y.double().cpu().numpy()))
    fd = []
    Yp, Ym = torch.empty_like(X), torch.empty_like(X)
    for i in range(dt):
        A.instantiate_derivative(t0, i, sp)
        A.matvec_ptr(X.data_ptr(), n, m, Z.data_ptr(), n, sp)
        tp, tm = t0.copy(), t0.copy()
        tp[i] += h
        tm[i] -= h
        A.instantiate(tp, sp)
        A.matvec_ptr(X.data_ptr(), n, m, Yp.data_ptr(), n, sp)
        A.instantiate(tm, sp)
        A.matvec_ptr(X.data_ptr(), n, m, Ym.data_ptr(), n, sp)
        torch.cuda.synchronize()
        num = (Yp.double() - Ym.double()) / (2 * h)
        fd.append(float(((num - Z.double()).norm() / Z.double().norm()).item()))
    out = {"metric": "differentiated online stage (theta*RHS)/s", "workload": wl.name, "n": n, "d": wl.d,
           "dtheta": dt, "degree": list(wl.degree), "m": m, "dtype": "f32", "data": "synthetic", "steps": K,
           "warmup": W, "results": res, "adjoint_identity_rel": ident,
           "fd_check_rel_err": {"step": h, "per_dim": fd,
                                "note": "central differences in FP32: rounding of the two products over 2h"},
           "structure": {k: info[k] for k in ("n_near", "n_far", "n_far_keys", "near_bytes", "far_rank_max")},
           "offline_seconds": info["offline_seconds"]}
    if not args.no_cpu_baseline:
        from oracle import pmatrix
        M = pmatrix.ParametricMatrix(wl.points(), wl.kernel, wl.theta_lo, wl.theta_hi, wl.degree, wl.p_s, wl.l_max,
                                     wl.eta, wl.tol, rank_cap=wl.rank_cap, fmt=wl.fmt)
        targets = M.leaves[:: max(1, len(M.leaves) // 2)][:2]
        log("oracle: sampled rows of the forward and derivative products")
        M.offline(targets)
        rows = np.sort(np.concatenate([c.idx for c in targets]))
        Xo = wl.rhs()
        errs = {}
        for name, deriv in (("forward", None),) + tuple((f"dtheta_{i}", i) for i in range(dt)):
            ref = M.matvec(M.instantiate(t0, targets, deriv=deriv), Xo, targets)[rows]
            if deriv is None:
                A.instantiate(t0, sp)
            else:
                A.instantiate_derivative(t0, deriv, sp)
            A.matvec_ptr(X.data_ptr(), n, m, Z.data_ptr(), n, sp)
            torch.cuda.synchronize()
            got = Z.double().cpu().numpy().T[rows]
            errs[name] = float((np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)).max())
        out["rel_err_vs_oracle"] = errs
        out["oracle_rows"] = int(len(rows))
    print(json.dumps(out), flush=True)
    A.close()


def run_surrogate(args):
    """The learned far-field cores against the degree-8 tensor-grid polynomial on the same
    handle: training on the GPU, then 64 theta x 16 RHS through each path; accuracy of each path's
    cores (against the exact projected cores) and of each product (against the product with the
    projected cores, and against the exact K(theta) X on sampled rows)."""
    import torch

    from oracle import kernels
    from paper_2511_03109_gb300 import ph

    wl = inputs.SURROGATE_3D_ANISO
    log(f"offline build {wl.name}")
    A = _make(wl, ph)
    info = A.info()
    n, m = wl.n, wl.m
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    n_train = args.sur_train
    tt = inputs.uniform_thetas(wl.theta_lo, wl.theta_hi, n_train, wl.theta_seed)
    tv = inputs.uniform_thetas(wl.theta_lo, wl.theta_hi, 64, wl.theta_seed + 1)
    log(f"training on {n_train} thetas")
    rep = A.surrogate_train(tt, tv, hidden=256, steps=args.sur_steps, batch=256, lr=1e-3, seed=7, stream=sp)
    X = torch.tensor(wl.rhs().T, dtype=torch.float32, device="cuda").contiguous()
    Y = torch.empty_like(X)
    th64 = inputs.uniform_thetas(wl.theta_lo, wl.theta_hi, 64, wl.theta_seed + 2)

    def step(k):
        A.instantiate(th64[k % 64], sp)
        A.matvec_ptr(X.data_ptr(), n, m, Y.data_ptr(), n, sp)

    def inst(k):
        A.instantiate(th64[k % 64], sp)

    paths = {}
    for use in (False, True):
        if use and not rep["accepted"]:
            continue
        A.surrogate_use(use)
        for k in range(3):
            step(k)
        ms = _timed(step, 64, stream)
        ms_i = _timed(inst, 64, stream)
        paths["network" if use else "polynomial"] = {"ms_per_theta": ms, "instantiate_ms": ms_i,
                                                     "value": m / (ms / 1e3), "unit": UNIT}
    # accuracy on four thetas: products with each path's cores against the product with the exact
    # projected cores (the far-field error) and against the exact K(theta) X on 200 sampled rows
    P = wl.points()
    Xh = wl.rhs()
    rows = inputs.sample_rows(n, 200, wl.theta_seed + 3)
    cores = torch.empty((1, info["far_core_elems"]), dtype=torch.float32, device="cuda")
    acc = {"far_field_err": {}, "total_err_vs_exact": {}}
    for th in tv[:4]:
        A.far_project_ptr([th], cores.data_ptr(), sp)
        A.instantiate_cores_ptr(th, cores.data_ptr(), sp)
        A.matvec_ptr(X.data_ptr(), n, m, Y.data_ptr(), n, sp)
        torch.cuda.synchronize()
        ystar = Y.double().cpu().numpy().T
        exact = kernels.dense_apply(wl.kernel, P, th, Xh, rows=rows)
        e = float((np.linalg.norm(ystar[rows] - exact, axis=0) / np.linalg.norm(exact, axis=0)).max())
        acc["total_err_vs_exact"].setdefault("projected_cores", []).append(e)
        for name, use in (("polynomial", False), ("network", True)):
            if use and not rep["accepted"]:
                continue
            A.surrogate_use(use)
            A.instantiate(th, sp)
            A.matvec_ptr(X.data_ptr(), n, m, Y.data_ptr(), n, sp)
            torch.cuda.synchronize()
            y = Y.double().cpu().numpy().T
            acc["far_field_err"].setdefault(name, []).append(
                float((np.linalg.norm(y - ystar, axis=0) / np.linalg.norm(ystar, axis=0)).max()))
            acc["total_err_vs_exact"].setdefault(name, []).append(
                float((np.linalg.norm(y[rows] - exact, axis=0) / np.linalg.norm(exact, axis=0)).max()))
    A.surrogate_use(False)
    out = {"metric": "learned far-field cores vs tensor-grid polynomial (theta*RHS)/s", "workload": wl.name,
           "n": n, "d": wl.d, "dtheta": len(wl.theta_lo), "far_degree": list(wl.degree),
           "near_degree": list(wl.near_degree), "m": m, "thetas_timed": 64, "dtype": "f32", "data": "synthetic",
           "network": {"shape": f"{len(wl.theta_lo)} -> 256 -> 256 -> {rep['out_dim']}", "params": rep["params"],
                       "weights": "BF16 copies in the products, FP32 accumulation and master weights",
                       "train_thetas": n_train, "steps": args.sur_steps},
           "training": rep, "paths": paths, "accuracy_on_4_thetas": acc,
           "network_weight_bytes_bf16": 2 * rep["params"],
           "structure": {k: info[k] for k in ("n_near", "n_far", "n_far_keys", "near_bytes", "far_rank_max",
                                              "far_core_elems", "far_bytes")},
           "offline_seconds": info["offline_seconds"]}
    print(json.dumps(out), flush=True)
    A.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--save", default="", help="profiling only: write the built handle to this file")
    ap.add_argument("--load", default="", help="profiling only: load a handle written by --save")
    ap.add_argument("--tensor-cores", type=int, default=None, choices=[0, 1],
                    help="phase 1 of the coupling on the tensor cores (1) or CUDA cores (0); default: the library's")
    ap.add_argument("--n", type=int, default=0,
                    help="profiling only: a smaller point count of the same workload (not a bench line)")
    ap.add_argument("--workload", default="plain", choices=["plain", "differentiation", "surrogate"],
                    help="plain: the headline line; differentiation / surrogate: the differentiated and the "
                         "learned forms on their own workloads (one JSON line each, one GPU)")
    ap.add_argument("--sur-train", type=int, default=4096, help="surrogate: training thetas")
    ap.add_argument("--sur-steps", type=int, default=1500, help="surrogate: Adam steps")
    args = ap.parse_args()
    if args.workload == "differentiation":
        return run_differentiation(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.n:
        global WL
        import dataclasses
        WL = dataclasses.replace(WL, n=args.n, name=WL.name.replace(str(WL.n), str(args.n)))
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
