#!/usr/bin/env python3
"""Benchmark: hybrid-query QPS at Recall@10 >= 0.95 on one GB300.

Workload (default): SIFT1M-shaped synthetic object set -- N = 1,000,000 vectors,
d = 128, integer components 0..255 stored as f32 (1,000 centroids), m = 3
attributes with cardinalities 3/10/20 (Zipf s = 1), 10,000 queries, k = 10,
graph out-degree R = 32.  Weights: constant w_v = 1, w_l = 10,000 (the
paper's best constant ratio, Sec. 6.5), under which the exact fused top-k is
the hybrid ground truth of Sec. 6.1, so hybrid Recall@10 can reach 1.

Flow: build the composite index on the GPU (exact K = 64 candidates, landing
zone selection, reverse pass), compute the hybrid ground truth with the GPU
brute force in filter mode, sweep ef (and the S1 fraction h, and the scoring
copy) for the cheapest setting whose hybrid Recall@10 >= 0.95, then time K
steps of one search over the whole query batch.  One JSON line on stdout.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs the full query batch on its own replica (no
collective on the data path; weak scaling); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QPS at Recall@10 >= 0.95 (hybrid recall, Sec. 6.1) on 1 GB300"
VEC_NAMES = {0: "f32", 1: "bf16", 2: "fp8e4m3"}
CONST_W = (1.0, 10000.0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--nq", type=int, default=10_000)
    ap.add_argument("--d", type=int, default=128)
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--R", type=int, default=32)
    ap.add_argument("--target", type=float, default=0.95)
    ap.add_argument("--target2", type=float, default=0.98,
                    help="a second recall level at which the forms are also compared")
    ap.add_argument("--efs", default="10,12,16,20,22,23,24,32,40,48,64,80,96,128,160,200,256,320,400,500")
    ap.add_argument("--hs", default="1,2")
    ap.add_argument("--cpu-sample", type=int, default=40, help="queries in the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="--impl reference: about this many seconds of oracle work in all")
    ap.add_argument("--fixed", default=None, help="skip the sweep: ef,h,vec (e.g. 64,1,1)")
    ap.add_argument("--seed-mode", type=int, default=1,
                    help="seed set B: 0 random (the paper's), 1 attribute entry")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned early stop")
    ap.add_argument("--wpq", type=int, default=1, help="warps per query of the search (1, 2, 4)")
    ap.add_argument("--cells", type=int, default=0,
                    help="entry cells E for the learned entry point (0: the workload's default)")
    ap.add_argument("--entry-T", type=int, default=1, help="entry cells taken per query")
    ap.add_argument("--train-q", type=int, default=100_000,
                    help="training queries for the learned entry point")
    ap.add_argument("--knn-dtype", type=int, default=1,
                    help="candidate build: 0 exact f32 SIMT, 1 bf16 tensor cores (exact here)")
    ap.add_argument("--learned-efs", default="16,24,32,48,64")
    ap.add_argument("--taus", default="0.7,0.8,0.9,0.95")
    ap.add_argument("--c4-build", default="nsw", choices=["kgraph", "nsw"],
                    help="c4 workload: graph built from exact candidates or incrementally")
    ap.add_argument("--workload", default="c2",
                    choices=["c2", "c3", "c4", "c5", "strategies", "curves", "builds",
                             "attrdim", "wildcard"],
                    help="c2: the headline workload (default); c4: the heterogeneous batch "
                         "(1M x 96, 100k queries with mixed k and ef) through "
                         "nhq_search_batched; c5: the 10M x 96 set (f16-valued), 50k queries; "
                         "strategies: NHQ against post-filtering on a "
                         "plain L2 graph and exact pre-filtering, on the c2 workload; curves: "
                         "the weightings i-v of Sec. 6.5 on the c2 workload; builds: exact "
                         "candidates, NN-descent and the incremental build compared; "
                         "attrdim: m = 3, 6 and 9 attributes on c2-shaped vectors; "
                         "wildcard: queries leaving one attribute open; each "
                         "prints one JSON line of its own")
    return ap.parse_args()


def workload_name(a):
    return (f"c2-shaped: N={a.n:,} d={a.d} int-valued f32 (1,000 centroids), m=3 attrs 3/10/20 "
            f"Zipf s=1, {a.nq:,} queries, k={a.k}, R={a.R}, weights w_v=1 w_l=10000")


def synth_c2_queries(a, nq, stream):
    """nq training queries of the c2-shaped workload from an independent query stream."""
    import copy

    b = copy.copy(a)
    b.nq = nq
    return make_workload(b, query_stream=stream)


def make_workload(a, query_stream=0):
    import synth

    n_comp = 1000 if a.n >= 100_000 else max(10, a.n // 100)
    return synth.c2(N=a.n, nq=a.nq, d=a.d, n_comp=n_comp, query_stream=query_stream)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
                pw.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "power_w_max": float(max(pw)) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def recorded_traffic(ef, h, vec, seed_mode, n, nq, learned):
    """DRAM bytes per launch of the search kernel from the committed ncu record, if the
    kernel sources still hash to the recorded value and the setting is the recorded one
    (otherwise None: counters of another kernel or setting would not apply)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "search_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    csrc = os.path.join(ROOT, "paper_2203_13601_gb300", "csrc")
    src = b"".join(open(os.path.join(csrc, x), "rb").read()
                   for x in ("k_search.cuh", "k_search.cu", "k_search_f32.cu",
                             "nhq_internal.cuh"))
    st = rec["setting"]
    same = (hashlib.sha256(src).hexdigest() == rec["kernel_sources_sha256"] and
            st == {"ef": ef, "h": h, "vec": VEC_NAMES[vec], "seed_mode": seed_mode} and
            n == 1_000_000 and nq == 10_000 and not learned)
    return float(rec["dram_bytes_per_launch"]) if same else None


def fp32_simt_peak(dev):
    """Measured FP32 throughput of the SIMT units: cuBLAS SGEMM with TF32 off (8192^3),
    TFLOP/s; the denominator of the brute force's ALU roofline."""
    import torch

    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        n = 8192
        g = torch.Generator(device=dev).manual_seed(0)
        x = torch.randn((n, n), device=dev, generator=g)
        y = torch.randn((n, n), device=dev, generator=g)
        for _ in range(2):
            torch.mm(x, y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record()
        for _ in range(reps):
            torch.mm(x, y)
        e1.record()
        e1.synchronize()
        return 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) / 1000.0) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def brute_force_roofline(nhq, ix, Qv, QA, k, n, d, dev, stream):
    """The brute-force fused top-k (every query against every object, constant weights)
    timed with CUDA events on its stream: 3 flops per (query, object, dimension) (the
    difference and its fused square-add) against the measured SGEMM rate."""
    import torch

    nq = Qv.shape[0]
    ids = torch.empty((nq, k), dtype=torch.uint32, device=dev)
    nhq.nhq_brute_force(ix.handle, Qv, QA, k, ids, weights=CONST_W, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 2
    e0.record(stream)
    for _ in range(reps):
        nhq.nhq_brute_force(ix.handle, Qv, QA, k, ids, weights=CONST_W, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    achieved = 3.0 * nq * n * d / (ms / 1000.0) / 1e12
    peak = fp32_simt_peak(dev)
    nominal = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x FMA flops x max clock
    return {"bound": "alu", "ms": ms, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "peak_kind": "cuBLAS SGEMM with TF32 off, measured",
            "nominal_fp32_peak": nominal, "frac_of_nominal": achieved / nominal,
            "flops_per_pair_dim": 3, "queries": nq, "objects": n}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- cpu baseline
def oracle_topk_threads(w, a, n_q, cores, ex=None):
    """Seconds for the oracle's exact fused top-k of the first n_q queries, the queries
    split into `cores` contiguous slices run by as many threads of `ex` (a pool of at
    least `cores` threads, made here when None; the oracle is C called through ctypes,
    which releases the interpreter lock during the call)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    oracle.build()
    bounds = np.linspace(0, n_q, cores + 1).astype(int)
    parts = [(lo, hi) for lo, hi in zip(bounds[:-1], bounds[1:]) if hi > lo]
    X, A = np.ascontiguousarray(w.X), np.ascontiguousarray(w.A)

    def run(pool):
        t0 = time.perf_counter()
        list(pool.map(lambda p: oracle.fused_topk(X, A, w.Qv[p[0]:p[1]], w.QA[p[0]:p[1]],
                                                  a.k, weights=CONST_W, prec=oracle.F32),
                      parts))
        return time.perf_counter() - t0

    if ex is not None:
        return run(ex)
    with ThreadPoolExecutor(max_workers=len(parts)) as pool:
        return run(pool)


def cpu_baseline(w, a, n_q):
    """The oracle as it stands: exact fused top-k (its answer to a hybrid query,
    recall 1.0) over all N objects for a bounded sample of the queries, 1 thread; and
    the same over all host cores (one slice of a larger sample per core)."""
    n_q = max(1, min(n_q, w.nq))
    dt = oracle_topk_threads(w, a, n_q, 1)
    cores = os.cpu_count() or 1
    n_all = max(1, min(n_q * cores, w.nq))
    dt_all = oracle_topk_threads(w, a, n_all, cores)
    return {"value": n_q / dt, "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n_q} of the {w.nq:,} queries, exact fused top-{a.k} over all "
                      f"{w.N:,} objects (oracle brute force, serial C, recall 1.0)",
            "seconds": dt,
            "all_cores": {"value": n_all / dt_all, "unit": "queries/s", "cores": cores,
                          "sample": f"first {n_all} queries, {cores} threads over contiguous "
                                    "slices", "seconds": dt_all}}


def oracle_search_threads(w, a, nbr, ef, seed_mode, n_q, cores, h=1, vec=0):
    """Seconds for the oracle's serial Alg. 2 (the same seed rule, ef and graph as the GPU
    search) over the first n_q queries, split into `cores` contiguous slices run by as
    many threads (the oracle is C called through ctypes, which releases the interpreter
    lock); returns (seconds, ids of those queries)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    oracle.build()
    bounds = np.linspace(0, n_q, cores + 1).astype(int)
    parts = [(lo, hi) for lo, hi in zip(bounds[:-1], bounds[1:]) if hi > lo]
    X, A = np.ascontiguousarray(w.X), np.ascontiguousarray(w.A)

    def one(pr):
        return oracle.search(X, A, nbr, w.Qv[pr[0]:pr[1]], w.QA[pr[0]:pr[1]], a.k, ef,
                             seed=12345, weights=CONST_W, prec=oracle.F32,
                             seed_mode=seed_mode, h=h, vec_round=vec, rerank=vec == 2)["ids"]

    with ThreadPoolExecutor(max_workers=len(parts)) as pool:
        t0 = time.perf_counter()
        out = list(pool.map(one, parts))
        dt = time.perf_counter() - t0
    return dt, np.concatenate(out, axis=0)


def cpu_search_baseline(w, a, nbr, ef, seed_mode, gpu_ids, n_q, h=1, vec=0):
    """The oracle's serial Alg. 2 on the bench's own graph at the chosen ef and seed rule
    (the same algorithm as the GPU search, so the two compare like with like): one thread
    over n_q queries, then one slice per host core.  Its ids equal the GPU's on these
    integer-valued data (every Gamma is exact), which the line reports."""
    n_q = max(1, min(n_q, w.nq))
    dt1, ids1 = oracle_search_threads(w, a, nbr, ef, seed_mode, n_q, 1, h, vec)
    cores = os.cpu_count() or 1
    n_all = max(1, min(n_q * cores, w.nq))
    dta, idsa = oracle_search_threads(w, a, nbr, ef, seed_mode, n_all, cores, h, vec)
    # the single call numbers its queries as the GPU launch does (the random fallback seed
    # depends on the row index), so its ids must equal the GPU's
    g = gpu_ids[:n_q].astype(np.int64)
    g[g == 0xFFFFFFFF] = -1
    return {"value": n_q / dt1, "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n_q} of the {w.nq:,} queries, serial Alg. 2 (oracle C) on the "
                      f"bench's graph, ef {ef}, h {h}, the same seed rule and scoring copy",
            "all_cores": {"value": n_all / dta, "unit": "queries/s", "cores": cores,
                          "sample": f"first {n_all} queries, {cores} threads over contiguous "
                                    "slices"},
            "ids_equal_gpu": bool((ids1 == g).all())}


def reference_arm(a, rank, world):
    if rank != 0:
        return
    w = make_workload(a)
    per = []
    cores = os.cpu_count() or 1
    steps = max(1, a.steps)
    # calibration (untimed): one query per thread on every core; the brute force costs the
    # same for every query, so this sizes the per-step sample to keep the whole run near
    # --ref-seconds (2 minutes by default).  Every regime below keeps all cores busy, so
    # `value` is always an all-cores rate.
    t1 = oracle_topk_threads(w, a, min(w.nq, cores), cores)
    budget = a.ref_seconds / steps
    frac = 1.0
    if t1 > budget:
        # even one query per thread over all objects is too long for one step: one query
        # per thread, each over a prefix of the objects sized to the budget (at least
        # max(k, 1024) objects, so the call's fixed cost stays small beside the scan; that
        # floor exceeds the budget only when a step may take less than t1 * 1024 / N; every
        # step also pays the thread pool's dispatch, about 2 ms on 8 cores), the rate scaled
        # by the fraction scanned (brute-force work is linear in N)
        per_thread = 1
        n_obj = min(w.N, max(a.k, 1024, int(w.N * budget / t1)))
        frac = n_obj / w.N
        w = type(w)(w.name, w.X[:n_obj], w.A[:n_obj], w.Qv, w.QA, w.cards, w.meta)
    else:
        per_thread = int(min(max(1, a.cpu_sample // 4), max(1.0, budget / t1)))
    n_q = min(w.nq, per_thread * cores)
    for _ in range(a.warmup):
        pass  # the oracle has no warm-up state
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=cores) as ex:
        for _ in range(steps):
            per.append(oracle_topk_threads(w, a, n_q, cores, ex))
    # the brute force's work is proportional to the objects scanned
    qps = n_q * len(per) / sum(per) * frac
    sample = (f"first {n_q} of the {a.nq:,} queries per step, exact fused top-{a.k} over "
              + (f"all {w.N:,} objects" if frac == 1.0 else
                 f"the first {w.N:,} objects, rate scaled by {frac:.4g} to all objects")
              + f" (oracle brute force in C, {cores} thread{'s' if cores > 1 else ''} over "
              "contiguous query slices, recall 1.0)")
    line = {"impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s",
            "n_gpus": a.gpus, "steps": len(per), "warmup": a.warmup,
            "ms_per_step": 1000 * float(np.mean(per)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(a), "sample_queries_per_step": n_q},
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- multi-rank timing
def max_over_ranks(ms, dist, device=None):
    """The slowest rank's timed-region length (every rank gets the same value)."""
    if dist is None:
        return float(ms)
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank_per_step, steps, world, max_ms):
    """Whole-job throughput: every rank processed its own batch each step."""
    return world * units_per_rank_per_step * steps / (max_ms / 1000.0)


# ---------------------------------------------------------------- heterogeneous batch
def c4_arm(a, rank, world, local):
    """One launch of nhq_search_batched over the c4-shaped batch per step: N = 1M,
    d = 96, attributes correlated with the cluster (5/20/100), 100,000 queries whose
    tuples have log-uniform selectivity in [1e-4, 1/3], k in {1, 10, 100} and ef
    uniform in [max(16, k), 512]; exact candidates on the tensor cores for the build."""
    import torch

    import paper_2203_13601_gb300 as nhq
    import synth
    from paper_2203_13601_gb300 import build as B

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    nhq.load_library()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    w = synth.c4()
    k_arr, ef_arr = synth.mixed_k_ef(w.nq)
    kmax = int(k_arr.max())
    X, A = torch.from_numpy(w.X).to(dev), torch.from_numpy(w.A).to(dev)
    Qv, QA = torch.from_numpy(w.Qv).to(dev), torch.from_numpy(w.QA).to(dev)
    kd, efd = torch.from_numpy(k_arr).to(dev), torch.from_numpy(ef_arr).to(dev)
    t0 = time.perf_counter()
    if a.c4_build == "nsw":
        ix = nhq.Index.create(X, A, CONST_W)
        nhq.nhq_index_build_nsw(ix.handle, a.R, L=64, wave_max=4096, rev_cap=64, seed=7, entry=1)
    else:
        ix = nhq.Index.build(X, A, degree=a.R, weights=CONST_W, K=64, knn_dtype=1)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    gt = torch.empty((w.nq, kmax), dtype=torch.uint32, device=dev)
    nhq.nhq_brute_force(ix.handle, Qv, QA, kmax, gt, weights="filter")
    ids = torch.empty((w.nq, kmax), dtype=torch.uint32, device=dev)
    dists = torch.empty((w.nq, kmax), dtype=torch.float32, device=dev)
    st = torch.empty(w.nq, dtype=torch.int32, device=dev)
    ndc = torch.empty(w.nq, dtype=torch.int32, device=dev)
    exps = torch.empty(w.nq, dtype=torch.int32, device=dev)

    shape = {}  # the tuned launch shape, once tuned

    def run(diag=False, mode=nhq.SEED_ATTRIBUTE_NEAR):
        nhq.nhq_search_batched(ix.handle, Qv, QA, kd, efd, kmax, ids, dists, None, st,
                               ndc=ndc if diag else None, expansions=exps if diag else None,
                               seed=12345, seed_mode=mode, **shape)

    gt_h = gt.cpu().numpy().astype(np.int64)
    # hybrid recall with each query's own k (Sec. 6.1)
    mult = np.array([1, 256, 65536])[: w.m]
    codes, qcodes = (w.A.astype(np.int64) * mult).sum(1), (w.QA.astype(np.int64) * mult).sum(1)
    uniq, cnt = np.unique(codes, return_counts=True)
    pos = np.minimum(np.searchsorted(uniq, qcodes), len(uniq) - 1)
    P = np.where(uniq[pos] == qcodes, cnt[pos], 0)
    sel = P / w.N

    def quality(mode):
        run(diag=True, mode=mode)
        torch.cuda.synchronize()
        ids_h = ids.cpu().numpy().astype(np.int64)
        nd, ex = ndc.cpu().numpy().astype(np.float64), exps.cpu().numpy().astype(np.float64)
        recq = np.full(w.nq, np.nan)
        for q in range(w.nq):
            kq = int(k_arr[q])
            if P[q] == 0:
                continue
            got = ids_h[q, :kq]
            got = got[got != 0xFFFFFFFF]
            got = got[(w.A[got] == w.QA[q]).all(axis=1)]
            g = gt_h[q, :kq]
            g = g[g != 0xFFFFFFFF]
            recq[q] = len(set(got.tolist()) & set(g.tolist())) / min(kq, int(P[q]))
        # per selectivity band (|P| / N of the query's tuple)
        bands = []
        for lo, hi in ((1e-4, 1e-3), (1e-3, 1e-2), (1e-2, 1e-1), (1e-1, 1.0)):
            m_ = (sel >= lo) & (sel < hi) & ~np.isnan(recq)
            if m_.any():
                bands.append({"selectivity": [lo, hi], "queries": int(m_.sum()),
                              "recall": float(np.nanmean(recq[m_])),
                              "mean_expansions": float(ex[m_].mean()),
                              "mean_ndc": float(nd[m_].mean())})
        return float(np.nanmean(recq)), bands, nd, ex

    recall_even, bands_even, _, _ = quality(nhq.SEED_ATTRIBUTE)
    recall, bands, ndc_h, exp_h = quality(nhq.SEED_ATTRIBUTE_NEAR)

    def timed_ms(fn, reps=5):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # the autotuner on this batch, then the tuned shape and a captured graph of it
    default_ms = timed_ms(run)
    tmp = torch.empty((w.nq, kmax), dtype=torch.uint32, device=dev)
    tuned = nhq.nhq_autotune_batched(ix.handle, Qv, QA, kd, efd, kmax, tmp, seed=12345,
                                     seed_mode=nhq.SEED_ATTRIBUTE_NEAR)
    shape.update({x: tuned[x] for x in ("warps_per_query", "tile_rows", "warps_per_block",
                                        "hash_bits")})
    tuned_ms = timed_ms(run)
    if tuned_ms > default_ms:  # the single-call tuner can mislead by noise: keep the better
        shape.clear()
    graph = nhq.nhq_search_graph_create_batched(ix.handle, Qv, QA, kd, efd, kmax, ids, dists,
                                                seed=12345, seed_mode=nhq.SEED_ATTRIBUTE_NEAR,
                                                **shape)
    graph_ms = timed_ms(lambda: graph.launch(stream))
    graph.close()
    bytes_q = ndc_h * (4 * w.d + 4) + exp_h * a.R * 4 + w.d * 4 + k_arr * 9
    alg_bytes = float(bytes_q.sum())
    for _ in range(max(3, a.warmup)):
        run()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(a.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s0, s1 in evs:
        s0.record(stream)
        run()
        s1.record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    total_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    clk = clocks.stop()
    launch_ms = float(np.mean([s0.elapsed_time(s1) for s0, s1 in evs]))
    peak, peak_kind = peaks()
    achieved = alg_bytes / (launch_ms / 1000.0) / 1e9
    line = {
        "metric": "QPS of the heterogeneous batch (mixed k and ef, correlated attributes)",
        "value": weak_scaling_value(w.nq, a.steps, world, total_ms), "unit": "queries/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "c4-shaped: N=1,000,000 d=96 f32 (1,000 centroids), m=3 attrs "
                               "5/20/100 correlated with the cluster, 100,000 queries with "
                               "log-uniform selectivity in [1e-4, 1/3], k in {1,10,100}, ef in "
                               "[max(16,k), 512], R=32, weights w_v=1 w_l=10000",
                   "launch": "nhq_search_batched, nearest attribute-entry seeds",
                   "recall": recall, "recall_kind": "hybrid Recall@k (each query's own k)",
                   "by_selectivity": bands,
                   "graph": ("NPG_nsw, attribute entry, insertion waves" if a.c4_build == "nsw"
                             else "NPG_kgraph, exact candidates K=64"),
                   "evenly_spaced_seeds": {"recall": recall_even,
                                           "by_selectivity": bands_even},
                   "mean_ef": float(ef_arr.mean()), "build_s": t_build,
                   "l2": "inputs larger than L2 (vectors 384 MB + adjacency 256 MB)",
                   "autotune": {"tuned": tuned, "default_ms": default_ms, "tuned_ms": tuned_ms,
                                "used": dict(shape) or "default (faster)",
                                "captured_graph_ms": graph_ms}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": launch_ms,
                     "mean_ndc": float(ndc_h.mean()), "mean_expansions": float(exp_h.mean())},
        "gpu_launches": a.steps * 3, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ix.close()
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- the largest set
def c5_arm(a):
    """The c5-shaped set: N = 10M, d = 96 FP16 vectors (passed to the library as f16 and
    scored from its f16 copy, 192-byte rows; every value is an f16, so the scores equal
    f32 scores), 4,096 centroids, m = 3 Zipf attributes (10/50/200), 50,000 queries,
    k = 10: build time, then QPS at hybrid Recall@10 >= target over an ef sweep for the
    plain form (attribute-entry seeds) and the learned entry point (cells and the entry
    model trained on 1,000,000 traces of the plain search); the faster is timed."""
    import types

    import torch

    import paper_2203_13601_gb300 as nhq
    import synth
    from paper_2203_13601_gb300 import build as B

    B.build()
    nhq.load_library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    w = synth.c5()
    t_gen = time.perf_counter() - t0
    X = torch.from_numpy(w.X.astype(np.float16)).to(dev)  # the configured FP16 input
    A = torch.from_numpy(w.A).to(dev)
    Qv, QA = torch.from_numpy(w.Qv).to(dev), torch.from_numpy(w.QA).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = nhq.Index.build(X, A, degree=a.R, weights=CONST_W, K=64, knn_dtype=1)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    del X
    k = a.k
    gt = torch.empty((w.nq, k), dtype=torch.uint32, device=dev)
    nhq.nhq_brute_force(ix.handle, Qv, QA, k, gt, weights="filter")
    gt_h = gt.cpu().numpy()
    P = match_counts(w.A, w.QA)
    ids, dd, ch = (torch.empty((w.nq, k), dtype=torch.uint32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.float32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.uint8, device=dev))
    ndc = torch.empty(w.nq, dtype=torch.int32, device=dev)
    exps = torch.empty(w.nq, dtype=torch.int32, device=dev)
    # the learned entry point, trained on 1M traces of the plain search
    ntr = min(a.train_q * 10, 1_000_000)
    Qt, QAt = synth.c5_queries(ntr, 1)
    wtr = types.SimpleNamespace(Qv=Qt, QA=QAt, nq=ntr)
    E = a.cells if a.cells > 0 else 1024
    model, t_train, n_tr = train_entry(nhq, ix, w, wtr, E, k, dev, epochs=6)
    del Qt, QAt, wtr

    shapes = {}  # tuned launch shape per form

    def form_kw(form):
        if form == "learned":
            return dict(seed_mode=nhq.SEED_CELL_LEARNED, entry_model=model,
                        entry_cells=a.entry_T)
        return dict(seed_mode=nhq.SEED_ATTRIBUTE)

    def run(form, ef, diag=False):
        nhq.nhq_search(ix.handle, Qv, QA, k, ef, ids, dd, ch, ndc=ndc if diag else None,
                       expansions=exps if diag else None, seed=12345,
                       vec_dtype=nhq.VEC_F16, stream=stream, **form_kw(form),
                       **shapes.get(form, {}))

    def timed(form, ef, reps):
        for _ in range(2):
            run(form, ef)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run(form, ef)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    sweeps, found = {}, {}
    for form in ("plain", "learned"):
        sweeps[form] = []
        for ef in (16, 20, 24, 32, 48, 64, 96):
            run(form, ef, diag=True)
            torch.cuda.synchronize()
            rec, _ = hybrid_recall(ids.cpu().numpy(), w.A, w.QA, gt_h, P, k)
            ms = timed(form, ef, 3)
            sweeps[form].append({"ef": ef, "recall": rec, "ms": ms,
                                 "mean_expansions": float(exps.float().mean().item()),
                                 "max_expansions": int(exps.max().item())})
            if rec >= a.target:
                found[form] = sweeps[form][-1]
                break
    # the autotuner on each form at its ef; the tuned shape is kept where it is faster
    tuned = {}
    for f in found:
        t = nhq.nhq_autotune(ix.handle, Qv, QA, k, found[f]["ef"], ids, seed=12345,
                             vec_dtype=nhq.VEC_F16, **form_kw(f))
        shape = {x: t[x] for x in ("warps_per_query", "tile_rows", "warps_per_block",
                                   "hash_bits")}
        before = timed(f, found[f]["ef"], 5)
        shapes[f] = shape
        after = timed(f, found[f]["ef"], 5)
        if after >= before:
            shapes.pop(f)
        tuned[f] = dict(t, default_ms=before, tuned_ms=after, used=f in shapes)
    chosen = min(found, key=lambda f: found[f]["ms"])
    ef = found[chosen]["ef"]
    run(chosen, ef, diag=True)
    torch.cuda.synchronize()
    ndc_h, exp_h = ndc.cpu().numpy().astype(np.float64), exps.cpu().numpy().astype(np.float64)
    alg_bytes = float((ndc_h * (2 * w.d + 4) + exp_h * a.R * 4 + w.d * 4 + k * 9).sum())
    steps = min(a.steps, 200)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    timed_ms = {f: timed(f, found[f]["ef"], steps) for f in found}
    clk = clocks.stop()
    total_ms = timed_ms[chosen] * steps
    peak, peak_kind = peaks()
    achieved = alg_bytes / (total_ms / steps / 1000.0) / 1e9
    print(json.dumps({
        "metric": f"QPS at hybrid Recall@{k} >= {a.target} on the 10M set",
        "value": w.nq * steps / (total_ms / 1000.0), "unit": "queries/s", "n_gpus": 1,
        "steps": steps, "warmup": a.warmup, "ms_per_step": total_ms / steps,
        "higher_is_better": True, "dtype": "f16", "data": "synthetic",
        "config": {"workload": "c5-shaped: N=10,000,000 d=96 FP16 (built from the f16 rows, "
                               "scored from the index's f16 copy, 192-byte rows), 4,096 "
                               "centroids, m=3 attrs 10/50/200 Zipf, 50,000 queries, k=10, "
                               "R=32, weights w_v=1 w_l=10000",
                   "chosen": chosen, "ef": ef, "recall": found[chosen]["recall"],
                   "build_s": t_build, "gen_s": t_gen,
                   "queries_with_no_match": int((P == 0).sum()),
                   "entry": {"cells": E, "cells_per_query": a.entry_T, "traces": n_tr,
                             "train_s": t_train}},
        "sweeps": sweeps,
        "timed_ms": timed_ms,
        "autotune": tuned,
        "qps": {f: w.nq / (timed_ms[f] / 1000.0) for f in timed_ms},
        "learned_vs_plain": (timed_ms["plain"] / timed_ms["learned"]
                             if "learned" in timed_ms and "plain" in timed_ms else None),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "mean_ndc": float(ndc_h.mean()), "mean_expansions": float(exp_h.mean())},
        "clocks": clk}), flush=True)
    ix.close()


def train_entry(nhq, ix, w, wtr, E, k, dev, epochs=6, batch=1024, lr=2e-3):
    """The learned entry point: cells, then the entry model trained on the cells of the
    first results of the plain search (attribute entry, ef 64) for the training queries.
    Returns (model, seconds, number of labelled traces)."""
    import torch

    t0 = time.perf_counter()
    nhq.nhq_index_build_cells(ix.handle, E)
    Qt, QAt = torch.from_numpy(wtr.Qv).to(dev), torch.from_numpy(wtr.QA).to(dev)
    idt = torch.empty((wtr.nq, k), dtype=torch.uint32, device=dev)
    nhq.nhq_search(ix.handle, Qt, QAt, k, 64, idt, seed=1, seed_mode=nhq.SEED_ATTRIBUTE)
    lab = torch.empty(wtr.nq, dtype=torch.int32, device=dev)
    nhq.nhq_entry_labels(ix.handle, idt, lab)
    keep = lab >= 0
    Qk, lk = Qt[keep].contiguous(), lab[keep].contiguous()
    rms = float(np.sqrt(np.mean(np.square(wtr.Qv[:2000].astype(np.float64)))))
    p = (np.random.default_rng(3).standard_normal(nhq.nhq_entry_param_count(w.d, E)) *
         0.05).astype(np.float32)
    p[0] = 1.0 / max(rms, 1e-12) / np.sqrt(w.d)  # inputs of about unit norm
    P = torch.from_numpy(p).to(dev)
    nhq.nhq_entry_train(P, E, Qk, lk, epochs=epochs, batch=batch, lr=lr)
    torch.cuda.synchronize()
    return P, time.perf_counter() - t0, int(keep.sum().item())


def f64_error(w, ids_h, dists_h, weights, n=200):
    """Max and mean relative error of returned Gamma values against Gamma computed in f64
    from the f32 rows (Eq. 1 and Eq. 6), over the first n queries."""
    errs = []
    for q in range(min(n, ids_h.shape[0])):
        for j in range(ids_h.shape[1]):
            v = int(ids_h[q, j])
            if v == 0xFFFFFFFF:
                continue
            dl = float(np.sqrt(np.sum((w.X[v].astype(np.float64) -
                                       w.Qv[q].astype(np.float64)) ** 2)))
            ch = int((w.A[v] != w.QA[q]).sum())
            g = weights[0] * dl + weights[1] * ch
            vec_part = weights[0] * dl  # the attribute term is exact
            errs.append(abs(float(dists_h[q, j]) - g) / max(vec_part, 1e-30))
    e = np.array(errs) if errs else np.zeros(1)
    return {"max_rel": float(e.max()), "mean_rel": float(e.mean()),
            "of": "the vector term w_v * delta"}


def c3_arm(a):
    """The c3-shaped set (GIST1M-shaped): N = 1M, d = 960 unit-normalised rows (1,000
    centroids), m = 4 uniform attributes (2/5/10/50), 10,000 queries, k = 10.  Every form
    -- scoring copy (f32; bf16; bf16 or fp8-e4m3 with the f32 re-rank), warps per query
    (1, 2, 4), seeds by attribute entry or by the learned entry cells -- is swept for the
    smallest ef reaching hybrid Recall@10 >= target; the fastest ("chosen") is autotuned
    and timed beside the plain f32 form (one warp per query, attribute entry), with its
    HBM roofline and the distance error of each scoring copy against f64 on the same
    results."""
    import torch

    import paper_2203_13601_gb300 as nhq
    import synth
    from paper_2203_13601_gb300 import build as B

    B.build()
    nhq.load_library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    w = synth.c3(N=a.n, nq=a.nq)
    wtr = synth.c3(N=a.n, nq=a.train_q, query_stream=1)
    t_gen = time.perf_counter() - t0
    X, A = torch.from_numpy(w.X).to(dev), torch.from_numpy(w.A).to(dev)
    Qv, QA = torch.from_numpy(w.Qv).to(dev), torch.from_numpy(w.QA).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = nhq.Index.build(X, A, degree=a.R, weights=CONST_W, K=64, knn_dtype=1)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    k = a.k
    gt = torch.empty((w.nq, k), dtype=torch.uint32, device=dev)
    t0 = time.perf_counter()
    nhq.nhq_brute_force(ix.handle, Qv, QA, k, gt, weights="filter")
    torch.cuda.synchronize()
    t_gt = time.perf_counter() - t0
    gt_h = gt.cpu().numpy()
    P_cnt = match_counts(w.A, w.QA)
    E = a.cells if a.cells > 0 else 512
    model, t_train, n_tr = train_entry(nhq, ix, w, wtr, E, k, dev)
    ids, dd, ch = (torch.empty((w.nq, k), dtype=torch.uint32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.float32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.uint8, device=dev))
    ndc = torch.empty(w.nq, dtype=torch.int32, device=dev)
    exps = torch.empty(w.nq, dtype=torch.int32, device=dev)

    def kw_of(form):
        kw = dict(seed=12345, vec_dtype=form["vec"], rerank=form["rerank"],
                  seed_mode=form["seeds"], warps_per_query=form["wpq"],
                  warps_per_block=form.get("wpb", 0), hash_bits=form.get("bits", 0))
        if form["seeds"] == nhq.SEED_CELL_LEARNED:
            kw.update(entry_model=model, entry_cells=a.entry_T)
        return kw

    def run(form, ef, diag=False):
        nhq.nhq_search(ix.handle, Qv, QA, k, ef, ids, dd, ch, ndc=ndc if diag else None,
                       expansions=exps if diag else None, stream=stream, **kw_of(form))

    def timed(form, ef, reps=5):
        run(form, ef)
        run(form, ef)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run(form, ef)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    efs = [int(x) for x in a.efs.split(",") if int(x) >= k]
    names = {(0, 0): "f32", (1, 0): "bf16", (1, 1): "bf16 + f32 re-rank",
             (2, 1): "fp8-e4m3 + f32 re-rank"}
    forms, sweep, errors = [], [], {}
    for (vec, rr), nm in names.items():
        for seeds in (nhq.SEED_ATTRIBUTE, nhq.SEED_CELL_LEARNED):
            at = None  # (ef, recall) reaching the target; it does not depend on wpq
            for wpq in (1, 2, 4):
                form = {"vec": vec, "rerank": rr, "seeds": seeds, "wpq": wpq}
                if wpq == 1:
                    for ef in efs:
                        run(form, ef)
                        torch.cuda.synchronize()
                        rec, _ = hybrid_recall(ids.cpu().numpy(), w.A, w.QA, gt_h, P_cnt, k)
                        if rec >= a.target:
                            at = (ef, rec)
                            break
                if at is None:
                    break
                found = (at[0], at[1], timed(form, at[0]))
                if wpq == 1 and seeds == nhq.SEED_ATTRIBUTE:
                    errors[nm] = f64_error(w, ids.cpu().numpy(), dd.cpu().numpy(), CONST_W)
                row = dict(form, scoring=nm, ef=found[0], recall=found[1], ms=found[2],
                           seeds_name=["random", "attribute entry", "given",
                                       "nearest attribute entry", "nearest cells",
                                       "learned cells"][seeds])
                sweep.append(row)
                forms.append(row)
    plain = next(r for r in forms if r["vec"] == 0 and r["seeds"] == nhq.SEED_ATTRIBUTE and
                 r["wpq"] == 1)
    chosen = dict(min(forms, key=lambda r: r["ms"]))
    # the autotuner on the chosen form: warps per query, warps per block, filter size
    tmp = torch.empty((w.nq, k), dtype=torch.uint32, device=dev)
    kwc = kw_of(chosen)
    wpq_t, wpb_t, bits_t, _ = nhq.nhq_autotune_search(
        ix.handle, Qv, QA, k, chosen["ef"], tmp, seed=12345, vec_dtype=chosen["vec"],
        rerank=chosen["rerank"], seed_mode=kwc["seed_mode"], return_wpq=True) \
        if chosen["seeds"] != nhq.SEED_CELL_LEARNED else (chosen["wpq"], 0, 0, 0)
    tuned = dict(chosen, wpq=wpq_t, wpb=wpb_t, bits=bits_t)
    if timed(tuned, chosen["ef"]) < chosen["ms"]:
        chosen = tuned
    run(chosen, chosen["ef"], diag=True)
    torch.cuda.synchronize()
    ndc_h, exp_h = ndc.cpu().numpy().astype(np.float64), exps.cpu().numpy().astype(np.float64)
    row_bytes = {0: 4, 1: 2, 2: 1}[chosen["vec"]] * w.d
    bpq = ndc_h * (row_bytes + 4) + exp_h * a.R * 4 + w.d * 4 + k * 9
    if chosen["rerank"]:
        bpq = bpq + chosen["ef"] * 4 * w.d  # the re-rank reads the pool's f32 rows
    alg_bytes = float(bpq.sum())
    steps = max(3, min(a.steps, 100))
    out = {}
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    for tag, form in (("plain_f32", plain), ("chosen", chosen)):
        for _ in range(max(3, a.warmup)):
            run(form, form["ef"])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            run(form, form["ef"])
        e1.record(stream)
        torch.cuda.synchronize()
        out[tag] = e0.elapsed_time(e1) / steps
    clk = clocks.stop()
    peak, peak_kind = peaks()
    achieved = alg_bytes / (out["chosen"] / 1000.0) / 1e9
    print(json.dumps({
        "metric": f"QPS at hybrid Recall@{k} >= {a.target} on the 1M x 960 set, chosen vs "
                  "plain f32",
        "value": w.nq / (out["chosen"] / 1000.0), "unit": "queries/s", "n_gpus": 1,
        "steps": steps, "warmup": a.warmup, "ms_per_step": out["chosen"],
        "higher_is_better": True, "dtype": ["f32", "bf16", "fp8-e4m3"][chosen["vec"]],
        "data": "synthetic",
        "config": {"workload": f"c3-shaped: N={w.N:,} d=960 unit rows (1,000 centroids), m=4 "
                               f"attrs 2/5/10/50 uniform, {w.nq:,} queries, k={k}, R={a.R}, "
                               "weights w_v=1 w_l=10000",
                   "chosen": chosen, "build_s": t_build, "gen_s": t_gen,
                   "ground_truth_s": t_gt, "entry_cells": E, "entry_T": a.entry_T,
                   "entry_train_s": t_train, "entry_traces": n_tr,
                   "queries_with_no_match": int((P_cnt == 0).sum())},
        "plain_f32": dict(plain, qps=w.nq / (out["plain_f32"] / 1000.0),
                          ms_timed=out["plain_f32"]),
        "chosen_beats_plain": out["chosen"] < out["plain_f32"],
        "speedup_vs_plain": out["plain_f32"] / out["chosen"],
        "forms": sweep,
        "f64_error": errors,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "mean_ndc": float(ndc_h.mean()), "mean_expansions": float(exp_h.mean())},
        "clocks": clk}), flush=True)
    ix.close()


# ---------------------------------------------------------------- weightings
def curves_arm(a):
    """The weightings of Sec. 6.5 on the c2 workload, each with its own composite index
    (exact candidates on the tensor cores) and attribute-entry seeds: i harmonic mean of
    delta and chi, ii the same with chi -> 1 / 100 chi, iii delta / delta_max + chi / m
    (delta_max = the bounding-box diagonal of the set, a bound known in advance), iv
    delta + delta chi / m (the library default), v delta + 10,000 chi.  For each: the
    cheapest ef reaching hybrid Recall@10 >= target, else the best recall of the sweep."""
    import torch

    import paper_2203_13601_gb300 as nhq
    from paper_2203_13601_gb300 import build as B

    B.build()
    nhq.load_library()
    dev = torch.device("cuda", 0)
    w = make_workload(a)
    X, A = torch.from_numpy(w.X).to(dev), torch.from_numpy(w.A).to(dev)
    Qv, QA = torch.from_numpy(w.Qv).to(dev), torch.from_numpy(w.QA).to(dev)
    k = a.k
    dmax = float(np.linalg.norm(w.X.max(axis=0).astype(np.float64) - w.X.min(axis=0)))
    curves = [("i", "harmonic"), ("ii", ("harmonic", 100.0)),
              ("iii", (1.0 / dmax, 1.0 / w.m)), ("iv", None), ("v", CONST_W)]
    mult = np.array([1, 256, 65536])[: w.m]
    codes, qcodes = (w.A.astype(np.int64) * mult).sum(1), (w.QA.astype(np.int64) * mult).sum(1)
    uniq, cnt = np.unique(codes, return_counts=True)
    pos = np.minimum(np.searchsorted(uniq, qcodes), len(uniq) - 1)
    P = np.where(uniq[pos] == qcodes, cnt[pos], 0)
    gt = torch.empty((w.nq, k), dtype=torch.uint32, device=dev)
    ids, dd, ch = (torch.empty((w.nq, k), dtype=torch.uint32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.float32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.uint8, device=dev))
    rows = []
    for name, wts in curves:
        t0 = time.perf_counter()
        ix = nhq.Index.build(X, A, degree=a.R, weights=wts, K=64, knn_dtype=1)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        if name == "i":
            nhq.nhq_brute_force(ix.handle, Qv, QA, k, gt, weights="filter")
            gt_h = gt.cpu().numpy()
        sweep = []
        for ef in (16, 24, 32, 48, 64, 96, 128, 200):
            run = lambda ef=ef: nhq.nhq_search(ix.handle, Qv, QA, k, ef, ids, dd, ch,
                                               seed=12345, seed_mode=nhq.SEED_ATTRIBUTE)
            for _ in range(2):
                run()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            rec, _ = hybrid_recall(ids.cpu().numpy(), w.A, w.QA, gt_h, P, k)
            ms = e0.elapsed_time(e1)
            sweep.append({"ef": ef, "recall": rec, "ms": ms, "qps": w.nq / ms * 1e3})
            if rec >= a.target:
                break
        ix.close()
        best = sweep[-1] if sweep[-1]["recall"] >= a.target else max(sweep,
                                                                        key=lambda r: r["recall"])
        rows.append({"curve": name, "weights": str(wts), "build_s": t_build, "best": best,
                     "reached_target": best["recall"] >= a.target, "sweep": sweep})
    print(json.dumps({"metric": f"hybrid Recall@{k} and QPS per weighting (Sec. 6.5)",
                      "config": {"workload": workload_name(a), "delta_max": dmax,
                                 "target": a.target},
                      "curves": rows}), flush=True)


# ---------------------------------------------------------------- attribute dimension
ATTR_CARDS = (3, 10, 20, 4, 5, 8, 2, 3, 6)


def match_counts(A, QA):
    """|P| for every query: the number of objects whose attribute rows equal its row."""
    rows = np.ascontiguousarray(np.concatenate([A, QA]))
    key = rows.view(np.dtype((np.void, rows.shape[1]))).ravel()
    _, inv = np.unique(key, return_inverse=True)
    inv = inv.ravel()
    cnt = np.bincount(inv[: len(A)], minlength=int(inv.max()) + 1)
    return cnt[inv[len(A):]]


def attrdim_arm(a):
    """The attribute dimension of Sec. 6.4 on c2-shaped vectors: m = 3, 6 and 9 Zipf
    attributes (cards 3/10/20, then 4/5/8, then 2/3/6; the first m columns are the same
    draws for every m), one composite index each (exact candidates on the tensor cores,
    constant weights).  For each, with attribute-entry and with random seeds: the cheapest
    ef reaching hybrid Recall@10 >= target, else the best recall; and the build time and
    |P| statistics."""
    import torch

    import paper_2203_13601_gb300 as nhq
    import synth
    from paper_2203_13601_gb300 import build as B

    B.build()
    nhq.load_library()
    dev = torch.device("cuda", 0)
    k = a.k
    rows = []
    for m in (3, 6, 9):
        w = synth.c2(N=a.n, nq=a.nq, d=a.d, cards=ATTR_CARDS[:m],
                     n_comp=1000 if a.n >= 100_000 else max(10, a.n // 100))
        P = match_counts(w.A, w.QA)
        X, A = torch.from_numpy(w.X).to(dev), torch.from_numpy(w.A).to(dev)
        Qv, QA = torch.from_numpy(w.Qv).to(dev), torch.from_numpy(w.QA).to(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ix = nhq.Index.build(X, A, degree=a.R, weights=CONST_W, K=64, knn_dtype=1)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        gt = torch.empty((w.nq, k), dtype=torch.uint32, device=dev)
        nhq.nhq_brute_force(ix.handle, Qv, QA, k, gt, weights="filter")
        gt_h = gt.cpu().numpy()
        ids, dd, ch = (torch.empty((w.nq, k), dtype=torch.uint32, device=dev),
                       torch.empty((w.nq, k), dtype=torch.float32, device=dev),
                       torch.empty((w.nq, k), dtype=torch.uint8, device=dev))
        by_seeds = {}
        for sname, smode in (("attribute_entry", nhq.SEED_ATTRIBUTE),
                             ("random", nhq.SEED_RANDOM)):
            sweep = []
            for ef in (16, 24, 32, 48, 64, 96, 128, 200, 320, 500):
                run = lambda ef=ef: nhq.nhq_search(ix.handle, Qv, QA, k, ef, ids, dd, ch,
                                                   seed=12345, seed_mode=smode)
                for _ in range(3):
                    run()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(5):
                    run()
                e1.record()
                torch.cuda.synchronize()
                rec, excl = hybrid_recall(ids.cpu().numpy(), w.A, w.QA, gt_h, P, k)
                ms = e0.elapsed_time(e1) / 5
                sweep.append({"ef": ef, "recall": rec, "ms": ms, "qps": w.nq / ms * 1e3})
                if rec >= a.target:
                    break
            best = sweep[-1] if sweep[-1]["recall"] >= a.target else max(
                sweep, key=lambda r: r["recall"])
            by_seeds[sname] = {"best": best, "reached_target": best["recall"] >= a.target,
                               "sweep": sweep}
        ix.close()
        del X, A
        pos = P[P > 0]
        rows.append({"m": m, "cards": list(ATTR_CARDS[:m]),
                     "distinct_tuples": int(len(np.unique(
                         np.ascontiguousarray(w.A).view(np.dtype((np.void, m)))))),
                     "queries_with_no_match": int((P == 0).sum()),
                     "median_P": float(np.median(pos)) if pos.size else 0.0,
                     "build_s": t_build, "seeds": by_seeds})
    print(json.dumps({"metric": f"hybrid Recall@{k} and QPS per attribute dimension m (Sec. 6.4)",
                      "config": {"workload": f"c2-shaped vectors N={a.n:,} d={a.d}, "
                                             f"{a.nq:,} queries, R={a.R}, weights w_v=1 "
                                             "w_l=10000, Zipf s=1 attributes",
                                 "target": a.target},
                      "dims": rows}), flush=True)


# ---------------------------------------------------------------- partial constraints
def wildcard_arm(a):
    """Partial constraints on the c2 workload: every query leaves one attribute open
    (code 255 with the wildcard switch on; attribute 0, 1 or 2 in turn), on the composite
    index of the headline (exact candidates, constant weights).  Ground truth: the
    filter-mode brute force under the same rule.  For each seed rule (nearest attribute
    entry, then attribute entry; the first only with --steps 1) the cheapest ef reaching
    hybrid Recall@10 >= target, else the best recall."""
    import torch

    import paper_2203_13601_gb300 as nhq
    from paper_2203_13601_gb300 import build as B

    B.build()
    nhq.load_library()
    dev = torch.device("cuda", 0)
    w = make_workload(a)
    k = a.k
    QA_h = w.QA.copy()
    QA_h[np.arange(w.nq), np.arange(w.nq) % w.m] = 255
    X, A = torch.from_numpy(w.X).to(dev), torch.from_numpy(w.A).to(dev)
    Qv, QA = torch.from_numpy(w.Qv).to(dev), torch.from_numpy(QA_h).to(dev)
    ix = nhq.Index.build(X, A, degree=a.R, weights=CONST_W, K=64, knn_dtype=1)
    gt = torch.empty((w.nq, k), dtype=torch.uint32, device=dev)
    gtd = torch.empty((w.nq, k), dtype=torch.float32, device=dev)
    nhq.nhq_brute_force(ix.handle, Qv, QA, k, gt, gtd, weights="filter", wildcard=1)
    gt_h = gt.cpu().numpy()
    # |P| under the partial constraint (the filter mode leaves +inf past the matches)
    P = np.minimum(np.isfinite(gtd.cpu().numpy()).sum(1), k)
    ids, dd, ch = (torch.empty((w.nq, k), dtype=torch.uint32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.float32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.uint8, device=dev))
    open_mask = QA_h == 255

    def recall_of(ids_h):
        hits = []
        for q in range(w.nq):
            if P[q] == 0:
                continue
            got = ids_h[q][ids_h[q] != 0xFFFFFFFF].astype(np.int64)
            cols = ~open_mask[q]
            got = got[(w.A[got][:, cols] == QA_h[q, cols]).all(axis=1)]
            g = gt_h[q][gt_h[q] != 0xFFFFFFFF]
            hits.append(len(set(got.tolist()) & set(g.tolist())) / min(k, int(P[q])))
        return float(np.mean(hits))

    by_seeds = {}
    modes = (("nearest_attribute_entry", nhq.SEED_ATTRIBUTE_NEAR),
             ("attribute_entry", nhq.SEED_ATTRIBUTE))
    for sname, smode in modes[: 1 if a.steps == 1 else 2]:
        sweep = []
        for ef in (16, 24, 32, 48, 64, 96, 128, 200, 320, 500):
            run = lambda ef=ef: nhq.nhq_search(ix.handle, Qv, QA, k, ef, ids, dd, ch, seed=12345,
                                               seed_mode=smode, wildcard=1)
            for _ in range(3):
                run()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                run()
            e1.record()
            torch.cuda.synchronize()
            rec = recall_of(ids.cpu().numpy())
            ms = e0.elapsed_time(e1) / 5
            sweep.append({"ef": ef, "recall": rec, "ms": ms, "qps": w.nq / ms * 1e3})
            if rec >= a.target:
                break
        best = sweep[-1] if sweep[-1]["recall"] >= a.target else max(sweep,
                                                                        key=lambda r: r["recall"])
        by_seeds[sname] = {"best": best, "reached_target": best["recall"] >= a.target,
                           "sweep": sweep}
    ix.close()
    print(json.dumps({"metric": f"hybrid Recall@{k} and QPS with one attribute left open",
                      "config": {"workload": workload_name(a) + "; each query leaves attribute "
                                 "q mod 3 open (wildcard)", "target": a.target,
                                 "queries_with_no_match": int((P == 0).sum())},
                      "seeds": by_seeds}), flush=True)


# ---------------------------------------------------------------- build methods
def builds_arm(a):
    """The ways to build the composite index on the c2 workload (constant weights,
    R = 32): NPG_kgraph on exact candidate sets (tensor cores), NPG_kgraph on NN-descent
    candidate sets (Sec. 4.3), and the incremental NPG_nsw build in insertion waves; for
    each the build time and the cheapest ef reaching hybrid Recall@10 >= target."""
    import torch

    import paper_2203_13601_gb300 as nhq
    from paper_2203_13601_gb300 import build as B

    B.build()
    nhq.load_library()
    dev = torch.device("cuda", 0)
    w = make_workload(a)
    X, A = torch.from_numpy(w.X).to(dev), torch.from_numpy(w.A).to(dev)
    Qv, QA = torch.from_numpy(w.Qv).to(dev), torch.from_numpy(w.QA).to(dev)
    k = a.k
    mult = np.array([1, 256, 65536])[: w.m]
    codes, qcodes = (w.A.astype(np.int64) * mult).sum(1), (w.QA.astype(np.int64) * mult).sum(1)
    uniq, cnt = np.unique(codes, return_counts=True)
    pos = np.minimum(np.searchsorted(uniq, qcodes), len(uniq) - 1)
    P = np.where(uniq[pos] == qcodes, cnt[pos], 0)
    ids, dd, ch = (torch.empty((w.nq, k), dtype=torch.uint32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.float32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.uint8, device=dev))
    gt = torch.empty((w.nq, k), dtype=torch.uint32, device=dev)
    rows, gt_h = [], None

    def make(method):
        if method == "kgraph_exact":
            return nhq.Index.build(X, A, degree=a.R, weights=CONST_W, K=64, knn_dtype=1)
        if method == "kgraph_nndescent":
            return nhq.Index.build(X, A, degree=a.R, weights=CONST_W, K=64, knn_dtype=2)
        ix = nhq.Index.create(X, A, CONST_W)
        nhq.nhq_index_build_nsw(ix.handle, a.R, L=64, wave_max=4096, rev_cap=64, seed=7,
                                entry=1 if method == "nsw_attribute_entry" else 0)
        return ix

    for method in ("kgraph_exact", "kgraph_nndescent", "nsw_id_entry", "nsw_attribute_entry"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ix = make(method)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        if gt_h is None:
            nhq.nhq_brute_force(ix.handle, Qv, QA, k, gt, weights="filter")
            gt_h = gt.cpu().numpy()
        sweep = []
        for ef in (16, 24, 32, 48, 64, 96, 128, 200):
            run = lambda ef=ef: nhq.nhq_search(ix.handle, Qv, QA, k, ef, ids, dd, ch,
                                               seed=12345, seed_mode=nhq.SEED_ATTRIBUTE)
            for _ in range(2):
                run()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            rec, _ = hybrid_recall(ids.cpu().numpy(), w.A, w.QA, gt_h, P, k)
            ms = e0.elapsed_time(e1)
            sweep.append({"ef": ef, "recall": rec, "ms": ms, "qps": w.nq / ms * 1e3})
            if rec >= a.target:
                break
        ix.close()
        best = sweep[-1] if sweep[-1]["recall"] >= a.target else max(sweep,
                                                                        key=lambda r: r["recall"])
        rows.append({"method": method, "build_s": t_build, "best": best, "sweep": sweep})
    print(json.dumps({"metric": f"build time and QPS at hybrid Recall@{k} >= {a.target} per "
                                "build method", "config": {"workload": workload_name(a)},
                      "builds": rows}), flush=True)


# ---------------------------------------------------------------- strategies
def strategies_arm(a):
    """The paper's comparison (Sec. 6.2) inside this framework, on one GPU and the c2
    workload: NHQ (composite index, constant weights, attribute-entry seeds) against
    B(1) post-filtering (a proximity graph on vector distance only, searched for k'
    records with random seeds, then the matching ones kept) and B(2) pre-filtering
    (exact top-k among the matching objects, the filter-mode brute force)."""
    import torch

    import paper_2203_13601_gb300 as nhq
    from paper_2203_13601_gb300 import build as B

    B.build()
    nhq.load_library()
    dev = torch.device("cuda", 0)
    w = make_workload(a)
    X, A = torch.from_numpy(w.X).to(dev), torch.from_numpy(w.A).to(dev)
    Qv, QA = torch.from_numpy(w.Qv).to(dev), torch.from_numpy(w.QA).to(dev)
    k = a.k
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    t0 = time.perf_counter()
    ix = nhq.Index.build(X, A, degree=a.R, weights=CONST_W, K=64, knn_dtype=1)
    torch.cuda.synchronize()
    t_nhq = time.perf_counter() - t0
    gt = torch.empty((w.nq, k), dtype=torch.uint32, device=dev)
    ms_pre = timed(lambda: nhq.nhq_brute_force(ix.handle, Qv, QA, k, gt, weights="filter"), 3)
    gt_h = gt.cpu().numpy()
    mult = np.array([1, 256, 65536])[: w.m]
    codes, qcodes = (w.A.astype(np.int64) * mult).sum(1), (w.QA.astype(np.int64) * mult).sum(1)
    uniq, cnt = np.unique(codes, return_counts=True)
    pos = np.minimum(np.searchsorted(uniq, qcodes), len(uniq) - 1)
    P = np.where(uniq[pos] == qcodes, cnt[pos], 0)

    ids, dd, ch = (torch.empty((w.nq, k), dtype=torch.uint32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.float32, device=dev),
                   torch.empty((w.nq, k), dtype=torch.uint8, device=dev))
    nhq_rows = []
    for ef in (16, 24, 32, 48):
        run = lambda ef=ef: nhq.nhq_search(ix.handle, Qv, QA, k, ef, ids, dd, ch, seed=12345,
                                           seed_mode=nhq.SEED_ATTRIBUTE)
        ms = timed(run)
        rec, _ = hybrid_recall(ids.cpu().numpy(), w.A, w.QA, gt_h, P, k)
        nhq_rows.append({"ef": ef, "recall": rec, "ms": ms, "qps": w.nq / ms * 1e3})
    ix.close()

    t0 = time.perf_counter()
    ixl = nhq.Index.build(X, A, degree=a.R, weights=(1.0, 0.0), K=64, knn_dtype=1)
    torch.cuda.synchronize()
    t_l2 = time.perf_counter() - t0
    # entry points of the L2 search: the 32 nearest of a 4,096-object sample (the objects
    # are in random order, so the first rows are a uniform sample); random seeds rarely
    # reach the query's cluster on a graph of exact nearest neighbours
    S = 4096
    ixs = nhq.Index.create(X[:S].contiguous(), A[:S].contiguous(), (1.0, 0.0))
    seeds = torch.empty((w.nq, 32), dtype=torch.uint32, device=dev)
    post_rows = []
    fi = torch.empty((w.nq, k), dtype=torch.uint32, device=dev)
    fd = torch.empty((w.nq, k), dtype=torch.float32, device=dev)
    for kp in (10, 32, 64, 128, 256):
        exact = torch.empty((w.nq, kp), dtype=torch.uint32, device=dev)
        nhq.nhq_brute_force(ixl.handle, Qv, QA, kp, exact)
        ex_h = exact.cpu().numpy()
        for ef in sorted({max(kp, 32), 2 * kp, 4 * kp}):
            if ef > 1024:
                continue
            i2, d2, c2 = (torch.empty((w.nq, kp), dtype=torch.uint32, device=dev),
                          torch.empty((w.nq, kp), dtype=torch.float32, device=dev),
                          torch.empty((w.nq, kp), dtype=torch.uint8, device=dev))

            def run(kp=kp, ef=ef, i2=i2, d2=d2, c2=c2):
                nhq.nhq_brute_force(ixs.handle, Qv, QA, 32, seeds)
                nhq.nhq_search(ixl.handle, Qv, QA, kp, ef, i2, d2, c2, seed=12345,
                               seed_mode=nhq.SEED_GIVEN, seeds=seeds)
                nhq.nhq_postfilter(i2, d2, c2, k, fi, fd)

            ms = timed(run)
            rec, _ = hybrid_recall(fi.cpu().numpy(), w.A, w.QA, gt_h, P, k)
            got = i2.cpu().numpy()
            l2rec = float(np.mean([len(set(x) & set(y)) / kp for x, y in zip(got, ex_h)]))
            post_rows.append({"k_prime": kp, "ef": ef, "recall": rec, "l2_recall": l2rec,
                              "ms": ms, "qps": w.nq / ms * 1e3})
    ixs.close()
    ixl.close()

    # pre-filtering on an attribute partition: the objects grouped by tuple (built before
    # the timed region, like an index), then for each tuple that queries ask for one exact
    # brute force over its objects only
    order = np.argsort(codes, kind="stable")
    starts = np.searchsorted(codes[order], uniq)
    parts = []
    for t in np.unique(qcodes):
        j = int(np.searchsorted(uniq, t))
        if j >= len(uniq) or uniq[j] != t:
            continue  # no object carries this tuple: the query has no answer
        members = order[starts[j]:starts[j] + cnt[j]]
        qi = np.nonzero(qcodes == t)[0]
        mt = torch.from_numpy(members).to(dev)
        sub = nhq.Index.create(X[mt].contiguous(), A[mt].contiguous(), (1.0, 0.0))
        out = torch.empty((len(qi), k), dtype=torch.uint32, device=dev)
        parts.append((sub, Qv[torch.from_numpy(qi).to(dev)].contiguous(),
                      QA[torch.from_numpy(qi).to(dev)].contiguous(), out, members, qi))
    torch.cuda.synchronize()

    def run_parts():
        for sub, qv, qa, out, _, _ in parts:
            nhq.nhq_brute_force(sub.handle, qv, qa, k, out)

    ms_part = timed(run_parts, 3)
    peak, _ = peaks()
    pre_bytes = float(P.sum()) * (4 * w.d + 4)
    pre_ms_bound = pre_bytes / (peak * 1e9) * 1e3
    part_ids = np.full((w.nq, k), 0xFFFFFFFF, np.uint32)
    for sub, _, _, out, members, qi in parts:
        loc = out.cpu().numpy().astype(np.int64)
        glob = np.where(loc == 0xFFFFFFFF, 0xFFFFFFFF, members[np.minimum(loc, len(members) - 1)])
        part_ids[qi] = glob.astype(np.uint32)
        sub.close()
    rec_part, _ = hybrid_recall(part_ids, w.A, w.QA, gt_h, P, k)

    def best(rows):
        ok = [r for r in rows if r["recall"] >= a.target]
        return min(ok, key=lambda r: r["ms"]) if ok else max(rows, key=lambda r: r["recall"])

    line = {
        "metric": f"QPS at hybrid Recall@{k} >= {a.target}: NHQ vs post- and pre-filtering",
        "unit": "queries/s", "n_gpus": 1, "data": "synthetic", "config": {
            "workload": workload_name(a),
            "nhq": "composite index (w_v=1, w_l=10000), attribute-entry seeds",
            "post_filter": "plain L2 graph (w_l=0, same build), seeds = the 32 nearest of a "
                           "4,096-object sample (brute force, timed), search k' records, keep "
                           "the matching ones (nhq_postfilter)",
            "pre_filter": "exact top-k among the matching objects: objects partitioned by "
                          "attribute tuple before timing, one brute force per queried tuple "
                          "over its objects only",
            "pre_filter_scan_all": "filter-mode brute force over all N objects",
            "build_s": {"nhq": t_nhq, "l2_graph": t_l2}},
        "nhq": {"best": best(nhq_rows), "sweep": nhq_rows},
        "post_filter": {"best": best(post_rows), "sweep": post_rows},
        "pre_filter": {"recall": rec_part, "ms": ms_part, "qps": w.nq / ms_part * 1e3,
                       "launches": len(parts)},
        "pre_filter_scan_all": {"recall": 1.0, "ms": ms_pre, "qps": w.nq / ms_pre * 1e3},
        # no pre-filter can do better than reading every matching object's row once per
        # query at the measured HBM bandwidth
        "pre_filter_roofline": {"bytes": pre_bytes, "ms": pre_ms_bound,
                                "qps": w.nq / pre_ms_bound * 1e3, "peak_gbs": peak},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def hybrid_recall(ids, A, QA, gt, P, k):
    """Sec. 6.1 recall: returned ids whose attributes equal the query's, against
    the k nearest matching objects; denominator min(k, |P|); |P| = 0 excluded."""
    ids = ids.astype(np.int64)
    ids[ids == 0xFFFFFFFF] = -1
    ok = ids >= 0
    match = np.zeros_like(ok)
    match[ok] = (A[ids[ok]] == np.repeat(QA, k, axis=0).reshape(len(QA), k, -1)[ok]).all(axis=-1)
    hits = np.zeros(len(ids))
    gt = gt.astype(np.int64)
    for q in range(len(ids)):
        f = set(ids[q][match[q]].tolist())
        g = set(gt[q][gt[q] != 0xFFFFFFFF].tolist())
        hits[q] = len(f & g)
    valid = P > 0
    den = np.minimum(k, P)
    return float(np.mean(hits[valid] / den[valid])), int((~valid).sum())


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        reference_arm(a, rank, world)
        return
    if a.workload == "c4":
        c4_arm(a, rank, world, local)
        return
    if a.workload == "strategies":
        if rank == 0:
            strategies_arm(a)
        return
    if a.workload == "c5":
        if rank == 0:
            c5_arm(a)
        return
    if a.workload == "c3":
        if rank == 0:
            c3_arm(a)
        return
    if a.workload == "curves":
        if rank == 0:
            curves_arm(a)
        return
    if a.workload == "builds":
        if rank == 0:
            builds_arm(a)
        return
    if a.workload == "attrdim":
        if rank == 0:
            attrdim_arm(a)
        return
    if a.workload == "wildcard":
        if rank == 0:
            wildcard_arm(a)
        return

    import torch

    import paper_2203_13601_gb300 as nhq
    from paper_2203_13601_gb300 import build as B

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    nhq.load_library()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    w = make_workload(a)
    t_gen = time.perf_counter() - t0
    X = torch.from_numpy(w.X).to(dev)
    A = torch.from_numpy(w.A).to(dev)
    Qv = torch.from_numpy(w.Qv).to(dev)
    QA = torch.from_numpy(w.QA).to(dev)
    torch.cuda.synchronize()

    t0 = time.perf_counter()
    ix = nhq.Index.build(X, A, degree=a.R, weights=CONST_W, K=64, knn_dtype=a.knn_dtype)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0

    # hybrid ground truth (Sec. 6.1) with the brute force in filter mode, and |P|
    gt = torch.empty((w.nq, a.k), dtype=torch.uint32, device=dev)
    t0 = time.perf_counter()
    nhq.nhq_brute_force(ix.handle, Qv, QA, a.k, gt, weights="filter")
    torch.cuda.synchronize()
    t_gt = time.perf_counter() - t0
    gt_h = gt.cpu().numpy()
    codes = (w.A.astype(np.int64) * np.array([1, 256, 65536])[: w.m]).sum(1)
    qcodes = (w.QA.astype(np.int64) * np.array([1, 256, 65536])[: w.m]).sum(1)
    uniq, cnt = np.unique(codes, return_counts=True)
    pos = np.searchsorted(uniq, qcodes)
    P = np.where((pos < len(uniq)) & (uniq[np.minimum(pos, len(uniq) - 1)] == qcodes),
                 cnt[np.minimum(pos, len(uniq) - 1)], 0)

    ids = torch.empty((w.nq, a.k), dtype=torch.uint32, device=dev)
    dists = torch.empty((w.nq, a.k), dtype=torch.float32, device=dev)
    chi = torch.empty((w.nq, a.k), dtype=torch.uint8, device=dev)
    ndc = torch.empty(w.nq, dtype=torch.int32, device=dev)
    exps = torch.empty(w.nq, dtype=torch.int32, device=dev)

    # the learned parts chosen by the sweep below (none until then)
    sel = {"model": None, "tau": 0.5, "stop_min": 4, "stop_every": 2, "entry": None}

    def seed_kw():
        if sel["entry"] is not None:
            return dict(seed_mode=nhq.SEED_CELL_LEARNED, entry_model=sel["entry"],
                        entry_cells=a.entry_T)
        return dict(seed_mode=a.seed_mode)

    def run(ef, h, vec, diag=False):
        # the reduced-precision copies are re-ranked in f32 (vec 2 = fp8 needs it; bf16 is
        # exact on this integer data and runs without)
        nhq.nhq_search(ix.handle, Qv, QA, a.k, ef, ids, dists, chi,
                       ndc=ndc if diag else None, expansions=exps if diag else None,
                       h=h, seed=12345, vec_dtype=vec, rerank=int(vec == nhq.VEC_FP8E4M3),
                       stop_model=sel["model"], stop_threshold=sel["tau"],
                       stop_min=sel["stop_min"], stop_every=sel["stop_every"], stream=stream,
                       warps_per_query=a.wpq, **seed_kw())

    def time_once(ef, h, vec, reps=2):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        run(ef, h, vec)
        ev0.record(stream)
        for _ in range(reps):
            run(ef, h, vec)
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / reps

    # sweep: smallest ef reaching the target per (h, scoring copy); keep the fastest
    sweep = []
    choices = []
    vecs = [nhq.VEC_F32, nhq.VEC_BF16, nhq.VEC_FP8E4M3]
    if a.fixed:
        ef, h, vec = (int(x) for x in a.fixed.split(","))
        cand_list = [(ef, h, vec)]
    else:
        cand_list = None
    plain = None
    for vec in vecs:
        for h in [int(x) for x in a.hs.split(",")]:
            found = None
            efs = [int(x) for x in a.efs.split(",") if int(x) >= a.k]
            if cand_list:
                if (vec, h) != (cand_list[0][2], cand_list[0][1]):
                    continue
                efs = [cand_list[0][0]]
            for ef in efs:
                run(ef, h, vec, diag=True)
                torch.cuda.synchronize()
                rec, excl = hybrid_recall(ids.cpu().numpy(), w.A, w.QA, gt_h, P, a.k)
                ms = time_once(ef, h, vec)
                sweep.append({"ef": ef, "h": h, "vec": VEC_NAMES[vec], "recall": rec,
                              "ms": ms, "mean_expansions": float(exps.float().mean().item())})
                if found is None and (rec >= a.target or cand_list):
                    found = (ef, h, vec, rec, ms)
                if rec >= a.target2 or cand_list:
                    break
            if found:
                choices.append(found)
                if vec == nhq.VEC_F32 and (plain is None or found[4] < plain[4]):
                    plain = found
    # learned early stop: traces of training queries (same mixture, independent
    # stream), the MLP trained on the GPU, then a sweep of (ef, threshold)
    learned = None
    stop_model = None
    if not a.no_learned and not a.fixed:
        t0 = time.perf_counter()
        wtr = make_workload(a, query_stream=1)
        Qtr = torch.from_numpy(wtr.Qv).to(dev)
        QAtr = torch.from_numpy(wtr.QA).to(dev)
        cap = 40 * wtr.nq
        feats = torch.empty((cap, nhq.MLP_INPUTS), dtype=torch.float32, device=dev)
        labels = torch.empty(cap, dtype=torch.uint8, device=dev)
        tq = torch.empty(cap, dtype=torch.int32, device=dev)
        ef_tr = max(int(x) for x in a.learned_efs.split(","))
        ntr = nhq.nhq_search_trace(ix.handle, Qtr, QAtr, a.k, ef_tr, feats, labels, tq,
                                   stop_min=4, stop_every=2, seed_mode=a.seed_mode)
        perm = torch.randperm(ntr, generator=torch.Generator().manual_seed(0)).to(dev)
        F = feats[:ntr][perm].contiguous()
        Y = labels[:ntr][perm].to(torch.float32).contiguous()
        init = np.random.default_rng(9).standard_normal(nhq.MLP_PARAMS).astype(np.float32) * 0.1
        init[-1] = 0.0
        stop_model = torch.from_numpy(init).to(dev)
        nhq.nhq_mlp_train(stop_model, F, Y, epochs=8, batch=2048, lr=2e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        del feats, labels, tq, F, Y
        # the learned entry point: cells and the entry model, trained on the cells of the
        # plain search's answers for another set of training queries
        E = a.cells if a.cells > 0 else 256
        wtr_e = synth_c2_queries(a, a.train_q, 2)
        entry_model, t_entry, n_entry = train_entry(nhq, ix, w, wtr_e, E, a.k, dev, epochs=20)
        lsweep = []
        schedules = [(4, 2), (8, 4)]
        for lef in [int(x) for x in a.learned_efs.split(",") if int(x) >= a.k]:
            combos = [(None, None, True)]  # the entry model alone
            for (smin, severy) in schedules:
                for tau in [float(x) for x in a.taus.split(",")]:
                    combos += [((smin, severy), tau, False), ((smin, severy), tau, True)]
            for sched, tau, use_entry in combos:
                def run_l(lef=lef, tau=tau, sched=sched, use_entry=use_entry, diag=False):
                    kw = dict(seed_mode=a.seed_mode)
                    if use_entry:
                        kw = dict(seed_mode=nhq.SEED_CELL_LEARNED, entry_model=entry_model,
                                  entry_cells=a.entry_T)
                    nhq.nhq_search(ix.handle, Qv, QA, a.k, lef, ids, dists, chi, h=1,
                                   expansions=exps if diag else None, seed=12345,
                                   stop_model=stop_model if sched else None,
                                   stop_threshold=tau if sched else 0.5,
                                   stop_min=sched[0] if sched else 4,
                                   stop_every=sched[1] if sched else 2, stream=stream, **kw)
                run_l(diag=True)
                torch.cuda.synchronize()
                rec, _ = hybrid_recall(ids.cpu().numpy(), w.A, w.QA, gt_h, P, a.k)
                mexp = float(exps.float().mean().item())
                ev0, ev1 = (torch.cuda.Event(enable_timing=True),
                            torch.cuda.Event(enable_timing=True))
                run_l()
                ev0.record(stream)
                run_l()
                run_l()
                ev1.record(stream)
                ev1.synchronize()
                ms = ev0.elapsed_time(ev1) / 2
                lsweep.append({"ef": lef, "tau": tau, "recall": rec, "ms": ms,
                               "mean_expansions": mexp, "entry": use_entry,
                               "stop": ({"stop_min": sched[0], "stop_every": sched[1]}
                                        if sched else None)})
        ok = [x for x in lsweep if x["recall"] >= a.target]
        if ok:
            learned = min(ok, key=lambda x: x["ms"])
        ok2 = [x for x in lsweep if x["recall"] >= a.target2]
        plain2 = [x for x in sweep if x["recall"] >= a.target2 and x["vec"] == "f32"]
        learned_info = {"traces": int(ntr), "train_s": t_train, "sweep": lsweep,
                        "entry": {"cells": E, "cells_per_query": a.entry_T,
                                  "train_s": t_entry, "traces": n_entry},
                        "chosen": learned,
                        "at_target2": {
                            "target": a.target2,
                            "learned": min(ok2, key=lambda x: x["ms"]) if ok2 else None,
                            "plain_f32": min(plain2, key=lambda x: x["ms"]) if plain2 else None}}

    if not choices:
        raise SystemExit(f"no setting reached hybrid Recall@{a.k} >= {a.target}: {sweep}")
    best = min(choices, key=lambda c: c[4])
    ef, h, vec, rec, _ = best
    # a learned form is taken only when it beats the plain choice by more than the sweep's
    # timing noise (2 %, three launches per setting)
    use_learned = learned is not None and learned["ms"] < 0.98 * best[4]
    tau = 0.5
    if use_learned:
        ef, h, vec, rec = learned["ef"], 1, nhq.VEC_F32, learned["recall"]
        if learned["stop"] is not None:
            tau = learned["tau"]
            sel.update(model=stop_model, tau=tau, stop_min=learned["stop"]["stop_min"],
                       stop_every=learned["stop"]["stop_every"])
        if learned["entry"]:
            sel["entry"] = entry_model
    # diagnostics at the chosen setting: NDC and expansions for the algorithmic bytes
    run(ef, h, vec, diag=True)
    torch.cuda.synchronize()
    ndc_h, exp_h = ndc.cpu().numpy().astype(np.float64), exps.cpu().numpy().astype(np.float64)
    row_bytes = {nhq.VEC_F32: 4, nhq.VEC_BF16: 2, nhq.VEC_FP8E4M3: 1}[vec] * a.d
    bytes_per_query = ndc_h * (row_bytes + 4) + exp_h * a.R * 4 + a.d * 4 + a.k * 9
    if vec == nhq.VEC_FP8E4M3:  # the f32 re-rank reads every pool member's f32 row once
        bytes_per_query = bytes_per_query + ef * 4 * a.d
    alg_bytes = float(bytes_per_query.sum())

    # timed region: K steps of one search over the whole batch, device-resident inputs
    for _ in range(max(3, a.warmup)):
        run(ef, h, vec)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(a.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for s0, s1 in evs:
        s0.record(stream)
        run(ef, h, vec)
        s1.record(stream)
    e_end.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    total_ms = e_start.elapsed_time(e_end)
    clk = clocks.stop()
    step_ms = [s0.elapsed_time(s1) for s0, s1 in evs]
    total_ms = max_over_ranks(total_ms, dist, dev)
    ms_per_step = total_ms / a.steps
    qps = weak_scaling_value(w.nq, a.steps, world, total_ms)
    launch_ms = float(np.mean(step_ms))
    achieved = alg_bytes / (launch_ms / 1000.0) / 1e9
    peak, peak_kind = peaks()

    # end to end through the public call with pinned host buffers
    Qh = torch.from_numpy(w.Qv).pin_memory()
    QAh = torch.from_numpy(w.QA).pin_memory()
    ids_h = torch.empty((w.nq, a.k), dtype=torch.uint32).pin_memory()
    d_h = torch.empty((w.nq, a.k), dtype=torch.float32).pin_memory()
    c_h = torch.empty((w.nq, a.k), dtype=torch.uint8).pin_memory()

    def run_host():
        nhq.nhq_search(ix.handle, Qh, QAh, a.k, ef, ids_h, d_h, c_h, h=h, seed=12345,
                       vec_dtype=vec, rerank=int(vec == nhq.VEC_FP8E4M3),
                       seed_mode=a.seed_mode, stop_model=sel["model"],
                       stop_threshold=sel["tau"], stop_min=4, stop_every=2, stream=stream,
                       warps_per_query=a.wpq)

    for _ in range(max(3, a.warmup)):
        run_host()
    e2e_steps = max(3, min(a.steps, 20))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        run_host()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_rec, _ = hybrid_recall(ids_h.numpy(), w.A, w.QA, gt_h, P, a.k)
    h2d = w.nq * a.d * 4 + w.nq * w.m
    d2h = w.nq * a.k * (4 + 4 + 1)

    line = {
        "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": world,
        "steps": a.steps, "warmup": max(3, a.warmup), "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": VEC_NAMES[vec], "data": "synthetic",
        "config": {"workload": workload_name(a), "ef": ef, "h": h,
                   "seed_set": ("learned entry cells" if sel["entry"] is not None else
                                ["random (Sec. 3.2)", "attribute entry"][a.seed_mode]),
                   "scoring_copy": VEC_NAMES[vec] + (" + f32 re-rank" if vec == 2 else ""),
                   "learned_stop": ({"threshold": tau, "stop_min": sel["stop_min"],
                                     "stop_every": sel["stop_every"]}
                                    if sel["model"] is not None else None),
                   "recall": rec,
                   "recall_kind": "hybrid Recall@10 vs filter-mode brute force",
                   "l2": "inputs larger than L2 (vectors 512 MB + adjacency 256 MB)",
                   "build_s": t_build, "build_candidates": ["f32 SIMT", "bf16 tensor cores"][a.knn_dtype],
                   "gen_s": t_gen, "ground_truth_s": t_gt,
                   "queries_with_no_match": int((P == 0).sum())},
        "plain_f32": ({"ef": plain[0], "h": plain[1], "recall": plain[3],
                       "qps": w.nq / (plain[4] / 1000.0)} if plain else None),
        "sweep": sweep,
        "learned": learned_info if (not a.no_learned and not a.fixed) else None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": recorded_traffic(ef, h, vec, a.seed_mode, a.n, a.nq,
                                                 use_learned),
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "launch_ms": launch_ms, "mean_ndc": float(ndc_h.mean()),
                     "mean_expansions": float(exp_h.mean()),
                     "step_ms": {"min": float(np.min(step_ms)),
                                 "median": float(np.median(step_ms)),
                                 "max": float(np.max(step_ms))}},
        "e2e": {"value": w.nq / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "recall": e2e_rec},
        # per step: the seed pre-pass and ordering (attribute seeds: 2 kernels; learned entry:
        # fp16 model copy, two dense layers, seeds, ordering), the stop model's fp16 copy,
        # the search kernel
        "gpu_launches": a.steps * ((5 if sel["entry"] is not None else
                                    2 if a.seed_mode in (1, 3) else 0) +
                                   (1 if sel["model"] is not None else 0) + 1),
        "clocks": clk,
    }
    if rank == 0:
        line["brute_force"] = brute_force_roofline(nhq, ix, Qv, QA, a.k, a.n, a.d, dev, stream)
    if rank == 0 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, a, a.cpu_sample)
        line["cpu_baseline"].pop("seconds", None)
        if not use_learned:  # the oracle has no learned stop
            g32 = torch.empty((w.N, a.R), dtype=torch.uint32, device=dev)
            nhq.nhq_index_get_graph(ix.handle, g32)
            nbr = g32.cpu().numpy().astype(np.int64)
            nbr[nbr == 0xFFFFFFFF] = -1
            del g32
            run(ef, h, vec)
            torch.cuda.synchronize()
            line["cpu_baseline"]["search"] = cpu_search_baseline(
                w, a, nbr, ef, a.seed_mode, ids.cpu().numpy(), 4 * a.cpu_sample, h, vec)
    ix.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
