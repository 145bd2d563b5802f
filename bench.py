#!/usr/bin/env python
"""Benchmark of the LSH query-workload path (qwLSH's method) on GB300.

One step = one call answering the whole synthetic query workload (project the
queries, collision counting over all levels, candidate selection, distances,
top-k) against an index already resident in HBM.  The default workload is the
largest single-GPU one: 10,000,000 x 128 float32 points (Gaussian mixture of
10,000 clusters), 64 projections, w = 4, 100,000 queries with mixed difficulty
(noise sigma 0.05, 0.5 and 2.0 in equal thirds), k = 10.

Two configurations of the same call are timed, with identical results: the
plain path (level path, queries in the given order, collision counting from
level 0, FP32 distances, host-driven loop) and the chosen path (the settings
qw_autotune picks on training queries of the same workload among the counting
paths, batch sizes, graph mode, workload order, learned first levels, the BF16
distance pre-filter and the persisting-L2 split).  ``value`` is the chosen
path's; the plain path's figures are reported beside it, with the roofline of
the dominant kernels, the end-to-end rate from pinned host memory, and the
CPU oracle timed on all host threads.  The start model is trained before the
timed region on queries drawn from the same workload.

Prints one JSON line.  ``--impl reference`` times the CPU oracle on a bounded
sample of the same workload instead; ``--l2-sweep`` adds the chosen path under
the paper's cache splits.  Under torchrun (``--gpus N``) every rank
answers its own copy of the workload against its own replica of the index
(the path has no exchange step); the timed region is bracketed by barriers and
the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Operating points (v, l) meeting recall >= 0.9 and ratio <= 1.05, from sweeps
# of v and l on the GPU (recall on 200 seeded queries against exact k-NN; l = 0
# derives l from Eq. 1): the paper's v = 100 gives recall 0.35 on mix1m_d128,
# 0.24 on mix4m_d512 and 0.34 on mix10m_d128; v = 1000 gives 0.9997 and 0.997
# on the latter two.  zipf1m_d256 cannot reach 0.9 within k + v <= 4096 (its
# largest clusters hold most points at nearly equal distances): 0.56 at
# v = 1000, 0.71 at v = 4086 and l = 32, the best measured, which it uses.
OPERATING_POINTS = {"mix1m_d128": (700, 43), "mix4m_d512": (1000, 0), "mix10m_d128": (1000, 0),
                    "zipf1m_d256": (4086, 32)}
# QALSH's query-aware buckets (--family qalsh) with the bucket width of the
# paper's experiments (Section 6: w = 2.719); l = 0 derives l from QALSH's
# collision probability.
QALSH_W = 2.719
QALSH_OPERATING_POINTS = {"mix1m_d128": (700, 0)}

METRIC = "workload queries/sec at recall>=0.9, ratio<=1.05 (plain vs chosen); HBM roofline %"
UNIT = "queries/s"
L2_BYTES = 129 * 1024 * 1024


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1)
    # default: about one second of timed GPU steps (so that clocks are sampled
    # while they run); 5 steps of the CPU reference arm
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--no-plain", action="store_true",
                   help="skip the plain path (profiler captures of the chosen path only)")
    p.add_argument("--plain-steps", type=int, default=2,
                   help="timed steps of the plain path (at most --steps)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="mix10m_d128")
    p.add_argument("--family", choices=["e2lsh", "qalsh"], default="e2lsh",
                   help="hash family: Section 3's bucketed h(v) = floor((a.v + b) / w), or "
                        "QALSH's query-centred intervals (level path, w = 2.719)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--quality-sample", type=int, default=1000,
                   help="queries checked against exact k-NN for recall / ratio")
    p.add_argument("--cpu-sample", type=int, default=2,
                   help="queries per host thread the CPU oracle answers (cpu_baseline entry; "
                        "each step of the reference arm)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--queries", type=int, default=0,
                   help="override the workload's query count (smaller cases for profiling)")
    p.add_argument("--n", type=int, default=0,
                   help="override the workload's point count (smaller cases for profiling)")
    p.add_argument("--clusters", type=int, default=0,
                   help="override the workload's cluster count (with --n)")
    p.add_argument("--batch", type=int, default=0, help="queries per pass (0 = library choice)")
    p.add_argument("--path", choices=["auto", "cluster", "levels", "bitmap"], default="auto",
                   help="execution path of the query loop (identical results)")
    p.add_argument("--order", choices=["auto", "signature", "given"], default="auto",
                   help="workload order: grouped by bucket signature, or as given")
    p.add_argument("--rerank", choices=["fp32", "bf16", "bf16_tc"], default="bf16",
                   help="distance arithmetic of the chosen path (identical results)")
    p.add_argument("--rerank-rows", type=int, choices=[0, 2, 4, 8], default=0,
                   help="candidate rows a warp of the distance kernels takes at a time "
                        "(0 = library choice; with --no-tune)")
    p.add_argument("--start", choices=["plain", "learned"], default="learned",
                   help="first level of the chosen path (identical results)")
    p.add_argument("--train-queries", type=int, default=20_000,
                   help="queries the start model is trained and the autotuner run on (untimed)")
    p.add_argument("--no-tune", action="store_true",
                   help="chosen path from --path/--order/--rerank/--start/--graph instead of "
                        "the autotuner")
    p.add_argument("--no-bitmaps", action="store_true",
                   help="build the index without the level bitmaps of the bitmap path")
    p.add_argument("--host-bitmaps", action="store_true",
                   help="keep the level bitmaps in pinned host memory, read over NVLink-C2C "
                        "(an index larger than the GPU's memory)")
    p.add_argument("--loads", choices=["tma", "direct", "fused"], default="direct",
                   help="with --no-tune and --path bitmap: how the bitmap kernel reads bitmaps")
    p.add_argument("--graph", action="store_true",
                   help="with --no-tune: run the level loop as a CUDA graph")
    p.add_argument("--l2", default="off",
                   help="with --no-tune: persisting-L2 split of the chosen path (off, model, or "
                        "the index window's permille of the set-aside)")
    p.add_argument("--l2-sweep", action="store_true",
                   help="also time the chosen path under the paper's cache splits (index share "
                        "1, 10, ..., 90, 99 %% of the persisting-L2 set-aside, off, cost model)")
    p.add_argument("--sweep-steps", type=int, default=20)
    p.add_argument("--cost-sweep", action="store_true",
                   help="instead of the benchmark line: the persisting-L2 index-window fraction "
                        "swept over a grid of (n, d) workloads, and a fit of the fastest "
                        "fraction as a function of (n, d) (one JSON line)")
    p.add_argument("--cost-grid", default="250000,500000,1000000,2000000:32,128,512",
                   help="n values : d values of the cost sweep")
    p.add_argument("--v", type=int, default=-1,
                   help="allowed false positives (-1 = the workload's operating point)")
    p.add_argument("--l", type=int, default=-1,
                   help="collision threshold (0 = derived from Eq. 1, -1 = operating point)")
    return p.parse_args(argv)


def size_overrides(args) -> dict:
    """make_workload keyword arguments of --n / --clusters."""
    kw = {}
    if args.n:
        kw["n"] = args.n
    if args.clusters:
        kw["n_clusters"] = args.clusters
    return kw


def operating_point(args, spec):
    """(v, l) for this run: explicit flags, else the workload's operating
    point, else the spec's v with l derived from Eq. 1 (l = 0)."""
    points = QALSH_OPERATING_POINTS if args.family == "qalsh" else OPERATING_POINTS
    dv, dl = points.get(args.workload, (spec.v, 0))
    v = args.v if args.v >= 0 else dv
    l = args.l if args.l >= 0 else dl
    return v, l


_T0 = time.perf_counter()


def log(msg: str):
    """Progress of the run on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


# ---------------------------------------------------------------- ranks
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int) -> float:
    """Largest value over all ranks (the slowest rank's time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clock_csv(out)


def parse_clock_csv(text: str):
    """Summary of nvidia-smi samples: median SM clock, max clock, and every
    throttle reason seen active."""
    rows = [r for r in csv.reader(io.StringIO(text)) if len(r) >= 9]
    if not rows:
        return None

    def num(x):
        try:
            return float(x)
        except ValueError:
            return None

    sm = [v for v in (num(r[1]) for r in rows) if v is not None]
    mx = [v for v in (num(r[2]) for r in rows) if v is not None]
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    reasons = sorted({nm for r in rows for nm, v in zip(names, r[5:9])
                      if v.strip().lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


def gpu_uuid(torch):
    try:
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


KERNEL_SOURCES = {
    "level_kernel": ("qw_query.cu", "qw_count.cuh", "qw_dir.cuh", "qw_internal.cuh"),
    "level_kernel_qalsh": ("qw_query.cu", "qw_count.cuh", "qw_internal.cuh", "qw_qalsh.cu"),
    "bm_filter_count": ("qw_bitmap.cu", "qw_dir.cuh", "qw_scan.cuh", "qw_internal.cuh"),
    "bm_fused_kernel": ("qw_bitmap.cu", "qw_dir.cuh", "qw_scan.cuh", "qw_internal.cuh"),
    "bm_level_tma_kernel": ("qw_bitmap.cu", "qw_tma.cuh", "qw_internal.cuh"),
    "cluster_query_kernel": ("qw_cluster.cu", "qw_count.cuh", "qw_internal.cuh"),
    "rerank_kernel": ("qw_rerank.cu", "qw_scan.cuh", "qw_internal.cuh"),
    "rerank_bf16_kernel": ("qw_rerank.cu", "qw_scan.cuh", "qw_internal.cuh"),
    "rerank_tc_kernel": ("qw_rerank.cu", "qw_scan.cuh", "qw_tc.cuh", "qw_internal.cuh"),
}


def kernel_source_sha(kernel: str) -> str:
    """sha256 (16 hex digits) of the source files a kernel is built from."""
    src = os.path.join(ROOT, "paper_1907_11803_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, ()):
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes (read + write) per launch of a kernel class from the
    committed ncu summary profiles/traffic.txt, if that was taken on the
    current source of the kernel (lines: kernel workload source-sha
    bytes-per-launch)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    sha = kernel_source_sha(kernel)
    try:
        with open(path) as fh:
            for line in fh:
                parts = line.split()
                if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel \
                        and parts[1] == workload and parts[2] == sha:
                    return float(parts[3])
    except OSError:
        pass
    return None


# ---------------------------------------------------------------- quality
def exact_knn_gpu(X, Qs, k):
    """Exact k-NN of a query sample in float64 on the GPU (measurement only)."""
    import torch
    Xd = X.double()
    xn = (Xd * Xd).sum(1)
    ids, dists = [], []
    for s in range(0, Qs.shape[0], 32):
        q = Qs[s:s + 32].double()
        d2 = xn[None, :] - 2.0 * (q @ Xd.T) + (q * q).sum(1)[:, None]
        d2.clamp_(min=0)
        v, i = torch.topk(d2, k, dim=1, largest=False, sorted=True)
        ids.append(i)
        dists.append(v.sqrt())
    del Xd
    return torch.cat(ids), torch.cat(dists)


def recall_ratio(ids, dists, tids, tdists):
    import torch
    k = ids.shape[1]
    hit = torch.zeros(ids.shape[0], dtype=torch.float64, device=ids.device)
    for j in range(k):
        hit += (tids == ids[:, j:j + 1]).any(dim=1).double()
    recall = float((hit / k).mean())
    ok = (ids >= 0) & (tdists > 0)
    ratio = float((dists.double()[ok] / tdists[ok]).mean()) if bool(ok.any()) else float("nan")
    return recall, ratio


# ---------------------------------------------------------------- CPU oracle leg
def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_query_threads(orc, wl, idx, Qs, HQ, *, k, v, l, c, threads):
    """The oracle's query procedure over Qs, the queries split into `threads`
    contiguous slices answered at the same time (the oracle is plain C called
    through ctypes, which releases the interpreter lock; it keeps no global
    state).  Returns the wall time in seconds."""
    import concurrent.futures as cf

    import numpy as np
    parts = [p for p in np.array_split(np.arange(Qs.shape[0]), threads) if p.size]

    def one(p):
        orc.query(wl.X, idx, Qs[p], HQ[p], k=k, v=v, l=l, c=c, want_candidates=False,
                  want_stats=False)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=len(parts)) as ex:
        list(ex.map(one, parts))
    return time.perf_counter() - t0


def oracle_hash_threads(orc, V, A, b, w, threads):
    """The oracle's hash of the rows of V, the rows split into `threads`
    contiguous slices hashed at the same time (each row's bucket ids depend on
    that row alone)."""
    import concurrent.futures as cf

    import numpy as np
    parts = [p for p in np.array_split(np.arange(V.shape[0]), max(1, threads)) if p.size]
    with cf.ThreadPoolExecutor(max_workers=len(parts)) as ex:
        Hs = list(ex.map(lambda p: orc.hash(V[p[0]:p[-1] + 1], A, b, w), parts))
    return np.concatenate(Hs) if Hs else np.empty((0, A.shape[0]), np.int32)


def oracle_index(wl, threads):
    """The oracle and its index of the workload's data (anchors and spans; the
    query procedure recounts collisions from the bucket-id rows)."""
    import oracle
    orc = oracle.get()
    H = oracle_hash_threads(orc, wl.X, wl.A, wl.b, wl.spec.w, threads)
    return orc, orc.build_index(H, sorted_arrays=False)


def oracle_qalsh_index(wl, threads):
    """The oracle and the FP64 projections of the workload's data (QALSH)."""
    import concurrent.futures as cf

    import numpy as np

    import oracle
    orc = oracle.get()
    parts = [p for p in np.array_split(np.arange(wl.X.shape[0]), max(1, threads)) if p.size]
    with cf.ThreadPoolExecutor(max_workers=len(parts)) as ex:
        Ps = list(ex.map(lambda p: orc.project(wl.X[p[0]:p[-1] + 1], wl.A), parts))
    return orc, np.concatenate(Ps)


def oracle_qalsh_threads(orc, wl, P, Qs, *, w, k, v, l, c, threads):
    """The oracle's QALSH query procedure over Qs (projections included), the
    queries split into `threads` slices answered at the same time.  Returns
    the wall time in seconds."""
    import concurrent.futures as cf

    import numpy as np
    parts = [p for p in np.array_split(np.arange(Qs.shape[0]), threads) if p.size]

    def one(p):
        PQ = orc.project(Qs[p], wl.A)
        orc.qalsh_query(wl.X, P, Qs[p], PQ, w=w, k=k, v=v, l=l, c=c)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=len(parts)) as ex:
        list(ex.map(one, parts))
    return time.perf_counter() - t0


def oracle_qalsh_sample(wl, w, l, n_queries, seed=1, v=None, threads=1, built=None):
    """oracle_sample for QALSH's query-aware buckets."""
    import numpy as np
    s = wl.spec
    orc, P = built if built is not None else oracle_qalsh_index(wl, threads)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(s.nq, size=min(n_queries, s.nq), replace=False))
    dt = oracle_qalsh_threads(orc, wl, P, wl.Q[pick], w=w, k=s.k, v=s.v if v is None else v,
                              l=l, c=s.c, threads=threads)
    return len(pick) / dt, dt, len(pick), (orc, P)


def oracle_sample(wl, l, n_queries, seed=1, v=None, threads=1, built=None):
    """Time the oracle's query procedure on a seeded sample of the workload's
    queries (the index build is excluded, as on the GPU) on `threads` host
    cores.  Returns (queries/s, seconds, sample size, (oracle, its index))."""
    import numpy as np
    s = wl.spec
    orc, idx = built if built is not None else oracle_index(wl, threads)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(s.nq, size=min(n_queries, s.nq), replace=False))
    Qs = wl.Q[pick]
    HQ = orc.hash(Qs, wl.A, wl.b, s.w)
    dt = oracle_query_threads(orc, wl, idx, Qs, HQ, k=s.k, v=s.v if v is None else v, l=l,
                              c=s.c, threads=threads)
    return len(pick) / dt, dt, len(pick), (orc, idx)


# ---------------------------------------------------------------- our arm
def train_start_model(qw, torch, index, Qt, k, args):
    """Train the first-level model on earlier queries of the same workload
    (labels: the level each one stops at on the plain path).  Untimed."""
    t0 = time.perf_counter()
    _, _, st = index.query(Qt, k, stats=True, start="plain")
    labels = (st[:, 0] - 1).clamp(0, 15).to(torch.int32).contiguous()
    F = index.features(Qt)
    mlp = qw.Mlp(F.shape[1], 256, 16)
    mlp.set_params(qw.mlp_init(F.shape[1], 256, 16, seed=args.seed + 5))
    loss = mlp.train(F, labels, epochs=20, batch=512, lr=1e-3)
    acc = float((mlp.predict(F).argmax(1) == labels).float().mean())
    index.set_start_model(mlp, eps=0.02)
    return mlp, {"train_queries": int(Qt.shape[0]), "epochs": 20, "final_loss": round(loss, 4),
                 "train_accuracy": round(acc, 4), "eps": 0.02,
                 "seconds": round(time.perf_counter() - t0, 2)}


def run_ours(args):
    import numpy as np
    import torch

    import paper_1907_11803_gb300 as qw
    import workloads

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    nq = args.queries or None
    # the timed queries and, from a separate stream, the training queries of
    # the start model and the autotuner (same data, cluster pool and noise mix)
    wl = workloads.make_workload(args.workload, seed=args.seed, nq=nq,
                                 n_train=args.train_queries, **size_overrides(args))
    s = wl.spec
    if world > 1 and rank > 0:
        # each rank answers its own seeded query workload against the same data
        wl.Q, _ = workloads.make_queries(
            wl.X, wl.labels, s.nq, np.random.default_rng(args.seed + 1000 * rank),
            n_clusters=s.n_clusters, query_clusters=s.query_clusters, zipf=s.zipf,
            noise=s.query_noise, pool=wl.extra["query_pool"])
    log(f"workload {s.name}: {s.n} x {s.d}, {s.nq} queries, {args.train_queries} training "
        f"queries drawn")
    X = torch.from_numpy(wl.X).to(dev)
    A = torch.from_numpy(wl.A).to(dev)
    b = torch.from_numpy(wl.b).to(dev)
    Q = torch.from_numpy(wl.Q).to(dev)
    v_used, l_arg = operating_point(args, s)
    qalsh = args.family == "qalsh"
    w_used = QALSH_W if qalsh else s.w
    if qalsh:
        # the query-aware family runs on the level path from level 0
        args.start = "plain"
        args.no_bitmaps = True
    index = qw.Index(X, A, b, w=w_used, c=s.c, v=v_used, l=l_arg,
                     shadow_bf16=args.rerank in ("bf16", "bf16_tc"), bitmaps=not args.no_bitmaps,
                     host_bitmaps=args.host_bitmaps, family=args.family)
    ids = torch.empty((s.nq, s.k), dtype=torch.int64, device=dev)
    dists = torch.empty((s.nq, s.k), dtype=torch.float32, device=dev)
    # the library's calls run on a created stream (persisting-L2 windows are
    # stream attributes; the legacy default stream takes none)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    plain_kw = dict(batch=args.batch, path="levels", order="given", rerank="fp32",
                    start="plain", graph=False)
    l2_arg = None if args.l2 == "off" else ("model" if args.l2 == "model" else int(args.l2))
    chosen_kw = dict(batch=args.batch, path=args.path, order=args.order, rerank=args.rerank,
                     start=args.start, graph=args.graph, loads=args.loads, l2=l2_arg)
    if args.rerank_rows:
        chosen_kw["rerank_rows"] = args.rerank_rows
    mlp = None
    train_info = None
    log(f"index built: {index.info.device_bytes / 1e9:.2f} GB on the device, "
        f"l = {index.l}")
    Qt = torch.from_numpy(wl.Q_train).to(dev)
    if args.start == "learned":
        mlp, train_info = train_start_model(qw, torch, index, Qt, s.k, args)
        log(f"start model trained: {train_info}")
        if args.no_tune and chosen_kw["path"] in ("auto", "cluster"):
            chosen_kw["path"] = "levels"  # learned first levels need a level loop
    tune = None
    if not args.no_tune:
        # settings from the autotuner, timed on earlier queries of the same workload
        t0 = time.perf_counter()
        chosen_kw, trials = index.autotune(Qt[:s.nq], s.k, reps=1)
        tune = {"seconds": round(time.perf_counter() - t0, 2), "queries": int(min(s.nq, Qt.shape[0])),
                "trials": [dict(t, ms=round(ms, 3)) for t, ms in trials]}
        log(f"autotuned in {tune['seconds']} s: {chosen_kw}")

    def timed(kw, steps, warmup=None, profiled=True):
        """`warmup` untimed steps, then `steps` timed ones bracketed by a
        barrier and a synchronize (CUDA events on the library's stream); the
        timed steps run uninstrumented.  With `profiled`, the same number of
        steps is then run again in profile mode (every launch timed by CUDA
        events on the stream) for the per-kernel breakdown.  Returns (ms, max
        over ranks, profile counters of the timed steps, of the profiled)."""
        for _ in range(args.warmup if warmup is None else warmup):
            index.query(Q, s.k, out=(ids, dists), **kw)
        torch.cuda.synchronize()
        index.profile(reset=True)
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            index.query(Q, s.k, out=(ids, dists), **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = e0.elapsed_time(e1)
        counted = index.profile(reset=True)
        prof = None
        if profiled:
            # the level loop driven from the host, so that every kernel class
            # (bucket numbers, filter + count, decide, ...) is timed on its own;
            # the kernels are those of the timed steps
            pkw = dict(kw, graph=False)
            for _ in range(steps):
                index.query(Q, s.k, out=(ids, dists), profile=True, **pkw)
            torch.cuda.synchronize()
            prof = index.profile(reset=True)
        return ms, max_over_ranks(ms, world), counted, prof

    # the plain path first: its results are the reference for the chosen one.
    # Its first call (statistics, every launch timed) is its first warm-up step
    # and gives its kernel breakdown; one more warm-up step follows (a plain
    # step over the large workloads takes tens of seconds).
    index.profile(reset=True)
    if args.no_plain:
        _, _, st = index.query(Q, s.k, stats=True, **chosen_kw)
    else:
        _, _, st = index.query(Q, s.k, stats=True, profile=True, **plain_kw)
    torch.cuda.synchronize()
    p_prof = index.profile(reset=True)
    st = st.cpu().numpy()
    if not args.no_plain:
        p_steps = max(1, min(args.steps, args.plain_steps))
        p_ms, p_ms_max, _, _ = timed(plain_kw, p_steps, warmup=min(args.warmup, 1),
                                     profiled=False)
        ids_plain, dists_plain = ids.clone(), dists.clone()
        log(f"plain path: {p_ms_max / p_steps:.2f} ms per step")

    clocks = ClockSampler(gpu_uuid(torch))
    clocks.start()
    ms, ms_max, counted, prof = timed(chosen_kw, args.steps)
    clk = clocks.stop()
    log(f"chosen path: {ms_max / args.steps:.3f} ms per step")
    l2_prof = {"setaside_bytes": prof["l2_setaside_bytes"],
               "index_permille": prof["l2_index_permille"]} if chosen_kw.get("l2") else None
    value = world * s.nq * args.steps / (ms_max / 1e3)
    plain = None
    if not args.no_plain:
        same = bool(torch.equal(ids, ids_plain) and torch.equal(dists, dists_plain))
        plain = {"value": world * s.nq * p_steps / (p_ms_max / 1e3),
                 "ms_per_step": p_ms_max / p_steps, "steps": p_steps, "settings": plain_kw,
                 "results_identical_to_chosen": same,
                 "warmup": 1 + min(args.warmup, 1),
                 "kernel_ms_first_step": {k2: round(v2, 3) for k2, v2 in p_prof["ms"].items()}}

    # the paper's cache-split grid (QALSH_Ci/Cd/CiCd/Opt settings, Section 6) on
    # the GPU's persisting L2, with the chosen path's other settings
    l2_sweep = None
    if args.l2_sweep:
        ids_c, dists_c = ids.clone(), dists.clone()
        grid = [None, 10, 100, 200, 300, 400, 500, 600, 700, 800, 900, 990, "model"]
        rows = []
        for g in grid:
            kw = dict(chosen_kw, l2=g)
            t_ms, t_max, t_prof, _ = timed(kw, args.sweep_steps, profiled=False)
            rows.append({"l2": "off" if g is None else g,
                         "ms_per_step": round(t_max / args.sweep_steps, 4),
                         "index_permille": t_prof["l2_index_permille"] if g is not None else None,
                         "setaside_bytes": t_prof["l2_setaside_bytes"] if g is not None else None,
                         "identical": bool(torch.equal(ids, ids_c) and torch.equal(dists, dists_c))})
        l2_sweep = {"steps": args.sweep_steps, "rows": rows}

    # end to end through the public API: pinned host queries in, host results out
    Qh = torch.from_numpy(wl.Q).pin_memory()
    ids_h = torch.empty((s.nq, s.k), dtype=torch.int64).pin_memory()
    dists_h = torch.empty((s.nq, s.k), dtype=torch.float32).pin_memory()
    index.query(Qh, s.k, out=(ids_h, dists_h), **chosen_kw)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        index.query(Qh, s.k, out=(ids_h, dists_h), **chosen_kw)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": world * s.nq * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(Qh.numel() * 4),
           "d2h_bytes_per_step": int(ids_h.numel() * 8 + dists_h.numel() * 4)}

    # quality on a seeded query sample (exact k-NN in float64)
    rng = np.random.default_rng(12345)
    pick = torch.from_numpy(np.sort(rng.choice(s.nq, size=min(args.quality_sample, s.nq),
                                               replace=False))).to(dev)
    tids, tdists = exact_knn_gpu(X, Q[pick], s.k)
    recall, ratio = recall_ratio(ids[pick], dists[pick], tids, tdists)
    log(f"quality: recall {recall:.4f}, ratio {ratio:.5f}; end to end {e2e['value']:.1f} q/s")

    # roofline of the dominant kernel and of the candidate-distance kernel;
    # the L2 read rate (a 64 MiB buffer read with the library's own kernel) is
    # the ceiling of kernels whose reads hit L2
    l2_gbs = qw.qw_measure_read_bandwidth(64 << 20, 10)
    peaks, peak_kind = measured_peaks()
    steps = args.steps
    hbm = float(peaks["hbm_gbs"])
    entries = float(st[:, 5].sum())      # index entries scanned per step (incremental flanks)
    # level path: the 16-bit ids of the flanks, and per (query, tile, level)
    # pass the tile's byte counters read and written (2 x 32 KiB); QALSH adds
    # the FP64 keys its range searches read (4 searches of ceil(log2 32768) + 1
    # probes per projection)
    tiles = index.info.n_tiles
    level_passes = prof["level_passes"] / steps
    count_bytes = entries * 2.0 + level_passes * tiles * 2 * 32768.0
    if qalsh:
        count_bytes += level_passes * tiles * s.m * 4 * 16 * 8.0
    dom = "cluster" if prof["ms"]["cluster"] >= prof["ms"]["level"] else "level"
    bitmap = chosen_kw.get("path") == "bitmap"
    dom_name = {"cluster": "cluster_query_kernel (all levels of collision counting, persistent)",
                "level": ("level_kernel (QALSH interval search on sorted FP64 projections + "
                          "collision counting)" if qalsh else
                          "level_kernel (bucket-range search + collision counting)")}[dom]
    if bitmap and dom == "level":
        if chosen_kw.get("loads", "tma") == "fused":
            # one pass: per (query, tile, level) the m bucket summaries (32 B);
            # per live 128-id group the previous and the new candidate word and
            # the bitmap words of the projections touching it (16 B each)
            dom_name = ("bm_fused_kernel (summary filter and bit-sliced collision counts of the "
                        "live 128-id groups in one launch)")
            count_bytes = ((prof["level_passes"] / steps) * index.info.n_tiles * s.m * 32.0
                           + (prof["bitmap_live_groups"] / steps) * 32.0
                           + (prof["bitmap_live_words"] / steps) * 16.0)
        elif chosen_kw.get("loads", "tma") == "direct":
            # the same algorithmic bytes as the one-pass form: per (query, tile,
            # level) the m bucket summaries (32 B); per live 128-id group the
            # previous and the new candidate word and the bitmap words of the
            # projections touching it (16 B each).  The work list between the
            # passes is the implementation's, not the method's.
            dom_name = ("bm_filter_kernel + bm_count_kernel (summary filter, then bit-sliced "
                        "collision counts of the live 128-id groups)")
            count_bytes = ((prof["level_passes"] / steps) * index.info.n_tiles * s.m * 32.0
                           + (prof["bitmap_live_groups"] / steps) * 32.0
                           + (prof["bitmap_live_words"] / steps) * 16.0)
        else:
            # per (query, level) pass and tile: the m bucket bitmaps, the previous
            # level's candidate bitmap and the new one, 4 KiB each
            dom_name = "bm_level_tma_kernel (bit-sliced collision counts, TMA-staged bitmaps)"
            count_bytes = (prof["level_passes"] / steps) * index.info.n_tiles * (s.m + 2) * 4096.0
    # launches actually run; for the two-pass bitmap level a "launch" is one
    # level pass (its filter and count launches; the bucket numbers of each
    # pass are timed apart in their own class)
    two_pass = bitmap and dom == "level" and chosen_kw.get("loads", "tma") in ("direct", "fused")
    dom_launches = (prof["timed_launches"]["bucket"] if two_pass else prof["launches"][dom]) / steps
    dom_ms = prof["ms"][dom] / steps
    per_launch_bytes = count_bytes / max(dom_launches, 1)
    per_launch_s = (dom_ms / 1e3) / max(dom_launches, 1)
    achieved = per_launch_bytes / per_launch_s / 1e9 if per_launch_s > 0 else 0.0
    kept = float(st[:, 3].sum())
    bf16_rr = chosen_kw.get("rerank") in ("bf16", "bf16_tc")
    if bf16_rr:
        # BF16 pass (both forms): per kept candidate its residual row (2 d) and
        # its three per-row constants (12 B; the group means, read once per
        # distinct group, are not counted); FP32 stage: 4 d bytes per survivor
        rr_bytes = (kept * (s.d * 2 + 12) + prof["rerank_fp32_rows"] / steps * s.d * 4
                    + s.nq * s.d * 4 + s.nq * s.k * 12)
        rr_name = ("rerank_tc_kernel (residual BF16 pre-filter with q.r on the tensor cores, "
                   "then FP32 gather + L2 + top-k of the survivors)"
                   if chosen_kw.get("rerank") == "bf16_tc" else
                   "rerank_bf16_kernel (residual BF16 pre-filter, then FP32 gather + L2 + "
                   "top-k of the survivors)")
    else:
        rr_bytes = kept * s.d * 4 + s.nq * s.d * 4 + s.nq * s.k * 12
        rr_name = "rerank_kernel (candidate gather + L2 + top-k)"
    rr_launches = prof["timed_launches"]["rerank"] / steps
    rr_ms = prof["ms"]["rerank"] / steps
    rr_achieved = (rr_bytes / max(rr_launches, 1)) / ((rr_ms / 1e3) / max(rr_launches, 1)) / 1e9 \
        if rr_ms > 0 else 0.0
    # ncu traffic records are taken on the named workload at its own sizes
    resized = bool(size_overrides(args)) or bool(args.queries)
    kname = "cluster_query_kernel" if dom == "cluster" else (
        {"direct": "bm_filter_count", "fused": "bm_fused_kernel"}.get(
            chosen_kw.get("loads", "tma"), "bm_level_tma_kernel") if bitmap else
        ("level_kernel_qalsh" if qalsh else "level_kernel"))
    roofline = {"kernel": dom_name, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": None if resized else ncu_traffic(kname, args.workload),
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": per_launch_bytes,
                "avg_launch_ms": per_launch_s * 1e3, "launches_per_step": dom_launches,
                "share_of_step": round(dom_ms / (ms / steps), 4),
                "l2_read_peak": round(l2_gbs, 1), "frac_l2": round(achieved / l2_gbs, 4)}
    roofline_gather = {"kernel": rr_name, "bound": "hbm",
                       "achieved": round(rr_achieved, 1), "peak": hbm,
                       "frac": round(rr_achieved / hbm, 4), "unit": "GB/s",
                       "traffic": None if resized else ncu_traffic(
                           {"bf16": "rerank_bf16_kernel", "bf16_tc": "rerank_tc_kernel"}.get(
                               chosen_kw.get("rerank"), "rerank_kernel"), args.workload),
                       "algorithmic_bytes_per_launch": rr_bytes / max(rr_launches, 1),
                       "avg_launch_ms": rr_ms / max(rr_launches, 1),
                       "l2_read_peak": round(l2_gbs, 1), "frac_l2": round(rr_achieved / l2_gbs, 4)}
    # kernels launched in the (uninstrumented) timed region
    launches = int(sum(counted["launches"].values()))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nth = host_threads()
        if qalsh:
            built = oracle_qalsh_index(wl, nth)
            qps, dt, nsamp, _ = oracle_qalsh_sample(wl, w_used, index.l,
                                                    max(1, args.cpu_sample) * nth, v=v_used,
                                                    threads=nth, built=built)
            qps1, dt1, nsamp1, _ = oracle_qalsh_sample(wl, w_used, index.l,
                                                       max(1, args.cpu_sample), seed=2,
                                                       v=v_used, threads=1, built=built)
        else:
            built = oracle_index(wl, nth)
            qps, dt, nsamp, _ = oracle_sample(wl, index.l, max(1, args.cpu_sample) * nth,
                                              v=v_used, threads=nth, built=built)
            qps1, dt1, nsamp1, _ = oracle_sample(wl, index.l, max(1, args.cpu_sample), seed=2,
                                                 v=v_used, threads=1, built=built)
        cpu = {"value": qps, "unit": UNIT, "cores": nth, "kind": "oracle",
               "sample": f"{nsamp} seeded queries of the same workload, query procedure only, "
                         f"split over {nth} host threads ({dt:.1f} s wall, FP64)",
               "single_thread": {"value": qps1, "unit": UNIT, "cores": 1,
                                 "sample": f"{nsamp1} other seeded queries on one host thread "
                                           f"({dt1:.1f} s wall, FP64)"}}
        log(f"cpu baseline: {qps:.2f} q/s on {nth} threads, {qps1:.3f} q/s on one")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "family": args.family, "n": s.n,
                   "clusters": s.n_clusters, "d": s.d, "m": s.m, "w": w_used, "c": s.c,
                   "k": s.k, "v": v_used, "l": index.l, "queries_per_gpu": s.nq,
                   "query_clusters": s.query_clusters, "seed": args.seed,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "chosen": chosen_kw, "start_model": train_info, "autotune": tune,
                   "bitmap_bytes": int(index.info.bitmap_bytes),
                   "l2": "inputs larger than L2 (index %.2f GB + data %.2f GB + counters)"
                         % (index.info.device_bytes / 1e9 - s.n * s.d * 4 / 1e9,
                            s.n * s.d * 4 / 1e9)},
        "quality": {"recall": round(recall, 4), "ratio": round(ratio, 5),
                    "sample": int(pick.numel()), "meets_target": recall >= 0.9 and ratio <= 1.05},
        "plain": plain,
        "l2_windows": l2_prof, "l2_sweep": l2_sweep,
        "roofline": roofline, "roofline_gather": roofline_gather,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk,
        "stats": {"levels_median": float(np.median(st[:, 0])),
                  "bitmap_live_items_per_step": prof["bitmap_live_items"] / steps,
                  "bitmap_live_groups_per_step": prof["bitmap_live_groups"] / steps,
                  "bitmap_live_words_per_step": prof["bitmap_live_words"] / steps,
                  "level_passes_per_step": prof["level_passes"] / steps,
                  "rerank_candidates_per_step": prof["rerank_candidates"] / steps,
                  "bitmap_fallbacks_per_step": prof["bitmap_fallbacks"] / steps,
                  "bitmap_overflows_per_step": prof["bitmap_overflows"] / steps,
                  "rerank_fp32_rows_per_step": prof["rerank_fp32_rows"] / steps,
                  "entries_scanned_per_query": float(np.mean(st[:, 5])),
                  "kernel_ms_per_step": {k2: round(v2 / steps, 3) for k2, v2 in prof["ms"].items()}},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if mlp is not None:
        mlp.free()
    index.free()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------- cost-model sweep
SWEEP_PERMILLE = [None, 10, 100, 200, 300, 400, 500, 600, 700, 800, 900, 990]


def fit_split_model(rows):
    """Least-squares fit of the fastest index-window permille over the windowed
    settings, p(n, d) = c0 + c1 log2(n) + c2 log2(d): a model from the data's
    cardinality and dimensionality to the index share of the cache (Section
    5.2), refitted to this GPU's measurements.  Returns the coefficients and
    the residual RMS in permille."""
    import numpy as np
    X = np.array([[1.0, np.log2(r["n"]), np.log2(r["d"])] for r in rows])
    y = np.array([float(r["best_windowed_permille"]) for r in rows])
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    rms = float(np.sqrt(np.mean((X @ coef - y) ** 2)))
    return {"form": "permille = c0 + c1 log2(n) + c2 log2(d)",
            "c": [round(float(c), 3) for c in coef], "rms_permille": round(rms, 1)}


def run_cost_sweep(args):
    """For every (n, d) of the grid: a synthetic mixture workload (n / 1000
    clusters, m = 64, w = 4, 5,000 queries, k = 10, v = 100), answered on the
    bitmap path (level loop in graph mode, plain starts) without an L2 window
    and with the index window given each permille of the persisting-L2
    set-aside (the rest to the data window); the median of --sweep-steps timed
    calls per setting; the fastest setting, the fastest windowed one and the
    library cost model's choice.  Then the fit of the fastest windowed share
    over (n, d).  Results never depend on the window (checked per setting)."""
    import numpy as np
    import torch

    import paper_1907_11803_gb300 as qw
    import workloads
    dev = torch.device("cuda", torch.cuda.current_device())
    ns_txt, ds_txt = args.cost_grid.split(":")
    ns = [int(x) for x in ns_txt.split(",")]
    ds = [int(x) for x in ds_txt.split(",")]
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    rows = []
    for n in ns:
        for d in ds:
            wl = workloads.make_workload("mix10k_d32", seed=args.seed, n=n, d=d, m=64,
                                         n_clusters=max(10, n // 1000), nq=5000, k=10, v=100)
            s = wl.spec
            index = qw.Index(torch.from_numpy(wl.X).to(dev), torch.from_numpy(wl.A).to(dev),
                             torch.from_numpy(wl.b).to(dev), w=4.0, c=2, v=100, l=0,
                             bitmaps=True)
            Q = torch.from_numpy(wl.Q).to(dev)
            ids = torch.empty((s.nq, s.k), dtype=torch.int64, device=dev)
            dists = torch.empty((s.nq, s.k), dtype=torch.float32, device=dev)
            base_kw = dict(path="bitmap", loads="direct", start="plain", graph=True,
                           order="signature", rerank="fp32")
            ref = None
            times = []
            for pm in SWEEP_PERMILLE + ["model"]:
                kw = dict(base_kw, l2=pm)
                for _ in range(2):
                    index.query(Q, s.k, out=(ids, dists), **kw)
                torch.cuda.synchronize()
                index.profile(reset=True)
                t = []
                for _ in range(args.sweep_steps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    index.query(Q, s.k, out=(ids, dists), **kw)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    t.append(e0.elapsed_time(e1))
                prof = index.profile(reset=True)
                same = True
                if ref is None:
                    ref = (ids.clone(), dists.clone())
                else:
                    same = bool(torch.equal(ids, ref[0]) and torch.equal(dists, ref[1]))
                times.append({"l2": "off" if pm is None else pm,
                              "ms": round(float(np.median(t)), 4), "identical": same,
                              "index_permille": int(prof["l2_index_permille"]) if pm else None,
                              "setaside_bytes": int(prof["l2_setaside_bytes"]) if pm else None})
            windowed = [r for r in times if isinstance(r["l2"], int)]
            best = min(times, key=lambda r: r["ms"])
            best_w = min(windowed, key=lambda r: r["ms"])
            model = next(r for r in times if r["l2"] == "model")
            rows.append({"n": n, "d": d, "index_bytes": int(index.info.device_bytes),
                         "data_bytes": n * d * 4, "best": best["l2"],
                         "best_windowed_permille": best_w["l2"],
                         "model_permille": model["index_permille"],
                         "off_ms": times[0]["ms"], "best_ms": best["ms"],
                         "all_identical": all(r["identical"] for r in times), "settings": times})
            log(f"n {n} d {d}: off {times[0]['ms']:.3f} ms, best {best['l2']} "
                f"{best['ms']:.3f} ms, best window {best_w['l2']} permille, model "
                f"{model['index_permille']} permille")
            index.free()
            del wl
    line = {"cost_sweep": rows, "fit": fit_split_model(rows), "steps": args.sweep_steps,
            "permille_grid": [p for p in SWEEP_PERMILLE if p is not None]}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    import workloads
    wl = workloads.make_workload(args.workload, seed=args.seed, nq=args.queries or None,
                                 **size_overrides(args))
    s = wl.spec
    v_used, l_arg = operating_point(args, s)
    qalsh = args.family == "qalsh"
    w_used = float(np.float32(QALSH_W)) if qalsh else s.w
    if l_arg > 0:
        l = l_arg
    elif qalsh:
        l = oracle.get().qalsh_threshold(s.m, w_used, s.c, s.n, v_used)
    else:
        l = oracle.get().threshold(s.m, s.w, s.c, s.n, v_used)
    nth = host_threads()
    per_step = max(1, args.cpu_sample) * nth
    if qalsh:
        orc, P = oracle_qalsh_index(wl, nth)
    else:
        orc, idx = oracle_index(wl, nth)
    rng = np.random.default_rng(99)
    times = []
    for step in range(args.warmup + args.steps):
        pick = np.sort(rng.choice(s.nq, size=per_step, replace=False))
        Qs = wl.Q[pick]
        if qalsh:
            dt = oracle_qalsh_threads(orc, wl, P, Qs, w=w_used, k=s.k, v=v_used, l=l, c=s.c,
                                      threads=nth)
        else:
            HQ = orc.hash(Qs, wl.A, wl.b, s.w)
            dt = oracle_query_threads(orc, wl, idx, Qs, HQ, k=s.k, v=v_used, l=l, c=s.c,
                                      threads=nth)
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per_step * len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / len(times) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "family": args.family, "n": s.n, "d": s.d,
                       "m": s.m, "w": w_used, "k": s.k, "v": v_used, "l": l},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nth, "kind": "oracle",
                             "sample": f"{per_step} seeded queries per step, query procedure "
                                       f"only, split over {nth} host threads, FP64"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.steps is None:
        args.steps = 5 if args.impl == "reference" else 20
    if args.steps < 1 or args.warmup < 0:
        raise SystemExit("--steps must be >= 1 and --warmup >= 0")
    if args.impl == "reference":
        run_reference(args)
    elif args.cost_sweep:
        run_cost_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
