"""Benchmark of the FGIM merge hot path on GB300.

One step = one full merge (stage a cross querying, 3 x (Visit + Update + indegree
repair), Alg. 5 prune + reverse-edge insertion, reachability fix) of the Sift-like
workload: N = 1,000,000 points, d = 128, integer values 0..255 from a 1,000-cluster
mixture, 4 shards of 250,000 with HNSW-style input PGs (M = 32, ef = 128), k = 64,
R = 32, alpha = 1.2. Inputs are synthetic and seeded; the input PGs are built on the
host before timing.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line. Under torchrun (N > 1) every rank merges its own replica of the
workload (weak scaling, no collective on the data path); value = all ranks' points /
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "merged points/sec (3 stages, 1 GB300) at recall@10 within 0.5pt of oracle"
UNIT = "points/s"
WORKLOAD = dict(name="medium", N=1_000_000, d=128, h=4, M=32, ef=128, k=64, R=32, alpha=1.2, iters=3)
# bounded CPU sample: the same recipe at N = 100,000 (4 shards of 25,000)
SAMPLE_N = 100_000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fgim", choices=["fgim", "reference"])
    ap.add_argument("--n", type=int, default=WORKLOAD["N"], help="points (default: the full workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--join-filter", default="tc", choices=["tc", "fp32"],
                    help="Update's pair filter: BF16 tensor-core tile (default) or FP32 SIMT tile")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain FP32 form alongside")
    ap.add_argument("--no-masked", action="store_true",
                    help="skip timing the merge with invalid vertices (a quarter of them) alongside")
    ap.add_argument("--no-hnsw", action="store_true",
                    help="skip building the HNSW upper layers over the merged graph (timed) and their search recall")
    ap.add_argument("--batched", type=int, default=0, metavar="M",
                    help="instead: time the batched form, M merges of the 768-d BF16 cosine recipe (sizes "
                         "log-uniform in [--batched-lo, --batched-hi]) in one fgim_merge_batch call, against "
                         "the plain FP32 form of the same merges; prints its own JSON line")
    ap.add_argument("--batched-lo", type=int, default=10_000)
    ap.add_argument("--batched-hi", type=int, default=200_000)
    ap.add_argument("--configs", default="small,precision,fp8,batched",
                    help="other workloads timed after the headline one, each in its own sub-record: "
                         "'precision' (1M d=96 IP, BF16 filter against plain FP32), 'fp8' (1M d=960, 8 uneven "
                         "shards), 'batched' (64 merges, ~4M points, d=768 BF16 cosine, one call), 'small' (20k, "
                         "d=32, with the single-thread oracle); '' or 'none' = none")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default beam-search launch shape (no fgim_autotune before the timed steps)")
    ap.add_argument("--no-pg-build", action="store_true",
                    help="skip building the headline's input PGs a second time on the GPU (timed, compared)")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip comparing the GPU merge with the oracle's (100k sample and the largest N the "
                         "oracle finishes in about two minutes)")
    return ap.parse_args()


# ---------------------------------------------------------------------------- distributed plumbing
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return dist


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """Largest value over all ranks (the slowest rank's time)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------- inputs
def make_inputs(n: int, seed_offset: int = 0):
    from synth import gen, pgbuild
    w = gen.make(WORKLOAD["name"], N=n, seed=gen.MASTER_SEED + seed_offset)
    graphs = pgbuild.build_all(w)
    return w, graphs


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (read-only query)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(parts)
                except ValueError:
                    pass
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------- oracle legs
def stage_a_work_model(w_full, graphs_full, n_queries_sample=2000):
    """The oracle's Alg. 1 counters (distance evaluations, expansions) per cross query, on
    sampled cross queries of the full workload: the per-query work model of stage a."""
    import oracle as O
    rng = np.random.default_rng(7)
    off = w_full.offsets
    L = -(-w_full.k // (w_full.h - 1))
    ndc = hops = nq = 0
    for g in rng.choice(w_full.N, max(1, n_queries_sample // (w_full.h - 1)), replace=False):
        i = int(np.searchsorted(off, g, side="right") - 1)
        for j in range(w_full.h):
            if j == i:
                continue
            adj, ep = graphs_full[j]
            _, _, st = O.knn_search(w_full.shard(j), adj, ep, w_full.X[g], L, L, w_full.metric)
            ndc += st["ndc"]
            hops += st["hops"]
            nq += 1
    return {"ndc": ndc / nq, "hops": hops / nq, "queries_sampled": nq, "L": L}


def cpu_baseline_leg(w_full, graphs_full, n_queries_sample=2000):
    """The oracle as it stands, on the host cores: (1) a full merge of a bounded sample of the
    workload (the same recipe at SAMPLE_N points), (2) its beam-search counters on sampled
    cross queries of the full workload (the per-query work model of stage a)."""
    import oracle as O
    cores = os.cpu_count() or 1
    w, graphs = make_inputs(SAMPLE_N)
    P = O.Problem.from_workload(w, graphs)
    t0 = time.perf_counter()
    r = O.merge(P, w.k, w.R, w.alpha, iters=WORKLOAD["iters"])
    dt = time.perf_counter() - t0
    return {"value": SAMPLE_N / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"full oracle merge (3 stages, iters=3) of the same recipe at N={SAMPLE_N} "
                      f"(4 shards of {SAMPLE_N // 4}), {dt:.2f} s on {cores} host threads",
            "seconds": dt, "stats": r.stats, "result": r, "inputs": (w, graphs),
            "stage_a_per_query": stage_a_work_model(w_full, graphs_full, n_queries_sample)}


def recall10(found, truth) -> float:
    hits = sum(len(set(a) & set(b)) for a, b in zip(found.tolist(), truth.tolist()))
    return hits / (10 * len(truth))


def exact_top10(X, Q, metric):
    """Exact top-10 of the queries over X on the GPU (evaluation only): torch matmul, chunked."""
    import torch
    out = []
    xx = (X * X).sum(1)
    for s in range(0, Q.shape[0], 256):
        q = Q[s:s + 256]
        ip = q @ X.T
        if metric == 0:
            d = (q * q).sum(1, keepdim=True) - 2 * ip + xx[None, :]
        elif metric == 1:
            d = 1 - ip
        else:
            d = 1 - ip / (torch.linalg.vector_norm(q, dim=1, keepdim=True) * torch.sqrt(xx)[None, :])
        out.append(torch.topk(d, 10, dim=1, largest=False).indices.cpu())
        del ip, d
    return torch.cat(out).numpy()


def oracle_check(fg, kw, w_full, graphs_full, out_full, cpu, dev, nq_eval=1000, budget_s=150.0):
    """The metric's condition, measured: (1) the GPU merge of the oracle's 100k sample against
    the oracle's merge of it (bit for bit on these integer data); (2) the oracle's merge of the
    largest N in {1M, 500k, 250k} expected to finish within `budget_s` on the host cores (its
    time extrapolated linearly from the sample), compared with the GPU merge of the same input,
    and both graphs' search recall@10 at beam 64 (the oracle's graph searched by the oracle)."""
    import torch
    import oracle as O
    res = {}
    if cpu is not None and "result" in cpu:
        w, graphs = cpu["inputs"]
        r = cpu["result"]
        inp = fg.MergeInput.from_flat(torch.from_numpy(w.X).to(dev), w.shard_sizes,
                                      torch.from_numpy(np.concatenate([g[0] for g in graphs])).to(dev),
                                      [g[1] for g in graphs], metric="l2")
        o = fg.merge(inp, **kw, return_knng=True)
        res["sample"] = {"N": w.N, "knng_equal": bool(np.array_equal(o["knng"]["ids"].cpu().numpy(), r.knn_ids)),
                         "graph_equal": bool(np.array_equal(o["ids"].cpu().numpy(), r.ids)),
                         "deg_equal": bool(np.array_equal(o["deg"].cpu().numpy(), r.deg)),
                         "entry_equal": o["entry"] == r.entry}
        per_point = cpu["seconds"] / w.N
        del inp, o
    else:
        per_point = None
    target = None
    for n in (w_full.N, w_full.N // 2, w_full.N // 4):
        if per_point is not None and per_point * n * 1.3 <= budget_s:
            target = n
            break
    if target is None:
        res["full"] = None
        return res
    if target == w_full.N:
        w, graphs = w_full, graphs_full
        o = out_full
    else:
        w, graphs = make_inputs(target)
        inp = fg.MergeInput.from_flat(torch.from_numpy(w.X).to(dev), w.shard_sizes,
                                      torch.from_numpy(np.concatenate([g[0] for g in graphs])).to(dev),
                                      [g[1] for g in graphs], metric="l2")
        o = fg.merge(inp, **kw)
    P = O.Problem.from_workload(w, graphs)
    t0 = time.perf_counter()
    r = O.merge(P, w.k, w.R, w.alpha, iters=WORKLOAD["iters"])
    dt = time.perf_counter() - t0
    Qn = np.ascontiguousarray(w.Q[:nq_eval])
    X = torch.from_numpy(w.X).to(dev)
    Q = torch.from_numpy(Qn).to(dev)
    gt = exact_top10(X, Q, 0)
    sid, _ = fg.search(X, o["ids"], o["entry"], Q, topk=10, beam=64)
    oid, _, _ = O.search(w.X, r.ids, r.entry, Qn, 64, 10, 0)
    rg, ro = recall10(sid.cpu().numpy(), gt), recall10(oid, gt)
    res["full"] = {"N": w.N, "oracle_seconds": dt, "cores": os.cpu_count() or 1,
                   "graph_equal": bool(np.array_equal(o["ids"].cpu().numpy(), r.ids)),
                   "entry_equal": o["entry"] == r.entry,
                   "recall@10_gpu": rg, "recall@10_oracle": ro, "recall_delta_pt": 100 * (rg - ro),
                   "queries": nq_eval, "beam": 64}
    return res


def run_reference(args):
    """The oracle arm: each step is one oracle merge of the bounded sample on the host cores."""
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    import oracle as O
    w, graphs = make_inputs(SAMPLE_N)
    P = O.Problem.from_workload(w, graphs)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.merge(P, w.k, w.R, w.alpha, iters=WORKLOAD["iters"])
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = SAMPLE_N * len(times) / total
    cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"Sift-like merge, oracle sample N={SAMPLE_N}, d=128, 4 shards, k=64, R=32",
                       "sample_of": "medium (N=1,000,000)", "iters": WORKLOAD["iters"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"oracle merge of the recipe at N={SAMPLE_N} per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- GPU arm
# FP32 SIMT issue rate: 152 SMs x 128 FP32 lanes; the direct-form distance costs one FSUB and
# one FFMA (3 flops in 2 issue slots) per element pair, so its ALU peak is 1.5 flop/lane/cycle.
SM_COUNT, FP32_LANES = 152, 128


def row_bytes(w) -> int:
    """Bytes per coordinate the searches and the prune read: 1 when the data qualify for byte
    rows (integers in [0, 255], d <= 128, d % 16 == 0), else 4."""
    X = w.X
    ok = w.d % 16 == 0 and w.d <= 128 and bool(np.all((X >= 0) & (X <= 255) & (X == np.round(X))))
    return 1 if ok else 4


# the sources each captured kernel family is compiled from (its own file plus the shared headers)
TRAFFIC_SOURCES = {
    "k_cross_query": ["k_cross.cu", "k_cross.cuh", "k_beam.cuh"],
    "k_join": ["k_refine.cu", "tc_sm100.cuh"],   # the Update launches: k_join_tc and k_join_sparse
    "k_prune": ["k_prune.cu"],
}


def roofline_kernels(kernels):
    """Per-kernel event times with the Update's two launch kinds (the tile, k_join, and the
    warp-per-vertex form, k_join_sparse) folded into one "k_join" family: its roofline divides
    the whole Update's algorithmic work by the whole Update's time."""
    out = dict(kernels)
    if "k_join_sparse" in out:
        sp = out.pop("k_join_sparse")
        j = out.get("k_join", {"launches": 0, "ms": 0.0})
        out["k_join"] = {"launches": j["launches"] + sp["launches"], "ms": j["ms"] + sp["ms"]}
    return out


def strip_comments(src: str) -> str:
    """C/C++ source without its comments and blank lines (string and character literals kept),
    so that a hash of it changes with the code only."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":   # a literal: copy it whole, escapes included
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(line.rstrip() for line in "".join(out).splitlines() if line.strip())


def kernel_sources_sha256(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in sorted(TRAFFIC_SOURCES[kernel] + ["fgim_internal.cuh"]):
        h.update(f.encode())
        h.update(strip_comments(open(os.path.join(ROOT, "paper_2603_21710_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()


def measured_traffic():
    """Per-launch DRAM bytes from the committed ncu capture (profiles/), keyed by kernel family,
    for the families whose sources are still the ones the capture was taken with (a family
    whose kernel changed since is left out: its figure is stale)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_sift_like_1M.json")
    if not os.path.exists(path):
        return {}
    doc = json.load(open(path))
    shas = doc.get("sources_sha256", {})
    return {k: v for k, v in doc.get("bytes_per_launch", {}).items()
            if k in TRAFFIC_SOURCES and shas.get(k) == kernel_sources_sha256(k)}


def roofline_for(kernel: str, per_launch_ms: float, launches_per_step: float, w, graphs, cpu, peaks, stats, s_row):
    """Algorithmic work of one launch of a kernel / its mean event time (the stage models of
    the measurement plan: bytes a launch must move at least, flops it must do)."""
    N, d, k, M, R = w.N, w.d, w.k, w.M, w.R
    # DRAM bytes per launch from the ncu capture of the full workload (null when stale or when
    # the workload is not the captured one)
    traffic = measured_traffic().get(kernel) if (N == 1_000_000 and getattr(w, "name", "") == "medium") else None
    out = {"kernel": kernel, "per_launch_ms": per_launch_ms, "traffic": traffic}
    hbm = dict(bound="hbm", unit="GB/s", peak=peaks.get("hbm_gbs"), peak_kind="measured copy (hbm_gbs), of measured")
    if kernel == "k_cross_query" and cpu is not None:
        pq = cpu["stage_a_per_query"]
        nq = N * (w.h - 1)
        mean_deg = float(np.mean([(g[0] >= 0).sum(1).mean() for g in graphs]))
        # per cross query: NDC rows (s_row bytes per coordinate) + their ids and `hops`
        # adjacency rows; per vertex: its own FP32 row, its local candidates' rows, its
        # adjacency row and the k-NNG row it writes (NDC, hops: the oracle's counters)
        work = nq * (pq["ndc"] * (d * s_row + 4) + pq["hops"] * M * 4) + N * (
            d * 4 + mean_deg * d * s_row + M * 4 + k * 9)
        out.update(hbm, algorithmic_bytes=work, row_bytes=s_row)
        out["achieved"] = work / (per_launch_ms * 1e-3) / 1e9
    elif kernel == "k_join":
        # Update (tile and warp-per-vertex launches together): every vertex joined reads its
        # candidates' rows (s_row bytes per coordinate, the exact representation) and lists,
        # (|C_n| + |C_o|) (d s_row + 4 k) bytes; flops: 2 d per cross-shard pair of
        # C_n^2 U C_n x C_o
        cands = stats.get("join_cands", 0) / max(launches_per_step, 1)
        pairs = stats["join_pairs"] / max(launches_per_step, 1)
        work = cands * (d * s_row + 4 * k)
        flops = pairs * 2 * d
        out.update(hbm, algorithmic_bytes=work, algorithmic_flops=flops)
        out["achieved"] = work / (per_launch_ms * 1e-3) / 1e9
        bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        out["tensor"] = {"achieved_tflops": flops / (per_launch_ms * 1e-3) / 1e12, "peak_tflops": bf16,
                         "frac": (flops / (per_launch_ms * 1e-3) / 1e12) / bf16 if bf16 else None,
                         "peak_kind": "cuBLAS bf16 sustained (bf16_tflops_sustained), of measured"}
    elif kernel == "k_prune":
        # every vertex gathers its k candidate rows and reads its list, writes R pruned entries
        work = N * (k * d * s_row + k * 8 + R * 8 + 4)
        out.update(hbm, algorithmic_bytes=work, row_bytes=s_row)
        out["achieved"] = work / (per_launch_ms * 1e-3) / 1e9
    else:
        out.update(hbm, achieved=None)
    out["frac"] = out["achieved"] / out["peak"] if out.get("achieved") and out.get("peak") else None
    return out


def gpu_graphs(fg, w, X_dev):
    """Input PGs of every shard built on the GPU (fgim_build_pg: the recipe of the host builder,
    bit for bit on integer data) and the milliseconds it took (CUDA events)."""
    import torch
    metric = {0: "l2", 1: "ip", 2: "cos"}[w.metric]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    out, o = [], 0
    for n in w.shard_sizes:
        out.append(fg.build_pg(X_dev[o:o + n], M=w.M, ef=w.ef, metric=metric))
        o += n
    b.record()
    torch.cuda.synchronize()
    return [(adj.cpu().numpy(), int(e)) for adj, e in out], a.elapsed_time(b)


# the other workloads of the measurement plan, timed after the headline one (one sub-record each)
CONFIGS = {
    "precision": dict(recipe="precision", metric="ip", filter="tc", others=(), oracle_n=100_000, tune=True,
                      workload="Deep-like merge: N=1,000,000 (2 x 500,000), d=96 unit-norm, inner product, "
                               "input PGs M=32 ef=128, k=48, R=32, alpha=1.0, I_max=3"),
    "fp8": dict(recipe="fp8", metric="l2", filter="fp8", others=("tc",), oracle_n=36_000,
                workload="Gist-like merge: N=1,000,000 (8 shards sized i*N/36), d=960 non-negative, squared L2, "
                         "input PGs M=32 ef=128, k=64, R=48, alpha=1.0, I_max=3"),
}


def timed_merges(fg, inp, kw, steps, warmup, profile=False):
    """`warmup` untimed merges, then `steps` merges each bracketed by CUDA events on the
    current stream; with `profile`, the library's per-kernel event times over the timed ones."""
    import torch
    stream = torch.cuda.current_stream()
    out = None
    for _ in range(warmup):
        out = fg.merge(inp, **kw)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kernels = {}
    launches0 = fg.launch_count()
    if profile:
        prof = fg.profiling()
        prof.__enter__()
    for a, b in ev:
        a.record(stream)
        out = fg.merge(inp, **kw)
        b.record(stream)
    torch.cuda.synchronize()
    if profile:
        prof.__exit__(None, None, None)
        for name in prof.names():
            n, ms = prof.query(name)
            if n:
                kernels[name] = {"launches": n, "ms": ms}
    return {"step_ms": [a.elapsed_time(b) for a, b in ev], "kernels": kernels, "out": out,
            "launches": fg.launch_count() - launches0}


def oracle_sample_check(fg, recipe, n, kw, metric_name, dev, filter_, nq=1000, host_graphs=False):
    """The recall delta against the FP64 oracle on a bounded sample of a workload: the same
    recipe at n points, merged by the GPU (chosen form) and by the oracle (all host cores), each
    graph searched by its own side (recall@10, beam 64, exact truth); plus the share of identical
    merged rows."""
    import torch
    import oracle as O
    from synth import gen, pgbuild
    w = gen.make(recipe, N=n, nq=nq)
    X = torch.from_numpy(w.X).to(dev)
    graphs = pgbuild.build_all(w) if host_graphs else gpu_graphs(fg, w, X)[0]
    adj = torch.from_numpy(np.concatenate([g[0] for g in graphs])).to(dev)
    inp = fg.MergeInput.from_flat(X, w.shard_sizes, adj, [g[1] for g in graphs], metric=metric_name)
    o = fg.merge(inp, **kw, join_filter=filter_)
    P = O.Problem.from_workload(w, graphs)
    t0 = time.perf_counter()
    r = O.merge(P, kw["k"], kw["R"], kw["alpha"], iters=kw["iters"])
    dt = time.perf_counter() - t0
    Q = torch.from_numpy(np.ascontiguousarray(w.Q)).to(dev)
    gt = exact_top10(X, Q, w.metric)
    sid, _ = fg.search(X, o["ids"], o["entry"], Q, topk=10, beam=64, metric=metric_name)
    oid, _, _ = O.search(w.X, r.ids, r.entry, np.ascontiguousarray(w.Q), 64, 10, w.metric)
    rg, ro = recall10(sid.cpu().numpy(), gt), recall10(oid, gt)
    gi = o["ids"].cpu().numpy()
    return {"N": n, "oracle_seconds": dt, "cores": os.cpu_count() or 1, "recall@10_gpu": rg,
            "recall@10_oracle": ro, "recall_delta_pt": 100 * (rg - ro), "queries": nq, "beam": 64,
            "rows_identical": float(np.mean(np.all(gi == r.ids, 1))), "entry_equal": o["entry"] == r.entry,
            "input_pgs": "host builder" if host_graphs else "GPU builder (the same recipe)"}


def measure_small(fg, dev, peaks):
    """The small parity workload (20,000 points, d = 32, 2 shards): the GPU forms, the oracle on
    one host thread and on all of them, and the recall of both merged graphs."""
    import torch
    import oracle as O
    from synth import gen, pgbuild
    w = gen.make("small")
    graphs = pgbuild.build_all(w)
    X = torch.from_numpy(w.X).to(dev)
    adj = torch.from_numpy(np.concatenate([g[0] for g in graphs])).to(dev)
    inp = fg.MergeInput.from_flat(X, w.shard_sizes, adj, [g[1] for g in graphs])
    kw = dict(k=w.k, R=w.R, alpha=w.alpha, iters=3)
    ch = timed_merges(fg, inp, dict(kw, join_filter="tc"), 5, 3)
    pl = timed_merges(fg, inp, dict(kw, join_filter="fp32", rows="fp32"), 5, 3)
    times = {}
    for threads in (1, 0):
        P = O.Problem.from_workload(w, graphs, nthreads=threads)
        t0 = time.perf_counter()
        r = O.merge(P, w.k, w.R, w.alpha, iters=3)
        times[threads] = time.perf_counter() - t0
    Q = torch.from_numpy(w.Q).to(dev)
    gt = exact_top10(X, Q, 0)
    sid, _ = fg.search(X, ch["out"]["ids"], ch["out"]["entry"], Q, topk=10, beam=64)
    oid, _, _ = O.search(w.X, r.ids, r.entry, w.Q, 64, 10, 0)
    ms_c, ms_p = float(np.mean(ch["step_ms"])), float(np.mean(pl["step_ms"]))
    gi = ch["out"]["ids"].cpu().numpy()
    return {"workload": "small: N=20,000 (2 x 10,000), d=32, 50-cluster Gaussian mixture, squared L2, input PGs "
                        "M=16 ef=64, k=16, R=32, alpha=1.2, I_max=3",
            "value": w.N / (ms_c * 1e-3), "unit": UNIT, "ms_per_step": ms_c, "steps": 5, "warmup": 3,
            "form": "BF16 tensor-core join filter", "l2_policy": "L2-resident (2.6 MB of vectors): a parity workload",
            "plain_fp32": {"value": w.N / (ms_p * 1e-3), "unit": UNIT, "ms_per_step": ms_p,
                           "same_graph": bool(torch.equal(pl["out"]["ids"], ch["out"]["ids"]))},
            "oracle": {"seconds_1_thread": times[1], "seconds_all_threads": times[0], "cores": os.cpu_count() or 1,
                       "value_1_thread": w.N / times[1], "value_all_threads": w.N / times[0]},
            "recall@10_gpu": recall10(sid.cpu().numpy(), gt), "recall@10_oracle": recall10(oid, gt),
            "rows_identical_to_oracle": float(np.mean(np.all(gi == r.ids, 1))),
            "entry_equal": ch["out"]["entry"] == r.entry}


def measure_config(fg, name, dev, peaks, steps=2, warmup=1, nq_eval=1000):
    """One sub-record: the chosen form (BF16 tensor-core join filter) and the plain FP32 form
    (FP32 rows, FP32 SIMT join filter) of one workload at full size, the roofline of the chosen
    form's dominant kernel and the merged graph's search recall@10 at beam 64."""
    import torch
    from synth import gen, pgbuild
    if name == "batched":
        return measure_batched(fg, dev, peaks, 64, 10_000, 200_000, steps, warmup)
    if name == "small":
        return measure_small(fg, dev, peaks)
    c = CONFIGS[name]
    t0 = time.perf_counter()
    w = gen.make(c["recipe"])
    X = torch.from_numpy(w.X).to(dev)
    graphs, pg_ms = gpu_graphs(fg, w, X)
    t_inputs = time.perf_counter() - t0
    adj = torch.from_numpy(np.concatenate([g[0] for g in graphs])).to(dev)
    inp = fg.MergeInput.from_flat(X, w.shard_sizes, adj, [g[1] for g in graphs], metric=c["metric"])
    kw = dict(k=w.k, R=w.R, alpha=w.alpha, iters=3)
    # tuned beam-search shape where a tuning run is short (a few seconds of cross queries)
    tune = fg.autotune(inp, k=w.k) if c.get("tune") else None
    ch = timed_merges(fg, inp, dict(kw, join_filter=c["filter"]), steps, warmup, profile=True)
    stats = ch["out"]["stats"]
    pl = timed_merges(fg, inp, dict(kw, join_filter="fp32", rows="fp32"), 1, 0)
    others = {}
    for jf in c["others"]:   # the other reduced-precision forms, same inputs
        ot = timed_merges(fg, inp, dict(kw, join_filter=jf), 1, 0)
        ms_o = float(np.mean(ot["step_ms"]))
        others[jf] = {"value": w.N / (ms_o * 1e-3), "unit": UNIT, "ms_per_step": ms_o, "steps": 1,
                      "same_graph": bool(torch.equal(ot["out"]["ids"], ch["out"]["ids"]))}
        del ot
    ms_c, ms_p = float(np.mean(ch["step_ms"])), float(np.mean(pl["step_ms"]))
    Q = torch.from_numpy(np.ascontiguousarray(w.Q[:nq_eval])).to(dev)
    gt = exact_top10(X, Q, w.metric)
    sid, _ = fg.search(X, ch["out"]["ids"], ch["out"]["entry"], Q, topk=10, beam=64, metric=c["metric"])
    model = {"stage_a_per_query": stage_a_work_model(w, graphs, 1000)}
    kernels = ch["kernels"]
    rk = roofline_kernels(kernels)
    dom = max(rk.items(), key=lambda kv: kv[1]["ms"])[0] if rk else None
    s_row = row_bytes(w)
    roof = (roofline_for(dom, rk[dom]["ms"] / rk[dom]["launches"], rk[dom]["launches"] / steps, w,
                         graphs, model, peaks, stats, s_row) if dom else None)
    roof_all = {k_: roofline_for(k_, rk[k_]["ms"] / rk[k_]["launches"], rk[k_]["launches"] / steps, w,
                                 graphs, model, peaks, stats, s_row)
                for k_ in ("k_cross_query", "k_join", "k_prune") if k_ in rk}
    rec = {"workload": c["workload"], "N": w.N, "d": w.d, "shards": w.shard_sizes, "value": w.N / (ms_c * 1e-3),
           "unit": UNIT, "ms_per_step": ms_c, "steps": steps, "warmup": warmup, "step_ms": ch["step_ms"],
           "form": {"tc": "BF16", "fp8": "FP8 E4M3 (per-vector scales)"}[c["filter"]] +
                   " tensor-core join filter with exact FP32 re-rank, FP32 rows elsewhere",
           "other_forms": {{"tc": "bf16"}.get(k_, k_): v for k_, v in others.items()},
           "plain_fp32": {"value": w.N / (ms_p * 1e-3), "unit": UNIT, "ms_per_step": ms_p, "steps": 1,
                          "form": "FP32 rows, FP32 SIMT join filter",
                          "same_graph": bool(torch.equal(pl["out"]["ids"], ch["out"]["ids"]))},
           "recall@10": recall10(sid.cpu().numpy(), gt), "recall_eval": {"queries": nq_eval, "beam": 64},
           "gpu_launches_per_step": ch["launches"] / steps, "roofline": roof, "roofline_by_kernel": roof_all,
           "beam_shape": ({"warps_per_block": tune["wpb"], "table_bits": tune["ht_bits"], "by": "fgim_autotune"}
                          if tune else "default"),
           "kernels": kernels, "merge_stats": stats, "inputs_seconds": t_inputs,
           "inputs": f"vectors drawn on the host; input PGs (M={w.M}, ef={w.ef}) built on the GPU by "
                     f"fgim_build_pg in {pg_ms:.0f} ms",
           "l2_policy": f"inputs larger than L2 ({w.N * w.d * 4 / 1e9:.2f} GB of vectors)"}
    del inp, X, adj, ch, pl
    torch.cuda.empty_cache()
    fg.trim_memory()
    if c.get("oracle_n"):   # the recall delta against the FP64 oracle, on a bounded sample
        rec["oracle_sample"] = oracle_sample_check(fg, c["recipe"], c["oracle_n"], kw, c["metric"], dev, c["filter"])
    return rec


def run_fgim(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        init_dist(ws, "nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_2603_21710_gb300 as fg
    from synth import gen, pgbuild
    fg.load()
    w = gen.make(WORKLOAD["name"], N=args.n, seed=gen.MASTER_SEED)
    t0 = time.perf_counter()
    graphs = pgbuild.build_all(w)
    t_pg_host = time.perf_counter() - t0
    X = torch.from_numpy(w.X).to(dev)
    # the same input PGs built on the GPU (outside every timed region): equal on these integer data
    pg_build = None
    if not args.no_pg_build:
        g_gpu, pg_gpu_ms = gpu_graphs(fg, w, X)
        pg_build = {"gpu_ms": pg_gpu_ms, "host_seconds": t_pg_host, "host_threads": os.cpu_count() or 1,
                    "equal": all(np.array_equal(a[0], b[0]) and a[1] == b[1] for a, b in zip(g_gpu, graphs)),
                    "recipe": f"batch-incremental insertion from the medoid, M={w.M}, ef={w.ef}, {w.h} shards"}
        del g_gpu
    adj_np = np.concatenate([g[0] for g in graphs])
    adj = torch.from_numpy(adj_np).to(dev)
    entries = [g[1] for g in graphs]
    inp = fg.MergeInput.from_flat(X, w.shard_sizes, adj, entries, metric="l2")
    kw = dict(k=w.k, R=w.R, alpha=w.alpha, iters=WORKLOAD["iters"], join_filter=args.join_filter)
    # the beam-search launch shape tuned on this merge's cross query (fgim_autotune; outside every
    # timed region, as a user would run it once per workload)
    tune = None if args.no_autotune else fg.autotune(inp, k=w.k)
    stream = torch.cuda.current_stream()
    out = None
    for _ in range(args.warmup):
        out = fg.merge(inp, **kw)
    torch.cuda.synchronize()
    barrier(ws)
    # ---- timed region (device-resident inputs)
    launches0 = fg.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk, fg.profiling() as prof:
        torch.cuda.synchronize()
        barrier(ws)
        for s in range(args.steps):
            ev[s][0].record(stream)
            out = fg.merge(inp, **kw)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        kernels = {}
        for name in prof.names():
            n, ms = prof.query(name)
            if n:
                kernels[name] = {"launches": n, "ms": ms}
    launches = fg.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    local_ms = sum(step_ms)
    total_ms = max_over_ranks(local_ms, ws, dev)
    stats = out["stats"]
    # ---- the plain FP32 form on the same inputs (FP32 rows everywhere, FP32 SIMT join filter):
    # outside the main timed region, same event timing, fewer steps
    plain = None
    if not args.no_plain:
        kwp = dict(kw, join_filter="fp32", rows="fp32")
        fg.merge(inp, **kwp)
        torch.cuda.synchronize()
        barrier(ws)
        ps = max(1, min(2, args.steps))
        pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ps)]
        for q in range(ps):
            pev[q][0].record(stream)
            outp = fg.merge(inp, **kwp)
            pev[q][1].record(stream)
        torch.cuda.synchronize()
        p_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in pev), ws, dev)
        plain = {"value": ws * w.N * ps / (p_ms * 1e-3), "unit": UNIT, "ms_per_step": p_ms / ps, "steps": ps,
                 "form": "FP32 rows, FP32 SIMT join filter", "same_graph": bool(torch.equal(outp["ids"], out["ids"]))}
    # ---- the same merge with a quarter of the vertices invalid (the ID mapping of deletion
    # merges): outside the main timed region, same event timing, fewer steps
    masked = None
    if not args.no_masked:
        gen_m = torch.Generator(device="cpu").manual_seed(20260321)
        valid = (torch.rand(w.N, generator=gen_m) >= 0.25).to(dev)
        inp_m = fg.MergeInput.from_flat(X, w.shard_sizes, adj, entries, metric="l2", valid=valid)
        fg.merge(inp_m, **kw)
        torch.cuda.synchronize()
        barrier(ws)
        ms_ = max(1, min(2, args.steps))
        mev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ms_)]
        for q in range(ms_):
            mev[q][0].record(stream)
            fg.merge(inp_m, **kw)
            mev[q][1].record(stream)
        torch.cuda.synchronize()
        m_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in mev), ws, dev)
        masked = {"value": ws * inp_m.N_out * ms_ / (m_ms * 1e-3), "unit": UNIT, "ms_per_step": m_ms / ms_,
                  "steps": ms_, "valid_points": inp_m.N_out, "input_points": w.N,
                  "form": "a quarter of the vertices invalid (seeded uniform mask); value counts valid points"}
        del inp_m, valid
    # ---- evaluation outside the timed region: recall@10 at beam 64 against exact k-NN
    nq_eval = min(1000, w.Q.shape[0])
    Q = torch.from_numpy(w.Q[:nq_eval]).to(dev)
    sid, _ = fg.search(X, out["ids"], out["entry"], Q, topk=10, beam=64)
    d2 = (Q * Q).sum(1, keepdim=True) - 2 * Q @ X.T + (X * X).sum(1)[None, :]
    gt = torch.topk(d2, 10, dim=1, largest=False).indices
    hits = sum(len(set(a) & set(b)) for a, b in zip(sid.cpu().tolist(), gt.cpu().tolist()))
    recall = hits / (10 * nq_eval)
    del d2
    # ---- HNSW-adaptive merging: upper layers over the merged graph (M = R / 2), timed with
    # events after one untimed build, and the recall of the layered search at the same beam
    hnsw = None
    if not args.no_hnsw:
        Mup = max(2, w.R // 2)
        fg.build_layers(X, M=Mup, ef=64, seed=20260321)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        built = fg.build_layers(X, M=Mup, ef=64, seed=20260321)
        h1.record(stream)
        torch.cuda.synchronize()
        hid, _, _ = fg.search_hnsw(X, out["ids"], built["layers"], built["entry"], Q, topk=10, beam=64, ef_up=8)
        hh = sum(len(set(a) & set(b)) for a, b in zip(hid.cpu().tolist(), gt.cpu().tolist()))
        hnsw = {"build_ms": h0.elapsed_time(h1), "M": Mup, "ef": 64,
                "layer_sizes": [int(ly["members"].shape[0]) for ly in built["layers"]],
                "recall@10": hh / (10 * nq_eval), "recall@10_flat": recall, "beam": 64, "ef_up": 8}
        del built
    # ---- end to end through the host-buffer entry point (pinned host inputs and outputs)
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(w.X).pin_memory()
        Ah = torch.from_numpy(adj_np).pin_memory()
        oi = torch.empty((w.N, w.R), dtype=torch.int32).pin_memory()
        od = torch.empty((w.N,), dtype=torch.int32).pin_memory()
        fg.merge_host(Xh, Ah, w.shard_sizes, entries, out_ids=oi, out_deg=od, **kw)
        torch.cuda.synchronize()
        barrier(ws)
        eev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        walls = []
        t0 = time.perf_counter()
        for q in range(args.steps):
            tq = time.perf_counter()
            eev[q][0].record(stream)
            fg.merge_host(Xh, Ah, w.shard_sizes, entries, out_ids=oi, out_deg=od, **kw)
            eev[q][1].record(stream)
            walls.append(1e3 * (time.perf_counter() - tq))
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
        e2e = {"value": ws * w.N * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(Xh.numel() * 4 + Ah.numel() * 4),
               "d2h_bytes_per_step": int(oi.numel() * 4 + od.numel() * 4 + 4),
               "step_wall_ms": walls, "step_device_ms": [a.elapsed_time(b) for a, b in eev]}
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline_leg(w, graphs)
    ocheck = None
    if not args.no_oracle_check and ws == 1:
        ocheck = oracle_check(fg, kw, w, graphs, out, cpu, dev)
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    rk = roofline_kernels(kernels)
    dom = max(rk.items(), key=lambda kv: kv[1]["ms"])[0] if rk else None
    s_row = row_bytes(w)
    roof = (roofline_for(dom, rk[dom]["ms"] / rk[dom]["launches"], rk[dom]["launches"] / args.steps,
                         w, graphs, cpu, peaks, stats, s_row) if dom else None)
    # the same figures for every modelled kernel, for the record
    roof_all = {name: roofline_for(name, rk[name]["ms"] / rk[name]["launches"],
                                   rk[name]["launches"] / args.steps, w, graphs, cpu, peaks, stats, s_row)
                for name in ("k_cross_query", "k_join", "k_prune") if name in rk}
    value = ws * w.N * args.steps / (total_ms * 1e-3)
    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Sift-like merge: N=1,000,000 (4 x 250,000), d=128 integer 0..255, "
                                   "input PGs M=32 ef=128, k=64, R=32, alpha=1.2, I_max=3",
                       "N": w.N, "d": w.d, "shards": w.shard_sizes, "k": w.k, "R": w.R, "alpha": w.alpha,
                       "iters": WORKLOAD["iters"], "l2_policy": "inputs larger than L2 (512 MB vectors)",
                       "parallelism": f"replicas x{ws}"},
            "recall@10": recall, "recall_eval": {"queries": nq_eval, "beam": 64, "truth": "exact (GPU brute force)"},
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks, "roofline": roof,
            "cpu_baseline": ({k_: v for k_, v in cpu.items() if k_ in ("value", "unit", "cores", "kind", "sample")}
                             if cpu else None),
            "stage_a_work_model": cpu["stage_a_per_query"] if cpu else None,
            "plain_fp32": plain,
            "masked": masked,
            "hnsw": hnsw,
            "oracle_check": ocheck,
            "input_pg_build": pg_build,
            "beam_shape": ({"warps_per_block": tune["wpb"], "table_bits": tune["ht_bits"],
                            "cross_query_ms": tune["ms"], "by": "fgim_autotune"} if tune else "default"),
            "roofline_by_kernel": roof_all, "kernels": kernels, "merge_stats": stats, "step_ms": step_ms,
            "ms_median": float(np.median(step_ms))}
    if ws == 1 and args.configs and args.configs != "none":
        # the other workloads, each outside the headline's timed region, in its own sub-record
        del X, adj, inp, out
        torch.cuda.empty_cache()
        fg.trim_memory()
        line["configs"] = {}
        for name in [c for c in args.configs.split(",") if c]:
            try:
                line["configs"][name] = measure_config(fg, name, dev, peaks)
            except Exception as ex:   # a sub-record that fails is reported, not fatal to the headline line
                line["configs"][name] = {"error": f"{type(ex).__name__}: {ex}"}
                torch.cuda.synchronize()
    print(json.dumps(line), flush=True)


def measure_batched(fg, dev, peaks, n_merges, lo, hi, steps, warmup):
    """The batched form: n_merges merges of the 768-d BF16 cosine recipe (sizes log-uniform in
    [lo, hi], h in 2..6) in one fgim_merge_batch call (run as one problem over the union of the
    merges), against the same batch run merge after merge and against the plain FP32 form (FP32
    storage of the same values, FP32 SIMT join filter); inputs resident on the device."""
    import torch
    from synth import gen
    t0 = time.perf_counter()
    ws_ = gen.batched(n_merges=n_merges, n_lo=lo, n_hi=hi, nq=200)
    chosen, plain, pg_ms = [], [], 0.0
    for w in ws_:
        xb = torch.from_numpy(w.bits().view(np.int16)).to(dev).view(torch.bfloat16)
        g, ms = gpu_graphs(fg, w, xb)
        pg_ms += ms
        adj = torch.from_numpy(np.concatenate([x[0] for x in g])).to(dev)
        ent = [x[1] for x in g]
        chosen.append(fg.MergeInput.from_flat(xb, w.shard_sizes, adj, ent, metric="cos"))
        plain.append(fg.MergeInput.from_flat(torch.from_numpy(w.X).to(dev), w.shard_sizes, adj, ent, metric="cos"))
    t_inputs = time.perf_counter() - t0
    w0 = ws_[0]
    kw = dict(k=w0.k, R=w0.R, alpha=w0.alpha, iters=3)
    stream = torch.cuda.current_stream()

    def timed(inps, nsteps, profile=False, **extra):
        out = None
        for _ in range(max(1, warmup)):
            out = fg.merge_batch(inps, **kw, **extra)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        kernels = {}
        if profile:
            prof = fg.profiling()
            prof.__enter__()
        for a, b in ev:
            a.record(stream)
            out = fg.merge_batch(inps, **kw, **extra)
            b.record(stream)
        torch.cuda.synchronize()
        if profile:
            prof.__exit__(None, None, None)
            for name in prof.names():
                n, ms = prof.query(name)
                if n:
                    kernels[name] = {"launches": n, "ms": ms}
        return sum(a.elapsed_time(b) for a, b in ev) / nsteps, out, kernels

    ms_c, out_c, kernels = timed(chosen, steps, profile=True)
    stats = fg.last_stats()
    fg._lib.test_set("batch_union", 0)
    try:
        ms_s, out_s, _ = timed(chosen, 1)
    finally:
        fg._lib.test_set("batch_union", 1)
    ms_p, out_p, _ = timed(plain, 1, join_filter="fp32")
    N = sum(w.N for w in ws_)
    # the recall delta against the FP64 oracle on the two smallest merges of the batch (each
    # merged alone by the oracle; GPU graphs from the batch call)
    import oracle as O
    osamp = []
    for m in sorted(range(len(ws_)), key=lambda i: ws_[i].N)[:2]:
        w = ws_[m]
        graphs = [(a.cpu().numpy(), e) for a, e in zip(chosen[m].adjs, chosen[m].entries)]
        r = O.merge(O.Problem.from_workload(w, graphs), w.k, w.R, w.alpha, iters=3)
        Xm = torch.from_numpy(w.X).to(dev)
        Qm = torch.from_numpy(np.ascontiguousarray(w.Q)).to(dev)
        gt = exact_top10(Xm, Qm, w.metric)
        sid, _ = fg.search(Xm, out_c[m]["ids"], out_c[m]["entry"], Qm, topk=10, beam=64, metric="cos")
        oid, _, _ = O.search(w.X, r.ids, r.entry, np.ascontiguousarray(w.Q), 64, 10, w.metric)
        rg, ro = recall10(sid.cpu().numpy(), gt), recall10(oid, gt)
        osamp.append({"merge": m, "N": w.N, "h": w.h, "recall@10_gpu": rg, "recall@10_oracle": ro,
                      "recall_delta_pt": 100 * (rg - ro), "queries": len(w.Q),
                      "rows_identical": float(np.mean(np.all(out_c[m]["ids"].cpu().numpy() == r.ids, 1)))})
        del Xm, Qm
    rk = roofline_kernels(kernels)
    dom = max(rk.items(), key=lambda kv: kv[1]["ms"])[0] if rk else None
    roof = None
    if dom in ("k_join", "k_prune"):
        class _W:   # the batch as one workload for the per-kernel work model
            pass
        wu = _W()
        wu.N, wu.d, wu.k, wu.M, wu.R, wu.h = N, w0.d, w0.k, w0.M, w0.R, 2
        roof = roofline_for(dom, rk[dom]["ms"] / rk[dom]["launches"], rk[dom]["launches"] / steps, wu,
                            None, None, peaks, stats, 4)
    rec = {"metric": "merged points/sec, batched form (one fgim_merge_batch call)", "value": N / (ms_c * 1e-3),
           "unit": UNIT, "ms_per_step": ms_c, "steps": steps, "warmup": max(1, warmup),
           "dtype": "bf16 storage, f32 arithmetic",
           "workload": f"{n_merges} merges of the 768-d cosine recipe, BF16 storage, sizes log-uniform in "
                       f"[{lo}, {hi}], h in 2..6, input PGs M=24 ef=96, k=32, R=24, I_max=3",
           "N_total": N, "sizes": [w.N for w in ws_], "shards": [w.h for w in ws_],
           "form": "the batch as one problem over the union of its merges (each stage's kernels once per batch)",
           "one_by_one": {"value": N / (ms_s * 1e-3), "unit": UNIT, "ms_per_step": ms_s, "steps": 1,
                          "form": "the same merges one after another in the same call",
                          "same_graphs": all(torch.equal(a["ids"], b["ids"]) for a, b in zip(out_c, out_s))},
           "plain_fp32": {"value": N / (ms_p * 1e-3), "unit": UNIT, "ms_per_step": ms_p, "steps": 1,
                          "form": "FP32 storage of the same values, FP32 SIMT join filter",
                          "same_graphs": all(torch.equal(a["ids"], b["ids"]) for a, b in zip(out_c, out_p))},
           "roofline": roof, "kernels": kernels, "merge_stats": stats, "inputs_seconds": t_inputs,
           "oracle_sample": osamp,
           "inputs": f"vectors drawn on the host; input PGs built on the GPU by fgim_build_pg in {pg_ms:.0f} ms",
           "l2_policy": f"inputs larger than L2 ({N * w0.d * 2 / 1e9:.2f} GB of BF16 vectors)"}
    del chosen, plain, out_c, out_s, out_p
    torch.cuda.empty_cache()
    fg.trim_memory()
    return rec


def run_batched(args):
    """The batched form on its own line (see measure_batched)."""
    import torch
    import paper_2603_21710_gb300 as fg
    dev = torch.device("cuda", 0)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    rec = measure_batched(fg, dev, peaks, args.batched, args.batched_lo, args.batched_hi, args.steps, args.warmup)
    line = {k: rec[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype")}
    line.update({"n_gpus": 1, "higher_is_better": True, "data": "synthetic",
                 "config": {"workload": rec["workload"], "sizes": rec["sizes"], "shards": rec["shards"]}})
    line.update({k: v for k, v in rec.items() if k not in line})
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.batched:
        run_batched(args)
        return
    run_fgim(args)
    ws, _, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
