"""FGIM merge hot path on GB300 (sm_103a): Python binding of the C ABI in include/fgim.h.

Argument marshalling only. PyTorch provides device memory and the current stream;
every step of the merge runs in libfgim.so's CUDA kernels.

    import paper_2603_21710_gb300 as fg
    inp = fg.MergeInput(vectors, adjs, entries, metric="l2")   # per-shard CUDA tensors
    out = fg.merge(inp, k=64, R=32, alpha=1.2)                 # merged PG on the device
    ids, dist = fg.search(inp.X, out["ids"], out["entry"], queries, topk=10, beam=64)
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import torch

from . import _lib
from ._lib import FgimError, KNNG, Graph, Params, Shard, check, last_stats, load  # noqa: F401

__all__ = ["MergeInput", "merge", "merge_batch", "merge_host", "hnsw_levels", "hnsw_layer", "build_layers",
           "search_hnsw", "build_pg", "cross_query", "refine_pass", "indegree_repair", "prune",
           "reverse_insert", "reach_fix", "search", "last_stats", "load", "launch_count", "FgimError",
           "FLAG_NEW", "FLAG_REPLACED", "profiling"]

FLAG_NEW = 1
FLAG_REPLACED = 2
# Update's candidate-distance precision: BF16 tensor-core tile, FP32 SIMT tile or FP8 E4M3
# tensor-core tile with per-vector scales (same results: survivors are re-ranked exactly)
JOIN_FILTERS = {"tc": 0, "bf16": 0, "fp32": 1, "simt": 1, "fp8": 2, "e4m3": 2, 0: 0, 1: 1, 2: 2}
# row storage: "auto" reads one byte per coordinate when the data allow it (integers in
# [0, 255], d <= 128, d % 16 == 0; distances are then exact integers, equal to the FP32
# ones), "fp32" always reads the FP32 rows
ROW_STORAGE = {"auto": 0, "fp32": 1, "off": 1, 0: 0, 1: 1}
# Alg. 5's neighbour-selection rule: alpha-RNG, MRNG or tau-MNG (with tau)
PRUNE_RULES = {"arng": 0, "alpha-rng": 0, "mrng": 1, "tmng": 2, "tau-mng": 2, 0: 0, 1: 1, 2: 2}


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _p(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


_VEC_DTYPES = {torch.float32: 0, torch.bfloat16: 1}


def _vec(t: torch.Tensor, name: str) -> torch.Tensor:
    """A vector tensor in one of the storages the library reads (FP32 or BF16)."""
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype not in _VEC_DTYPES:
        raise ValueError(f"{name} must be float32 or bfloat16, got {t.dtype}")
    return t.contiguous()


def _dev(t: torch.Tensor, dtype: torch.dtype, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


class MergeInput:
    """The h input indexes: per-shard vectors [n_i, d] float32 or bfloat16 and PGs [n_i, M_i] int32
    (local ids).

    Shards are stored back to back in one [N, d] tensor ``X`` (phi order), so the library
    never copies FP32 ones; BF16 ones are decoded into an FP32 working copy per call.
    """

    def __init__(self, vectors: Sequence[torch.Tensor], adjs: Sequence[torch.Tensor], entries: Sequence[int],
                 metric="l2", valid: Optional[Sequence[Optional[torch.Tensor]]] = None):
        """valid: per shard an optional [n_i] bool / uint8 CUDA tensor (the ID mapping phi of
        Sec. 4.1.3): invalid vertices get no row in the merged index and are nobody's
        neighbour. Merged ids number the valid vertices in (shard, local id) order."""
        if len(vectors) != len(adjs) or len(vectors) != len(entries):
            raise ValueError("vectors, adjs and entries must have one item per shard")
        if valid is not None and len(valid) != len(vectors):
            raise ValueError("valid must have one item (or None) per shard")
        self.metric = _lib.METRICS[metric]
        vs = [_vec(v, "vectors") for v in vectors]
        if len({v.dtype for v in vs}) != 1:
            raise ValueError("all shards must use the same vector dtype")
        self.dtype = _VEC_DTYPES[vs[0].dtype]
        self.sizes = [int(v.shape[0]) for v in vs]
        self.d = int(vs[0].shape[1])
        self.X = vs[0] if len(vs) == 1 else torch.cat(vs, 0).contiguous()
        self.adjs = [_dev(a, torch.int32, "adj") for a in adjs]
        self.entries = [int(e) for e in entries]
        self.N = int(sum(self.sizes))
        self.valid = None
        if valid is not None and any(m is not None for m in valid):
            self.valid = []
            for m, n in zip(valid, self.sizes):
                if m is None:
                    self.valid.append(None)
                    continue
                if not m.is_cuda or m.shape != (n,):
                    raise ValueError("each valid mask must be a CUDA tensor of shape [n_i]")
                self.valid.append(m.to(torch.uint8).contiguous())
        # rows of the merged index: the valid vertices
        self.N_out = self.N if self.valid is None else int(
            sum(n if m is None else int(m.count_nonzero()) for m, n in zip(self.valid, self.sizes)))
        self._shards = (Shard * len(vs))()
        o = 0
        for i, (n, a, e) in enumerate(zip(self.sizes, self.adjs, self.entries)):
            m = None if self.valid is None else self.valid[i]
            self._shards[i] = Shard(self.X[o:o + n].data_ptr(), a.data_ptr(), n, int(a.shape[1]), e, 0,
                                    None if m is None else m.data_ptr())
            o += n

    @property
    def h(self) -> int:
        return len(self.sizes)

    @classmethod
    def from_flat(cls, X: torch.Tensor, sizes: Sequence[int], adj: torch.Tensor, entries: Sequence[int],
                  metric="l2", valid: Optional[torch.Tensor] = None) -> "MergeInput":
        """X [N, d] with shards consecutive; adj [N, M] local ids; valid: optional [N] mask."""
        vs, ads, ms, o = [], [], [], 0
        for n in sizes:
            vs.append(X[o:o + n])
            ads.append(adj[o:o + n])
            ms.append(None if valid is None else valid[o:o + n])
            o += n
        return cls(vs, ads, entries, metric, None if valid is None else ms)

    def params(self, k=16, R=32, alpha=1.0, L=0, iters=3, rev_cap=0, ensure_reachable=True,
               reach_beam=0, join_filter="tc", rows="auto", rule="arng", tau=0.0) -> Params:
        p = Params()
        p.dim, p.dtype, p.metric = self.d, self.dtype, self.metric
        p.k, p.R, p.alpha, p.L, p.iters, p.rev_cap = k, R, float(alpha), L, iters, rev_cap
        p.ensure_reachable, p.reach_beam = int(bool(ensure_reachable)), reach_beam
        p.join_filter = JOIN_FILTERS[join_filter]
        p.byte_rows = ROW_STORAGE[rows]
        p.prune_rule, p.tau = PRUNE_RULES[rule], float(tau)
        return p


def _knng_struct(ids, dist, flags) -> KNNG:
    return KNNG(ids.data_ptr(), dist.data_ptr(), flags.data_ptr(), ids.shape[0], ids.shape[1], 0)


def _new_knng(N: int, k: int, device) -> dict:
    return {"ids": torch.empty((N, k), dtype=torch.int32, device=device),
            "dist": torch.empty((N, k), dtype=torch.float32, device=device),
            "flags": torch.empty((N, k), dtype=torch.uint8, device=device)}


def trim_memory() -> None:
    """Return the unused part of the library's scratch pools to the device (see fgim.h)."""
    load().fgim_trim_memory()


def merge(inp: MergeInput, k: int, R: int, alpha: float = 1.0, L: int = 0, iters: int = 3, rev_cap: int = 0,
          ensure_reachable: bool = True, reach_beam: int = 0, return_knng: bool = False,
          join_filter="tc", rows="auto", rule="arng", tau: float = 0.0) -> dict:
    """Full merge (stages a, b, c and the reachability fix). Returns device tensors. rule: Alg. 5's
    neighbour selection ("arng" alpha-RNG, "mrng", "tmng" tau-MNG with `tau`)."""
    L_ = load()
    p = inp.params(k, R, alpha, L, iters, rev_cap, ensure_reachable, reach_beam, join_filter, rows, rule, tau)
    dev = inp.X.device
    N = inp.N_out
    out = {"ids": torch.empty((N, R), dtype=torch.int32, device=dev),
           "dist": torch.empty((N, R), dtype=torch.float32, device=dev),
           "deg": torch.empty((N,), dtype=torch.int32, device=dev)}
    g = Graph(out["ids"].data_ptr(), out["dist"].data_ptr(), out["deg"].data_ptr(), N, R, 0)
    kn = None
    if return_knng:
        kd = _new_knng(N, k, dev)
        kn = _knng_struct(kd["ids"], kd["dist"], kd["flags"])
    check(L_.fgim_merge(inp._shards, inp.h, ctypes.byref(p), ctypes.byref(kn) if kn else None, ctypes.byref(g),
                        _stream()))
    out["entry"] = int(g.entry)
    out["stats"] = last_stats()
    if return_knng:
        out["knng"] = kd
    return out


def merge_batch(inputs: Sequence[MergeInput], k: int, R: int, alpha: float = 1.0, L: int = 0, iters: int = 3,
                rev_cap: int = 0, ensure_reachable: bool = True, reach_beam: int = 0, join_filter="tc",
                rows="auto") -> List[dict]:
    """Independent merges with one set of params in one library call (fgim_merge_batch)."""
    L_ = load()
    inputs = list(inputs)
    n = len(inputs)
    if n == 0:
        return []
    if any((i.d, i.dtype, i.metric) != (inputs[0].d, inputs[0].dtype, inputs[0].metric) for i in inputs):
        raise ValueError("all merges of a batch share dim, dtype and metric")
    p = inputs[0].params(k, R, alpha, L, iters, rev_cap, ensure_reachable, reach_beam, join_filter, rows)
    outs, graphs = [], (Graph * n)()
    shard_ptrs = (ctypes.c_void_p * n)()
    hs = (ctypes.c_int32 * n)()
    for m, inp in enumerate(inputs):
        dev = inp.X.device
        o = {"ids": torch.empty((inp.N_out, R), dtype=torch.int32, device=dev),
             "dist": torch.empty((inp.N_out, R), dtype=torch.float32, device=dev),
             "deg": torch.empty((inp.N_out,), dtype=torch.int32, device=dev)}
        graphs[m] = Graph(o["ids"].data_ptr(), o["dist"].data_ptr(), o["deg"].data_ptr(), inp.N_out, R, 0)
        shard_ptrs[m] = ctypes.cast(inp._shards, ctypes.c_void_p)
        hs[m] = inp.h
        outs.append(o)
    check(L_.fgim_merge_batch(shard_ptrs, hs, n, ctypes.byref(p), graphs, _stream()))
    for m, o in enumerate(outs):
        o["entry"] = int(graphs[m].entry)
    return outs


def merge_host(X, adj, sizes, entries, k: int, R: int, alpha: float = 1.0, metric="l2", L: int = 0, iters: int = 3,
               rev_cap: int = 0, ensure_reachable: bool = True, out_ids=None, out_deg=None, join_filter="tc",
               rows="auto") -> dict:
    """Merge from host memory (CPU tensors, pinned for speed); results land in host tensors."""
    L_ = load()
    if X.is_cuda or adj.is_cuda:
        raise ValueError("merge_host takes host tensors")
    X = X.contiguous()
    adj = adj.contiguous()
    if X.dtype not in _VEC_DTYPES or adj.dtype != torch.int32:
        raise ValueError("X must be float32 or bfloat16 and adj int32")
    N = int(X.shape[0])
    p = Params()
    p.dim, p.dtype, p.metric = int(X.shape[1]), _VEC_DTYPES[X.dtype], _lib.METRICS[metric]
    p.k, p.R, p.alpha, p.L, p.iters, p.rev_cap, p.ensure_reachable = k, R, float(alpha), L, iters, rev_cap, int(
        bool(ensure_reachable))
    p.join_filter = JOIN_FILTERS[join_filter]
    p.byte_rows = ROW_STORAGE[rows]
    sz = (ctypes.c_int32 * len(sizes))(*[int(s) for s in sizes])
    en = (ctypes.c_int32 * len(entries))(*[int(e) for e in entries])
    if out_ids is None:
        out_ids = torch.empty((N, R), dtype=torch.int32).pin_memory()
    if out_deg is None:
        out_deg = torch.empty((N,), dtype=torch.int32).pin_memory()
    entry = ctypes.c_int32(0)
    check(L_.fgim_merge_host(_p(X), _p(adj), sz, en, len(sizes), int(adj.shape[1]), ctypes.byref(p), _p(out_ids),
                             _p(out_deg), ctypes.byref(entry), _stream()))
    return {"ids": out_ids, "deg": out_deg, "entry": int(entry.value), "stats": last_stats()}


def cross_query(inp: MergeInput, k: int, L: int = 0, rows="auto") -> dict:
    """Stage (a), Alg. 2: PGs -> k-NNG (one row per valid vertex)."""
    L_ = load()
    p = inp.params(k=k, L=L, rows=rows)
    kd = _new_knng(inp.N_out, k, inp.X.device)
    kn = _knng_struct(kd["ids"], kd["dist"], kd["flags"])
    check(L_.fgim_cross_query(inp._shards, inp.h, ctypes.byref(p), ctypes.byref(kn), _stream()))
    kd["stats"] = last_stats()
    return kd


def refine_pass(inp: MergeInput, knng: dict, rev_cap: int = 0, join_filter="tc", rows="auto") -> dict:
    """One synchronous Visit + Update pass of Alg. 3, in place on ``knng``."""
    L_ = load()
    k = int(knng["ids"].shape[1])
    p = inp.params(k=k, rev_cap=rev_cap, join_filter=join_filter, rows=rows)
    kn = _knng_struct(knng["ids"], knng["dist"], knng["flags"])
    check(L_.fgim_refine_pass(inp._shards, inp.h, ctypes.byref(p), ctypes.byref(kn), _stream()))
    return last_stats()


def indegree_repair(inp: MergeInput, knng: dict):
    """Alg. 4 in place on ``knng``; returns (T, stats)."""
    L_ = load()
    k = int(knng["ids"].shape[1])
    p = inp.params(k=k)
    T = torch.empty((inp.N,), dtype=torch.int32, device=inp.X.device)
    kn = _knng_struct(knng["ids"], knng["dist"], knng["flags"])
    check(L_.fgim_indegree_repair(inp._shards, inp.h, ctypes.byref(p), ctypes.byref(kn), _p(T), _stream()))
    return T, last_stats()


def prune(inp: MergeInput, knng: dict, T: torch.Tensor, R: int, alpha: float = 1.0, rows="auto", rule="arng",
          tau: float = 0.0):
    """Alg. 5 neighbour selection with `rule` (see merge): returns (e_ids [N, R], e_dist, e_cnt)."""
    L_ = load()
    k = int(knng["ids"].shape[1])
    p = inp.params(k=k, R=R, alpha=alpha, rows=rows, rule=rule, tau=tau)
    dev = inp.X.device
    e_ids = torch.empty((inp.N, R), dtype=torch.int32, device=dev)
    e_dist = torch.empty((inp.N, R), dtype=torch.float32, device=dev)
    e_cnt = torch.empty((inp.N,), dtype=torch.int32, device=dev)
    flags = knng.get("flags")
    if flags is None:
        flags = torch.zeros_like(knng["ids"], dtype=torch.uint8)
    kn = _knng_struct(knng["ids"], knng["dist"], flags)
    T = _dev(T, torch.int32, "T")
    check(L_.fgim_prune(inp._shards, inp.h, ctypes.byref(p), ctypes.byref(kn), _p(T), _p(e_ids), _p(e_dist),
                        _p(e_cnt), _stream()))
    return e_ids, e_dist, e_cnt


def reverse_insert(e_ids: torch.Tensor, e_dist: torch.Tensor, e_cnt: torch.Tensor) -> dict:
    """Alg. 5 connectivity enhancement."""
    L_ = load()
    N, R = int(e_ids.shape[0]), int(e_ids.shape[1])
    dev = e_ids.device
    out = {"ids": torch.empty((N, R), dtype=torch.int32, device=dev),
           "dist": torch.empty((N, R), dtype=torch.float32, device=dev),
           "deg": torch.empty((N,), dtype=torch.int32, device=dev)}
    g = Graph(out["ids"].data_ptr(), out["dist"].data_ptr(), out["deg"].data_ptr(), N, R, 0)
    check(L_.fgim_reverse_insert(N, R, _p(_dev(e_ids, torch.int32, "e_ids")), _p(_dev(e_dist, torch.float32, "e_dist")),
                                 _p(_dev(e_cnt, torch.int32, "e_cnt")), ctypes.byref(g), _stream()))
    return out


def reach_fix(inp: MergeInput, graph: dict, entry: int, k: int = 16, beam: int = 0, rows="auto") -> dict:
    """Reachability fix in place on ``graph`` (ids, dist, deg)."""
    L_ = load()
    R = int(graph["ids"].shape[1])
    p = inp.params(k=k, R=R, reach_beam=beam, rows=rows)
    g = Graph(graph["ids"].data_ptr(), graph["dist"].data_ptr(), graph["deg"].data_ptr(), inp.N, R, int(entry))
    check(L_.fgim_reach_fix(inp._shards, inp.h, ctypes.byref(p), ctypes.byref(g), _stream()))
    return last_stats()


def search(X: torch.Tensor, graph_ids: torch.Tensor, entry: int, queries: torch.Tensor, topk: int = 10,
           beam: int = 64, metric="l2"):
    """Alg. 1 over a merged graph: returns (ids [nq, topk], dist). X and queries are both float32
    or both bfloat16."""
    L_ = load()
    X = _vec(X, "X")
    Q = _vec(queries, "queries")
    if Q.dtype != X.dtype:
        raise ValueError("X and queries must have the same dtype")
    G = _dev(graph_ids, torch.int32, "graph_ids")
    nq = int(Q.shape[0])
    ids = torch.empty((nq, topk), dtype=torch.int32, device=X.device)
    dist = torch.empty((nq, topk), dtype=torch.float32, device=X.device)
    check(L_.fgim_search(_p(X), int(X.shape[0]), int(X.shape[1]), _VEC_DTYPES[X.dtype], _lib.METRICS[metric], _p(G),
                         int(G.shape[1]),
                         int(entry), _p(Q), nq, topk, beam, _p(ids), _p(dist), _stream()))
    return ids, dist


# --------------------------------------------------------------------------- HNSW-adaptive merging
def hnsw_levels(n: int, M: int, seed: int, device=None):
    """Levels of n vertices (SplitMix64 from `seed`, P(level >= l) = M^-l): (levels [n] int32
    device tensor, counts[l] = #{v : level >= l} for l = 0 .. MAX_LEVELS)."""
    L_ = load()
    dev = device or torch.device("cuda", torch.cuda.current_device())
    levels = torch.empty((n,), dtype=torch.int32, device=dev)
    counts = (ctypes.c_int64 * (_lib.MAX_LEVELS + 1))()
    check(L_.fgim_hnsw_levels(int(n), int(M), ctypes.c_uint64(seed & ((1 << 64) - 1)), _p(levels), counts,
                              _stream()))
    return levels, [int(x) for x in counts]


def hnsw_layer(X: torch.Tensor, levels: torch.Tensor, level: int, n_layer: int, M: int, ef: int = 64,
               metric="l2") -> dict:
    """Layer `level` >= 1 over the vertices of that level or higher (Sec. 4.3.3): members
    (ascending ids), adj [n_layer, M] (positions in members, -1 padded), deg."""
    L_ = load()
    X = _vec(X, "X")
    lv = _dev(levels, torch.int32, "levels")
    dev = X.device
    out = {"members": torch.empty((n_layer,), dtype=torch.int32, device=dev),
           "adj": torch.empty((n_layer, M), dtype=torch.int32, device=dev),
           "deg": torch.empty((n_layer,), dtype=torch.int32, device=dev)}
    check(L_.fgim_hnsw_layer(_p(X), int(X.shape[0]), int(X.shape[1]), _VEC_DTYPES[X.dtype], _lib.METRICS[metric],
                             _p(lv), int(level), int(M), int(ef), _p(out["members"]), _p(out["adj"]),
                             _p(out["deg"]), int(n_layer), _stream()))
    return out


def build_pg(X: torch.Tensor, M: int, ef: int = 64, metric="l2"):
    """An input PG for one shard on the GPU by batch-incremental insertion from the medoid (see
    fgim_build_pg): (adj [n, M] int32 local ids, -1 padded; entry = the medoid)."""
    L_ = load()
    X = _vec(X, "X")
    n = int(X.shape[0])
    adj = torch.empty((n, M), dtype=torch.int32, device=X.device)
    deg = torch.empty((n,), dtype=torch.int32, device=X.device)
    entry = ctypes.c_int32(0)
    check(L_.fgim_build_pg(_p(X), n, int(X.shape[1]), _VEC_DTYPES[X.dtype], _lib.METRICS[metric], int(M), int(ef),
                           _p(adj), _p(deg), ctypes.byref(entry), _stream()))
    return adj, int(entry.value)


def build_layers(X: torch.Tensor, M: int, ef: int = 64, seed: int = 0, metric="l2") -> dict:
    """All upper layers over the vertices of X: {levels, counts, layers (layer 1 first), entry}."""
    levels, counts = hnsw_levels(int(X.shape[0]), M, seed, X.device)
    layers = []
    for l in range(1, _lib.MAX_LEVELS + 1):
        if counts[l] == 0:
            break
        layers.append(hnsw_layer(X, levels, l, counts[l], M, ef, metric))
    top = len(layers)
    entry = int(torch.nonzero(levels == top)[0, 0]) if top else 0
    return {"levels": levels, "counts": counts, "layers": layers, "entry": entry}


def search_hnsw(X: torch.Tensor, graph_ids: torch.Tensor, layers: Sequence[dict], entry: int, queries: torch.Tensor,
                topk: int = 10, beam: int = 64, metric="l2", ef_up: int = 8):
    """The layered search: each upper layer searched with Alg. 1 (pool ef_up; 1 = greedy) from
    the top, then Alg. 1 on the base graph: (ids [nq, topk], dist, start [nq] = the base vertex
    each query started from)."""
    L_ = load()
    X = _vec(X, "X")
    Q = _vec(queries, "queries")
    if Q.dtype != X.dtype:
        raise ValueError("X and queries must have the same dtype")
    G = _dev(graph_ids, torch.int32, "graph_ids")
    nq = int(Q.shape[0])
    arr = (_lib.Layer * max(1, len(layers)))()
    for i, ly in enumerate(layers):
        arr[i] = _lib.Layer(ly["members"].data_ptr(), ly["adj"].data_ptr(), int(ly["members"].shape[0]),
                            int(ly["adj"].shape[1]), 0)
    ids = torch.empty((nq, topk), dtype=torch.int32, device=X.device)
    dist = torch.empty((nq, topk), dtype=torch.float32, device=X.device)
    start = torch.empty((nq,), dtype=torch.int32, device=X.device)
    check(L_.fgim_search_hnsw(_p(X), int(X.shape[0]), int(X.shape[1]), _VEC_DTYPES[X.dtype], _lib.METRICS[metric],
                              _p(G), int(G.shape[1]), arr, len(layers), int(entry), _p(Q), nq, topk, beam,
                              int(ef_up), _p(ids), _p(dist), _p(start), _stream()))
    return ids, dist, start


def autotune(inp: MergeInput, k: int, L: int = 0, cache_path: Optional[str] = None, rows="auto") -> dict:
    """Time the beam-search launch shapes on this merge's cross query and keep the fastest for
    its workload (see fgim_autotune): {"wpb", "ht_bits", "ms"}."""
    L_ = load()
    p = inp.params(k=k, L=L, rows=rows)
    wpb, hb, ms = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_float(0.0)
    check(L_.fgim_autotune(inp._shards, inp.h, ctypes.byref(p), cache_path.encode() if cache_path else None,
                           ctypes.byref(wpb), ctypes.byref(hb), ctypes.byref(ms), _stream()))
    return {"wpb": int(wpb.value), "ht_bits": int(hb.value), "ms": float(ms.value)}


def autotune_load(cache_path: str) -> None:
    check(load().fgim_autotune_load(cache_path.encode()))


def autotune_clear() -> None:
    load().fgim_autotune_clear()


def launch_count() -> int:
    return int(load().fgim_launch_count())


class profiling:
    """Context manager: per-kernel CUDA-event timing of every launch inside the block."""

    def __enter__(self):
        L_ = load()
        L_.fgim_prof_reset()
        L_.fgim_prof_enable(1)
        return self

    def __exit__(self, *exc):
        load().fgim_prof_enable(0)

    @staticmethod
    def names():
        L_ = load()
        n = L_.fgim_prof_names(None, 0)
        buf = ctypes.create_string_buffer(n + 1)
        L_.fgim_prof_names(buf, n + 1)
        return [x for x in buf.value.decode().split(",") if x]

    @staticmethod
    def query(kernel: str):
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0.0)
        load().fgim_prof_query(kernel.encode(), ctypes.byref(n), ctypes.byref(ms))
        return int(n.value), float(ms.value)
