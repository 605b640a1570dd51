"""Python front end of the FGIM merge oracle (``fgim_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``. The product path never imports it.

All arrays are host numpy arrays; see ``fgim_oracle.h`` for the layouts.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fgim_oracle.c")
_HDR = os.path.join(_HERE, "fgim_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libfgim_oracle.so")
_lock = threading.Lock()
_lib = None

FLAG_NEW = 1
FLAG_REPLACED = 2

_i32p = ctypes.c_void_p
_c = ctypes


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("ndc", "hops", "pairs", "updates", "zero_before", "zero_after", "replaced",
                 "prune_dist", "unreached", "attached")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class _Input(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("N", ctypes.c_int64), ("d", ctypes.c_int32),
                ("metric", ctypes.c_int32), ("h", ctypes.c_int32), ("off", ctypes.c_void_p),
                ("adj", ctypes.c_void_p), ("M", ctypes.c_int32), ("entry", ctypes.c_void_p),
                ("nthreads", ctypes.c_int32), ("valid", ctypes.c_void_p)]


def compile_lib(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(compile_lib())
            vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
            sig = {
                "or_delta64": (ctypes.c_double, [vp, vp, i32, i32]),
                "or_delta": (f32, [vp, vp, i32, i32]),
                "or_knn_search": (i32, [vp, i64, i32, i32, vp, i32, i32, vp, i32, i32, vp, vp, vp]),
                "or_knn_exact": (None, [vp, i64, i32, i32, vp, i64, vp, i32, i32, vp, vp]),
                "or_stage_a": (i32, [vp, i32, i32, vp, vp, vp, vp]),
                "or_refine_iter": (None, [vp, i32, i32, vp, vp, vp, vp]),
                "or_indegree_repair": (None, [vp, i32, vp, vp, vp, vp, vp]),
                "or_indegree": (None, [vp, i64, i32, vp]),
                "or_prune": (None, [vp, i32, vp, vp, vp, i32, f32, vp, vp, vp, vp]),
                "or_prune_rule": (None, [vp, i32, vp, vp, vp, i32, i32, f32, f32, vp, vp, vp, vp]),
                "or_merge_rule": (i32, [vp, i32, i32, i32, i32, i32, i32, f32, f32, i32, vp, vp, vp, vp, vp, vp,
                                        vp]),
                "or_reverse_insert": (None, [i64, i32, vp, vp, vp, vp, vp, vp]),
                "or_reach_fix": (None, [vp, i32, i32, i32, vp, vp, vp, vp]),
                "or_merged_entry": (i32, [vp]),
                "or_phi": (i64, [vp, vp]),
                "or_knn_prefix": (None, [vp, i64, i32, i32, i32, i32, vp, vp]),
                "or_refine_dfs": (None, [vp, i32, i32, vp, vp, vp, vp, vp]),
                "or_merge": (i32, [vp, i32, i32, i32, i32, i32, f32, i32, vp, vp, vp, vp, vp, vp, vp]),
                "or_search": (None, [vp, i64, i32, i32, vp, i32, i32, vp, i64, i32, i32, i32, vp, vp, vp]),
                "or_hnsw_insert": (None, [vp, i64, i32, i32, vp, i32, i32, i32, vp, vp, vp]),
                "or_reach_fix_seq": (None, [vp, i32, i32, i32, vp, i32, vp, vp, vp, vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


@dataclass
class Problem:
    """The merge input: vectors in shard order plus the h input PGs (local ids), and optionally
    the validity of every vertex (the boolean part of phi, Sec. 4.1.3)."""
    X: np.ndarray          # [N, d] float32
    sizes: List[int]
    adj: np.ndarray        # [N, M] int32 local ids
    entry: np.ndarray      # [h] int32 local
    metric: int
    nthreads: int = 0
    valid: Optional[np.ndarray] = None   # [N] bool / uint8; None = every vertex valid

    def __post_init__(self):
        self.X = np.ascontiguousarray(self.X, dtype=np.float32)
        self.adj = np.ascontiguousarray(self.adj, dtype=np.int32)
        self.entry = np.ascontiguousarray(self.entry, dtype=np.int32)
        if self.valid is not None:
            self.valid = np.ascontiguousarray(self.valid, dtype=np.uint8)
            assert self.valid.shape == (self.X.shape[0],)
        off = [0]
        for s in self.sizes:
            off.append(off[-1] + int(s))
        self.off = np.asarray(off, dtype=np.int64)
        assert self.off[-1] == self.X.shape[0] == self.adj.shape[0]
        self._in = _Input(self.X.ctypes.data, self.X.shape[0], self.X.shape[1], self.metric, len(self.sizes),
                          self.off.ctypes.data, self.adj.ctypes.data, self.adj.shape[1],
                          self.entry.ctypes.data, self.nthreads, _p(self.valid))

    @property
    def N(self):
        return int(self.X.shape[0])

    @property
    def N_valid(self) -> int:
        return self.N if self.valid is None else int(np.count_nonzero(self.valid))

    def phi(self) -> np.ndarray:
        """[N] global id of every vertex in the merged index, -1 for invalid ones."""
        out = np.empty(self.N, np.int32)
        lib().or_phi(self.ref, out.ctypes.data)
        return out

    def compact(self) -> "Problem":
        """The valid vertices alone, renumbered by phi: the problem stages (b) and (c) see.
        Its input PGs are not carried (those stages do not read them)."""
        keep = np.ones(self.N, bool) if self.valid is None else self.valid.astype(bool)
        sizes = [int(np.count_nonzero(keep[self.off[i]:self.off[i + 1]])) for i in range(self.h)]
        Nv = int(sum(sizes))
        return Problem(self.X[keep], sizes, np.full((Nv, 1), -1, np.int32), np.zeros(self.h, np.int32),
                       self.metric, self.nthreads)

    @property
    def h(self):
        return len(self.sizes)

    @property
    def ref(self):
        return ctypes.byref(self._in)

    @staticmethod
    def from_workload(w, graphs: Sequence[Tuple[np.ndarray, int]], nthreads: int = 0) -> "Problem":
        adj = np.concatenate([g[0] for g in graphs], axis=0)
        entry = np.asarray([g[1] for g in graphs], dtype=np.int32)
        return Problem(w.X, list(w.shard_sizes), adj, entry, w.metric, nthreads)


def delta(x: np.ndarray, y: np.ndarray, metric: int) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    return float(lib().or_delta(x.ctypes.data, y.ctypes.data, x.shape[0], metric))


def knn_search(X_local, adj_local, ep, q, L, k, metric):
    X_local = np.ascontiguousarray(X_local, dtype=np.float32)
    adj_local = np.ascontiguousarray(adj_local, dtype=np.int32)
    q = np.ascontiguousarray(q, dtype=np.float32)
    ids = np.full(k, -1, np.int32)
    dist = np.full(k, np.inf, np.float32)
    st = Stats()
    r = lib().or_knn_search(X_local.ctypes.data, X_local.shape[0], X_local.shape[1], metric, adj_local.ctypes.data,
                            adj_local.shape[1], ep, q.ctypes.data, L, k, ids.ctypes.data, dist.ctypes.data,
                            ctypes.byref(st))
    return ids[:r], dist[:r], st.as_dict()


def knn_exact(X, Q, k, metric, exclude=None, nthreads=0):
    X = np.ascontiguousarray(X, dtype=np.float32)
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    nq = Q.shape[0]
    ids = np.empty((nq, k), np.int32)
    dist = np.empty((nq, k), np.float32)
    ex = None if exclude is None else np.ascontiguousarray(exclude, dtype=np.int64)
    lib().or_knn_exact(X.ctypes.data, X.shape[0], X.shape[1], metric, Q.ctypes.data, nq, _p(ex), k, nthreads,
                       ids.ctypes.data, dist.ctypes.data)
    return ids, dist


class KNNG:
    def __init__(self, N, k):
        self.ids = np.full((N, k), -1, np.int32)
        self.dist = np.full((N, k), np.inf, np.float32)
        self.flags = np.zeros((N, k), np.uint8)

    def copy(self):
        c = KNNG.__new__(KNNG)
        c.ids, c.dist, c.flags = self.ids.copy(), self.dist.copy(), self.flags.copy()
        return c


def stage_a(P: Problem, k: int, L: int = 0):
    """Alg. 2; with validity the k-NNG has one row per valid vertex, in phi order."""
    g = KNNG(P.N_valid, k)
    st = Stats()
    Lu = lib().or_stage_a(P.ref, k, L, g.ids.ctypes.data, g.dist.ctypes.data, g.flags.ctypes.data, ctypes.byref(st))
    return g, int(Lu), st.as_dict()


def refine_iter(P: Problem, g: KNNG, rev_cap: int = 0):
    """One synchronous Visit + Update pass, in place on ``g``."""
    k = g.ids.shape[1]
    st = Stats()
    lib().or_refine_iter(P.ref, k, rev_cap, g.ids.ctypes.data, g.dist.ctypes.data, g.flags.ctypes.data,
                         ctypes.byref(st))
    return st.as_dict()


def refine_dfs(P: Problem, g: KNNG, iters: int):
    """Alg. 3 as printed (DFS order, streamlined Visit + Update, lists updated at once), each
    iteration followed by Alg. 4; in place on ``g``. Returns (T, stats)."""
    k = g.ids.shape[1]
    T = np.empty(P.N, np.int32)
    st = Stats()
    lib().or_refine_dfs(P.ref, k, iters, g.ids.ctypes.data, g.dist.ctypes.data, g.flags.ctypes.data, T.ctypes.data,
                        ctypes.byref(st))
    return T, st.as_dict()


def indegree(ids: np.ndarray) -> np.ndarray:
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    T = np.empty(ids.shape[0], np.int32)
    lib().or_indegree(ids.ctypes.data, ids.shape[0], ids.shape[1], T.ctypes.data)
    return T


def indegree_repair(P: Problem, g: KNNG):
    k = g.ids.shape[1]
    T = np.empty(P.N, np.int32)
    st = Stats()
    lib().or_indegree_repair(P.ref, k, g.ids.ctypes.data, g.dist.ctypes.data, g.flags.ctypes.data, T.ctypes.data,
                             ctypes.byref(st))
    return T, st.as_dict()


PRUNE_RULES = {"arng": 0, "mrng": 1, "tmng": 2, 0: 0, 1: 1, 2: 2}


def prune(P: Problem, g: KNNG, T: np.ndarray, R: int, alpha: float, rule="arng", tau: float = 0.0):
    """Alg. 5 neighbour selection with the rule `rule` ("arng" alpha-RNG, "mrng", "tmng" tau-MNG)."""
    k = g.ids.shape[1]
    T = np.ascontiguousarray(T, dtype=np.int32)
    e_ids = np.empty((P.N, R), np.int32)
    e_dist = np.empty((P.N, R), np.float32)
    e_cnt = np.empty(P.N, np.int32)
    st = Stats()
    lib().or_prune_rule(P.ref, k, g.ids.ctypes.data, g.dist.ctypes.data, T.ctypes.data, R, PRUNE_RULES[rule], alpha,
                        tau, e_ids.ctypes.data, e_dist.ctypes.data, e_cnt.ctypes.data, ctypes.byref(st))
    return e_ids, e_dist, e_cnt, st.as_dict()


def reverse_insert(e_ids, e_dist, e_cnt):
    N, R = e_ids.shape
    e_ids = np.ascontiguousarray(e_ids, dtype=np.int32)
    e_dist = np.ascontiguousarray(e_dist, dtype=np.float32)
    e_cnt = np.ascontiguousarray(e_cnt, dtype=np.int32)
    o_ids = np.empty((N, R), np.int32)
    o_dist = np.empty((N, R), np.float32)
    o_deg = np.empty(N, np.int32)
    lib().or_reverse_insert(N, R, e_ids.ctypes.data, e_dist.ctypes.data, e_cnt.ctypes.data, o_ids.ctypes.data,
                            o_dist.ctypes.data, o_deg.ctypes.data)
    return o_ids, o_dist, o_deg


def reach_fix(P: Problem, o_ids, o_dist, o_deg, entry, beam: int = 64):
    """In place on (o_ids, o_dist, o_deg)."""
    R = o_ids.shape[1]
    st = Stats()
    lib().or_reach_fix(P.ref, R, entry, beam, o_ids.ctypes.data, o_dist.ctypes.data, o_deg.ctypes.data,
                       ctypes.byref(st))
    return st.as_dict()


def reach_fix_seq(P: Problem, o_ids, o_dist, o_deg, entry, beam: int = 64, knn_ids=None):
    """The plain sequential reachability fix, in place (the quality reference for reach_fix)."""
    R = o_ids.shape[1]
    kn = None if knn_ids is None else np.ascontiguousarray(knn_ids, dtype=np.int32)
    st = Stats()
    lib().or_reach_fix_seq(P.ref, R, entry, beam, _p(kn), 0 if kn is None else kn.shape[1], o_ids.ctypes.data,
                           o_dist.ctypes.data, o_deg.ctypes.data, ctypes.byref(st))
    return st.as_dict()


def merged_entry(P: Problem) -> int:
    """Entry of the merged graph (a global id after phi)."""
    return int(lib().or_merged_entry(P.ref))


@dataclass
class MergeResult:
    ids: np.ndarray
    dist: np.ndarray
    deg: np.ndarray
    entry: int
    knn_ids: np.ndarray
    knn_dist: np.ndarray
    L: int
    stats: dict


def merge(P: Problem, k: int, R: int, alpha: float, L: int = 0, iters: int = 3, rev_cap: int = 0,
          ensure_reachable: bool = True, rule="arng", tau: float = 0.0) -> MergeResult:
    if P.valid is not None:
        return _merge_valid(P, k, R, alpha, L, iters, rev_cap, ensure_reachable, rule, tau)
    N = P.N
    o_ids = np.empty((N, R), np.int32)
    o_dist = np.empty((N, R), np.float32)
    o_deg = np.empty(N, np.int32)
    entry = np.zeros(1, np.int32)
    k_ids = np.empty((N, k), np.int32)
    k_dist = np.empty((N, k), np.float32)
    st = Stats()
    Lu = lib().or_merge_rule(P.ref, k, L, iters, rev_cap, R, PRUNE_RULES[rule], alpha, tau, int(ensure_reachable),
                             o_ids.ctypes.data, o_dist.ctypes.data, o_deg.ctypes.data, entry.ctypes.data,
                             k_ids.ctypes.data, k_dist.ctypes.data, ctypes.byref(st))
    return MergeResult(o_ids, o_dist, o_deg, int(entry[0]), k_ids, k_dist, int(Lu), st.as_dict())


def _merge_valid(P: Problem, k, R, alpha, L, iters, rev_cap, ensure_reachable, rule="arng", tau=0.0) -> MergeResult:
    """The merge with invalid vertices: Alg. 2 over the input PGs with phi dropping invalid
    vertices, then the stages of ``or_merge`` in the same order on the valid vertices alone."""
    g, Lu, st = stage_a(P, k, L)
    Pc = P.compact()
    T = None
    for _ in range(iters):
        refine_iter(Pc, g, rev_cap)
        T, _ = indegree_repair(Pc, g)
    if iters <= 0:
        T = indegree(g.ids)
    e_ids, e_dist, e_cnt, _ = prune(Pc, g, T, R, alpha, rule, tau)
    o_ids, o_dist, o_deg = reverse_insert(e_ids, e_dist, e_cnt)
    entry = merged_entry(P)
    if ensure_reachable:
        reach_fix(Pc, o_ids, o_dist, o_deg, entry, 64)
    return MergeResult(o_ids, o_dist, o_deg, entry, g.ids.copy(), g.dist.copy(), Lu, st)


def search(X, g_ids, entry, Q, beam, topk, metric, nthreads=0):
    X = np.ascontiguousarray(X, dtype=np.float32)
    g_ids = np.ascontiguousarray(g_ids, dtype=np.int32)
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    nq = Q.shape[0]
    ids = np.empty((nq, topk), np.int32)
    dist = np.empty((nq, topk), np.float32)
    st = Stats()
    lib().or_search(X.ctypes.data, X.shape[0], X.shape[1], metric, g_ids.ctypes.data, g_ids.shape[1], entry,
                    Q.ctypes.data, nq, beam, topk, nthreads, ids.ctypes.data, dist.ctypes.data, ctypes.byref(st))
    return ids, dist, st.as_dict()


def recall_at(found: np.ndarray, truth: np.ndarray, k: int) -> float:
    """Recall@k (Sec. 2.1): |R intersect R~| / k averaged over queries."""
    hits = 0
    for f, t in zip(found[:, :k], truth[:, :k]):
        hits += len(set(int(x) for x in f if x >= 0) & set(int(x) for x in t if x >= 0))
    return hits / (k * found.shape[0])


# --------------------------------------------------------------------------- HNSW-adaptive merging
# Sec. 4.3.3: upper layers rebuilt over the merged base graph. Every vertex draws a level from
# HNSW's distribution, P(level >= l) = M^-l (mL = 1 / ln M). Readings (each one also in the
# design notes): the level of v comes from the v-th output of SplitMix64 seeded with `seed`
# (its published definition: state += 0x9E3779B97F4A7C15, then the two xor-shift-multiply
# rounds), as the number of l >= 1 with r_v < floor((2^64 - 1) / M^l); each layer l is built
# from its own vertices at once instead of by one-at-a-time insertion: the exact ef nearest
# members inserted before it in id order (the limit of HNSW's candidate search at insertion:
# early members link far, as in HNSW), the RNG heuristic down to M (Alg. 5's rule with
# alpha = 1 and no indegree clause), bidirectional edges, and the same heuristic over the
# union of a member's own and reverse edges (its 128 nearest when larger).
_GAMMA = 0x9E3779B97F4A7C15
_U64 = (1 << 64) - 1
MAX_LEVELS = 16


def splitmix64(seed: int, i: int) -> int:
    """The i-th output (i >= 0) of SplitMix64 started from state `seed`."""
    z = (seed + (i + 1) * _GAMMA) & _U64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _U64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _U64
    return z ^ (z >> 31)


def level_thresholds(M: int, max_level: int = MAX_LEVELS) -> List[int]:
    """T_l = floor((2^64 - 1) / M^l) for l = 1 .. while M^l < 2^64 (at most max_level)."""
    out, p = [], M
    while len(out) < max_level and p <= _U64:
        out.append(_U64 // p)
        p *= M
    return out


def hnsw_levels(n: int, M: int, seed: int) -> np.ndarray:
    T = level_thresholds(M)
    lv = np.zeros(n, np.int32)
    for v in range(n):
        r = splitmix64(seed, v)
        lv[v] = sum(1 for t in T if r < t)
    return lv


def hnsw_layer(X: np.ndarray, metric: int, levels: np.ndarray, level: int, M: int, ef: int):
    """Layer `level` >= 1: (members [n_l] ascending global ids, adj [n_l, M] positions in
    members, -1 padded, deg [n_l])."""
    members = np.nonzero(levels >= level)[0].astype(np.int32)
    n = len(members)
    if n == 0:
        return members, np.zeros((0, M), np.int32), np.zeros(0, np.int32)
    Xl = np.ascontiguousarray(X[members], dtype=np.float32)
    Pl = Problem(Xl, [n], np.full((n, 1), -1, np.int32), np.zeros(1, np.int32), metric)
    kk = min(ef, max(n - 1, 1))
    ids = np.empty((n, kk), np.int32)
    dist = np.empty((n, kk), np.float32)
    lib().or_knn_prefix(Xl.ctypes.data, n, Xl.shape[1], metric, kk, 0, ids.ctypes.data, dist.ctypes.data)
    g = KNNG(n, kk)
    g.ids[:], g.dist[:] = ids, dist
    T = np.full(n, 2, np.int32)   # the indegree clause never fires
    e_ids, e_dist, e_cnt, _ = prune(Pl, g, T, M, 1.0)
    wide = 128   # the union of own and reverse edges (its 128 nearest if larger)
    pad_i = np.full((n, wide), -1, np.int32)
    pad_d = np.full((n, wide), np.inf, np.float32)
    pad_i[:, :M], pad_d[:, :M] = e_ids, e_dist
    u_ids, u_dist, u_deg = reverse_insert(pad_i, pad_d, e_cnt)
    g2 = KNNG(n, wide)
    g2.ids[:], g2.dist[:] = u_ids, u_dist
    f_ids, f_dist, f_cnt, _ = prune(Pl, g2, T, M, 1.0)
    return members, f_ids, f_cnt


def hnsw_entry(levels: np.ndarray) -> int:
    """The first vertex of the highest level."""
    return int(np.argmax(levels))


def hnsw_search(X, metric, base_ids, layers, entry, Q, beam, topk, ef_up: int = 8):
    """The layered search: from the entry (top layer) down, each upper layer is searched with
    Alg. 1 (pool ef_up; ef_up = 1 is HNSW's greedy descent) from the vertex the layer above
    gave, its nearest result starting the next layer; then Alg. 1 on the base graph from the
    vertex reached. layers[l - 1] = (members, adj) of layer l."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    rows = [np.ascontiguousarray(X[m]) for m, _ in layers]
    out_i = np.empty((len(Q), topk), np.int32)
    out_d = np.empty((len(Q), topk), np.float32)
    starts = np.empty(len(Q), np.int32)
    for qi, q in enumerate(np.ascontiguousarray(Q, dtype=np.float32)):
        cur = entry
        for (members, adj), Xl in zip(reversed(layers), reversed(rows)):
            if len(members) == 0:
                continue
            pos = int(np.searchsorted(members, cur))
            if pos >= len(members) or members[pos] != cur:
                continue
            i, _, _ = search(Xl, adj, pos, q[None], ef_up, 1, metric)
            cur = int(members[i[0][0]])
        starts[qi] = cur
        i, d, _ = search(X, base_ids, cur, q[None], beam, topk, metric)
        out_i[qi], out_d[qi] = i[0], d[0]
    return out_i, out_d, starts


def build_pg(X: np.ndarray, metric: int, M: int, ef: int):
    """An input PG built like one HNSW layer over every vertex (the vertices in id order):
    (adj [n, M] local ids, -1 padded, entry 0). The GPU input-PG builder's definition."""
    n = X.shape[0]
    _, adj, _ = hnsw_layer(X, metric, np.ones(n, np.int32), 1, M, ef)
    return adj, 0


def hnsw_insert_layers(X: np.ndarray, metric: int, levels: np.ndarray, M: int, ef: int):
    """The upper layers as HNSW's sequential insertion builds them (the literal form of Sec.
    4.3.3, the quality reference for ``hnsw_layer``): ([(members, adj positions, deg) per layer
    1 .. top], entry)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    N = X.shape[0]
    top = int(lv.max()) if N else 0
    if top < 1:
        return [], 0
    adj = np.empty((top, N, M), np.int32)
    entry = np.zeros(1, np.int32)
    st = Stats()
    lib().or_hnsw_insert(X.ctypes.data, N, X.shape[1], metric, lv.ctypes.data, top, M, ef, adj.ctypes.data,
                         entry.ctypes.data, ctypes.byref(st))
    layers = []
    for l in range(1, top + 1):
        members = np.nonzero(lv >= l)[0].astype(np.int32)
        pos = np.full(N, -1, np.int32)
        pos[members] = np.arange(len(members), dtype=np.int32)
        A = adj[l - 1][members]
        P = np.where(A >= 0, pos[np.maximum(A, 0)], -1).astype(np.int32)
        layers.append((members, P, (P >= 0).sum(1).astype(np.int32)))
    return layers, int(entry[0])
