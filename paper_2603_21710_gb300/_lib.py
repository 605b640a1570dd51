"""ctypes declarations of the C ABI in include/fgim.h and the loader of libfgim.so.

The library is the only compute path: if it cannot be built or loaded, every call
raises. There is no CPU or PyTorch fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_lock = threading.Lock()
_lib = None

FGIM_OK, FGIM_EINVAL, FGIM_ENOMEM, FGIM_ECUDA, FGIM_ETIMEOUT, FGIM_EUNSUPPORTED, FGIM_EINTERNAL = 0, -1, -2, -3, -4, -5, -6
METRICS = {"l2": 0, "ip": 1, "cos": 2, 0: 0, 1: 1, 2: 2}


class Shard(ctypes.Structure):
    _fields_ = [("vectors", ctypes.c_void_p), ("adj", ctypes.c_void_p), ("n", ctypes.c_int32),
                ("max_degree", ctypes.c_int32), ("entry", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("valid", ctypes.c_void_p)]


class Layer(ctypes.Structure):
    _fields_ = [("members", ctypes.c_void_p), ("adj", ctypes.c_void_p), ("n", ctypes.c_int64), ("M", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


MAX_LEVELS = 16


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("dtype", ctypes.c_int32), ("metric", ctypes.c_int32),
                ("k", ctypes.c_int32), ("R", ctypes.c_int32), ("alpha", ctypes.c_float), ("L", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("rev_cap", ctypes.c_int32), ("ensure_reachable", ctypes.c_int32),
                ("reach_beam", ctypes.c_int32), ("join_filter", ctypes.c_int32), ("byte_rows", ctypes.c_int32),
                ("prune_rule", ctypes.c_int32), ("tau", ctypes.c_float), ("reserved", ctypes.c_int32)]


class KNNG(ctypes.Structure):
    _fields_ = [("ids", ctypes.c_void_p), ("dist", ctypes.c_void_p), ("flags", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("k", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Graph(ctypes.Structure):
    _fields_ = [("ids", ctypes.c_void_p), ("dist", ctypes.c_void_p), ("deg", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("R", ctypes.c_int32), ("entry", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("ndc", "hops", "join_pairs", "proposals", "zero_indegree",
                                              "repaired", "attached", "unreached", "join_reruns", "join_cands")] + [
        ("join_class", ctypes.c_int64 * 5)]

    def as_dict(self):
        d = {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "join_class"}
        d["join_class"] = [int(x) for x in self.join_class]
        return d


class FgimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fgim status {status}: {msg}")
        self.status = status


EXPORTS = {
    "fgim_trim_memory": (None, []),
    "fgim_merge": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "fgim_merge_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "fgim_merge_host": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                                ctypes.c_void_p]),
    "fgim_cross_query": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "fgim_refine_pass": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "fgim_indegree_repair": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "fgim_prune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fgim_reverse_insert": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fgim_reach_fix": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "fgim_search": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fgim_hnsw_levels": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "fgim_hnsw_layer": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "fgim_search_hnsw": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fgim_build_pg": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "fgim_search_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fgim_last_stats": (None, [ctypes.c_void_p]),
    "fgim_graph_alloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]),
    "fgim_graph_free": (None, [ctypes.c_void_p]),
    "fgim_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_char_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fgim_autotune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "fgim_autotune_clear": (None, []),
    "fgim_test_set": (ctypes.c_int32, [ctypes.c_char_p, ctypes.c_int64]),
    "fgim_test_get": (ctypes.c_int64, [ctypes.c_char_p]),
    "fgim_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "fgim_last_error": (ctypes.c_char_p, []),
    "fgim_version": (ctypes.c_char_p, []),
    "fgim_launch_count": (ctypes.c_int64, []),
    "fgim_prof_enable": (None, [ctypes.c_int32]),
    "fgim_prof_reset": (None, []),
    "fgim_prof_query": (ctypes.c_int32, [ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fgim_prof_names": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
}


def lib_path() -> str:
    from . import build as _build
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load libfgim.so (compiling it first when sources are newer). Raises if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        path = _build.build() if build_if_stale else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"FGIM CUDA library missing at {path}; build it with __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int):
    if status != FGIM_OK:
        L = load()
        raise FgimError(status, f"{L.fgim_strerror(status).decode()}: {L.fgim_last_error().decode()}")


def last_stats() -> dict:
    s = Stats()
    load().fgim_last_stats(ctypes.byref(s))
    return s.as_dict()


def test_set(knob: str, value: int) -> None:
    """Set one of the library's test hooks (see fgim_test_set in fgim.h)."""
    if load().fgim_test_set(knob.encode(), int(value)) != 1:
        raise KeyError(knob)


def test_get(what: str) -> int:
    return int(load().fgim_test_get(what.encode()))
