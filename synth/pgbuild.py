"""ctypes front end of ``pgbuild.c`` (input proximity graphs, built on the host)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pgbuild.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libpgbuild.so")
_lock = threading.Lock()
_lib = None


def compile_lib(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(compile_lib())
            lib.pg_build.restype = ctypes.c_int
            lib.pg_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p]
            _lib = lib
    return _lib


def build_pg(X: np.ndarray, M: int, ef: int, metric: int, max_batch: int = 1024, threads: int = 0):
    """Build one input PG over the rows of X. Returns (adj [n, M] int32 padded -1, entry)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, d = X.shape
    adj = np.empty((n, M), dtype=np.int32)
    entry = np.zeros(1, dtype=np.int32)
    rc = _load().pg_build(X.ctypes.data, n, d, metric, M, ef, max_batch, threads,
                          adj.ctypes.data, entry.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"pg_build failed with {rc}")
    return adj, int(entry[0])


def build_all(w, threads: int = 0):
    """Input PGs of every shard of workload ``w``: list of (adj, entry) in shard order."""
    return [build_pg(w.shard(i), w.M, w.ef, w.metric, threads=threads) for i in range(w.h)]
