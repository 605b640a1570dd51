"""Seeded synthetic workloads for the FGIM merge path.

This module only draws random vectors and splits them into shards. It holds
none of the merge method's arithmetic: the input proximity graphs come from
``synth.pgbuild`` (a separate incremental builder), and everything the merge
computes lives either in ``oracle/`` (CPU reference) or in the CUDA library.

The recipes stand in for the real datasets the paper evaluates on (Sec. 5.1,
Table "dataset"): Sift1M (128-d integers, Euclidean), Deep1M (96-d, cosine),
Gist1M (960-d, Euclidean) and the 768-d Internet Search set. None of those
datasets is used; only their shapes and metrics are imitated.

Global ids follow the ID mapping phi of Sec. 4.1.3 as plain offsets: shard i
occupies rows [offset_i, offset_i + n_i) of ``X``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

MASTER_SEED = 20260321

METRIC_L2 = 0
METRIC_IP = 1
METRIC_COS = 2


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray            # [N, d] float32, phi order (BF16-representable values when dtype == "bf16")
    Q: np.ndarray            # [nq, d] float32 queries from the same distribution
    shard_sizes: List[int]
    metric: int
    M: int                   # max degree of each input PG
    ef: int                  # build pool of each input PG
    k: int                   # k of the merged k-NNG
    R: int                   # degree bound of the merged PG
    alpha: float
    perm: np.ndarray         # original index of each phi-ordered row
    dtype: str = "f32"

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    @property
    def h(self) -> int:
        return len(self.shard_sizes)

    @property
    def offsets(self) -> List[int]:
        o = [0]
        for s in self.shard_sizes:
            o.append(o[-1] + s)
        return o

    def shard(self, i: int) -> np.ndarray:
        o = self.offsets
        return self.X[o[i]:o[i + 1]]

    def bits(self) -> np.ndarray:
        """The stored BF16 encodings of X (exact: X holds BF16-representable values)."""
        assert self.dtype == "bf16"
        return (self.X.view(np.uint32) >> 16).astype(np.uint16)


def _streams(seed: int, n: int = 4):
    ss = np.random.SeedSequence(seed)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(n)]


def _split(rng, N: int, sizes: List[int]):
    assert sum(sizes) == N
    return rng.permutation(N)


def _mixture(rng_pts, centers: np.ndarray, n: int, sigma, chunk: int = 1 << 16) -> np.ndarray:
    """n points: a uniformly chosen center plus isotropic/anisotropic Gaussian noise."""
    c, d = centers.shape
    out = np.empty((n, d), dtype=np.float64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        comp = rng_pts.integers(0, c, size=e - s)
        noise = rng_pts.standard_normal((e - s, d))
        sig = sigma if np.isscalar(sigma) else sigma[comp]
        out[s:e] = centers[comp] + noise * sig
    return out


def small(seed: int = MASTER_SEED, N: int = 20_000, d: int = 32, h: int = 2, nq: int = 1000) -> Workload:
    """50-component isotropic mixture, centers U[-10,10], sigma 1, squared L2."""
    r_c, r_p, r_s, r_q = _streams(seed)
    centers = r_c.uniform(-10.0, 10.0, size=(50, d))
    X = _mixture(r_p, centers, N, 1.0).astype(np.float32)
    Q = _mixture(r_q, centers, nq, 1.0).astype(np.float32)
    sizes = _equal_sizes(N, h)
    perm = _split(r_s, N, sizes)
    return Workload("small", np.ascontiguousarray(X[perm]), Q, sizes, METRIC_L2,
                    M=16, ef=64, k=16, R=32, alpha=1.2, perm=perm)


def medium(seed: int = MASTER_SEED, N: int = 1_000_000, d: int = 128, h: int = 4, nq: int = 10_000,
           n_centers: int = 1000) -> Workload:
    """Sift-like: 1,000 centers U[0,255]^d, per-dim sigma 20, clipped to [0,255] and rounded."""
    r_c, r_p, r_s, r_q = _streams(seed)
    centers = r_c.uniform(0.0, 255.0, size=(n_centers, d))

    def draw(rng, n):
        return np.rint(np.clip(_mixture(rng, centers, n, 20.0), 0.0, 255.0)).astype(np.float32)

    X = draw(r_p, N)
    Q = draw(r_q, nq)
    sizes = _equal_sizes(N, h)
    perm = _split(r_s, N, sizes)
    return Workload("medium", np.ascontiguousarray(X[perm]), Q, sizes, METRIC_L2,
                    M=32, ef=128, k=64, R=32, alpha=1.2, perm=perm)


def precision(seed: int = MASTER_SEED, N: int = 1_000_000, d: int = 96, h: int = 2, nq: int = 10_000,
              n_centers: int = 2000, sigma: float = 0.5) -> Workload:
    """Deep-like: 2,000 centers N(0,I), noise sigma 0.5 (unstated in the recipe), L2-normalised; IP."""
    r_c, r_p, r_s, r_q = _streams(seed)
    centers = r_c.standard_normal((n_centers, d))

    def draw(rng, n):
        x = _mixture(rng, centers, n, sigma)
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        return x.astype(np.float32)

    X = draw(r_p, N)
    Q = draw(r_q, nq)
    sizes = _equal_sizes(N, h)
    perm = _split(r_s, N, sizes)
    return Workload("precision", np.ascontiguousarray(X[perm]), Q, sizes, METRIC_IP,
                    M=32, ef=128, k=48, R=32, alpha=1.0, perm=perm)


def fp8(seed: int = MASTER_SEED, N: int = 1_000_000, d: int = 960, nq: int = 10_000,
        n_centers: int = 1000) -> Workload:
    """Gist-like: |mixture| with centers U[0,0.3]^d, sigma 0.05; 8 shards sized i*N/36."""
    r_c, r_p, r_s, r_q = _streams(seed)
    centers = r_c.uniform(0.0, 0.3, size=(n_centers, d))

    def draw(rng, n):
        return np.abs(_mixture(rng, centers, n, 0.05)).astype(np.float32)

    X = draw(r_p, N)
    Q = draw(r_q, nq)
    sizes = [(i * N) // 36 for i in range(1, 9)]
    sizes[-1] += N - sum(sizes)
    perm = _split(r_s, N, sizes)
    return Workload("fp8", np.ascontiguousarray(X[perm]), Q, sizes, METRIC_L2,
                    M=32, ef=128, k=64, R=48, alpha=1.0, perm=perm)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest BF16 value (round to nearest, ties to even), returned as float32.

    Storage step of the batched recipe; the inputs are finite, so the NaN case is not handled.
    """
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (b.astype(np.uint32) << 16).view(np.float32)


def batched_one(seed: int = MASTER_SEED, N: int = 20_000, h: int = 3, d: int = 768, nq: int = 1000,
                n_centers: int = 500) -> Workload:
    """One merge of the batched form: 500 centers N(0, I_d), per-cluster per-dimension sigma
    U[0.1, 1.0] (anisotropic; the spread is not given, this is the stated reading), normalised,
    stored in BF16 (round to nearest even); cosine. Shards: a random split, sizes as equal as
    possible."""
    r_c, r_p, r_s, r_q = _streams(seed)
    centers = r_c.standard_normal((n_centers, d))
    sig = r_c.uniform(0.1, 1.0, size=(n_centers, d))

    def draw(rng, n):
        x = _mixture(rng, centers, n, sig)
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        return bf16_round(x.astype(np.float32))

    X = draw(r_p, N)
    Q = draw(r_q, nq)
    sizes = _equal_sizes(N, h)
    perm = _split(r_s, N, sizes)
    return Workload("batched", np.ascontiguousarray(X[perm]), Q, sizes, METRIC_COS,
                    M=24, ef=96, k=32, R=24, alpha=1.0, perm=perm, dtype="bf16")


def batched(seed: int = MASTER_SEED, n_merges: int = 64, n_lo: int = 10_000, n_hi: int = 200_000, d: int = 768,
            nq: int = 1000) -> List[Workload]:
    """The batched form: n_merges independent merges, h ~ U{2..6}, total size log-uniform in
    [n_lo, n_hi]; each merge drawn by ``batched_one`` from its own seed."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 4])))
    hs = rng.integers(2, 7, size=n_merges)
    Ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=n_merges)).astype(np.int64)
    seeds = rng.integers(0, 2**31 - 1, size=n_merges)
    return [batched_one(int(seeds[m]), N=int(Ns[m]), h=int(hs[m]), d=d, nq=nq) for m in range(n_merges)]


def _equal_sizes(N: int, h: int) -> List[int]:
    base = N // h
    sizes = [base] * h
    for i in range(N - base * h):
        sizes[i] += 1
    return sizes


RECIPES = {"small": small, "medium": medium, "precision": precision, "fp8": fp8, "batched_one": batched_one}


def make(name: str, seed: int = MASTER_SEED, **kw) -> Workload:
    return RECIPES[name](seed=seed, **kw)

