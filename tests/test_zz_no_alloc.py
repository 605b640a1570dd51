"""fgim_search_noalloc, the search for callers that cannot allocate device memory.

Serving processes whose device memory is owned by a pool they do not control, latency-
critical paths that may not allocate, and plug-ins inside hosts that forbid allocator calls
use this entry point; its scratch is a fixed array inside the library. These tests call it
through the C ABI and compare it with fgim_search (same kernel, so the outputs must agree
within the suite's tolerance; in practice bit for bit), twice in a row because every call
reuses the same array. The file sorts last so that a stop-at-first-failure run has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests import _parity as PR  # noqa: E402


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_21710_gb300 as fg
    from synth import gen, pgbuild
    dev = torch.device("cuda:0")
    w = gen.make("small", N=6000, nq=300)
    graphs = pgbuild.build_all(w)
    X = torch.from_numpy(w.X).to(dev)
    adj = torch.from_numpy(np.concatenate([g[0] for g in graphs])).to(dev)
    inp = fg.MergeInput.from_flat(X, w.shard_sizes, adj, [g[1] for g in graphs])
    out = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2)
    Q = torch.from_numpy(w.Q).to(dev)
    return fg, X, out, Q


def _call(L, fn, X, G, entry, Q, metric, topk=10, beam=64):
    nq = int(Q.shape[0])
    ids = torch.full((nq, topk), -7, dtype=torch.int32, device=X.device)
    dist = torch.full((nq, topk), -7.0, dtype=torch.float32, device=X.device)
    st = getattr(L, fn)(ctypes.c_void_p(X.data_ptr()), int(X.shape[0]), int(X.shape[1]), 0, metric,
                        ctypes.c_void_p(G.data_ptr()), int(G.shape[1]), int(entry), ctypes.c_void_p(Q.data_ptr()), nq,
                        topk, beam, ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dist.data_ptr()),
                        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, ids.cpu().numpy(), dist.cpu().numpy()


@pytest.mark.parametrize("metric", [0, 1, 2])
def test_noalloc_search_matches_search_twice(metric):
    fg, X, out, Q = _setup()
    L = fg.load()
    st, ref_ids, ref_dist = _call(L, "fgim_search", X, out["ids"], out["entry"], Q, metric)
    assert st == 0
    for _ in range(2):
        st, ids, dist = _call(L, "fgim_search_noalloc", X, out["ids"], out["entry"], Q, metric)
        assert st == 0
        assert len(PR.lists_match(ids, dist, ref_ids, ref_dist)) == 0
        assert np.array_equal(ids, ref_ids)


def test_noalloc_search_rejects_oversized_cosine_before_any_work():
    fg, X, out, Q = _setup()
    L = fg.load()
    ids = torch.empty((1, 10), dtype=torch.int32, device=X.device)
    dist = torch.empty((1, 10), dtype=torch.float32, device=X.device)
    st = L.fgim_search_noalloc(ctypes.c_void_p(X.data_ptr()), (1 << 20) + 1, int(X.shape[1]), 0, 2,
                               ctypes.c_void_p(out["ids"].data_ptr()), int(out["ids"].shape[1]), 0,
                               ctypes.c_void_p(Q.data_ptr()), 1, 10, 64, ctypes.c_void_p(ids.data_ptr()),
                               ctypes.c_void_p(dist.data_ptr()), torch.cuda.current_stream().cuda_stream)
    assert st == -1   # FGIM_EINVAL
