"""GPU parity: the CUDA path through the C ABI against the CPU oracle, stage by stage.

Each stage receives the SAME input on both sides (the oracle's output of the previous
stage), so the comparison isolates one kernel family. Exact stages must satisfy the
list rule of tests/_parity.py; the approximate stage (beam search) must give
bit-identical rows for almost every query and the same recall within 0.5 point.
"""
import numpy as np
import pytest

import oracle as O
from tests import _parity as PR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _inp(w, graphs):
    import paper_2603_21710_gb300 as fg
    dev = _dev()
    X = torch.from_numpy(w.X).to(dev)
    adj = torch.from_numpy(np.concatenate([g[0] for g in graphs])).to(dev)
    return fg.MergeInput.from_flat(X, w.shard_sizes, adj, [g[1] for g in graphs],
                                   metric={0: "l2", 1: "ip", 2: "cos"}[w.metric])


def _to_dev(g: "O.KNNG"):
    dev = _dev()
    return {"ids": torch.from_numpy(g.ids.copy()).to(dev), "dist": torch.from_numpy(g.dist.copy()).to(dev),
            "flags": torch.from_numpy(g.flags.copy()).to(dev)}


def _np(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def small(small_problem):
    w, graphs, P = small_problem
    return w, graphs, P, _inp(w, graphs)


@pytest.fixture(scope="module")
def sift_like():
    """Sift-like recipe (integer values 0..255, d=128, 4 shards) at N=40,000: FP32 sums are exact."""
    from synth import gen, pgbuild
    w = gen.make("medium", N=40_000, nq=500, n_centers=40)
    graphs = pgbuild.build_all(w)
    P = O.Problem.from_workload(w, graphs)
    return w, graphs, P, _inp(w, graphs)


@pytest.fixture(scope="module")
def high_dim():
    """The d = 960 recipe (non-negative floats, 8 shards sized 1..8) at N = 6,000: the join's
    Gram tile accumulates eight 128-dimension K chunks."""
    from synth import gen, pgbuild
    w = gen.make("fp8", N=6_000, nq=100)
    graphs = pgbuild.build_all(w)
    P = O.Problem.from_workload(w, graphs)
    return w, graphs, P, _inp(w, graphs)


# --------------------------------------------------------------------------- stage (a)
def test_cross_query_small(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    g = fg.cross_query(inp, w.k)
    o, L, _ = O.stage_a(P, w.k)
    gi, gd = _np(g["ids"]), _np(g["dist"])
    PR.check_lists(gi, gd, w.N)
    assert np.all(_np(g["flags"])[gi >= 0] == fg.FLAG_NEW)
    same = np.all(gi == o.ids, 1).mean()
    assert same >= 0.99, same
    # where the ids agree, distances agree within the FP32 tolerance
    m = gi == o.ids
    assert np.all(PR.close(gd[m], o.dist[m]))
    rng = np.random.default_rng(3)
    samp = rng.choice(w.N, 1000, replace=False)
    tid, _ = O.knn_exact(w.X, w.X[samp], w.k, w.metric, exclude=samp)
    assert abs(O.recall_at(gi[samp], tid, w.k) - O.recall_at(o.ids[samp], tid, w.k)) <= 0.005


def test_cross_query_integer_data_bit_exact(sift_like):
    """Integer inputs make every FP32 partial sum exact: the GPU rows equal the oracle's bit for bit."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    g = fg.cross_query(inp, w.k)
    o, L, ost = O.stage_a(P, w.k)
    assert L == 22
    assert np.array_equal(_np(g["ids"]), o.ids)
    assert np.array_equal(_np(g["dist"]), o.dist)
    # the GPU's lossy visited table may re-evaluate, never skip: its count is >= the oracle's
    assert g["stats"]["ndc"] >= ost["ndc"]


# --------------------------------------------------------------------------- stage (b)
def test_refine_pass_small(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    o, _, _ = O.stage_a(P, w.k)
    g = _to_dev(o)
    st = fg.refine_pass(inp, g)
    O.refine_iter(P, o)
    bad = PR.lists_match(_np(g["ids"]), _np(g["dist"]), o.ids, o.dist)
    assert len(bad) == 0, bad[:10]
    same = np.all(_np(g["ids"]) == o.ids, 1)
    assert np.array_equal(_np(g["flags"])[same], o.flags[same])
    assert st["join_pairs"] > 0


def test_refine_pass_integer_bit_exact(sift_like):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    o, _, _ = O.stage_a(P, w.k)
    g = _to_dev(o)
    st = fg.refine_pass(inp, g)
    ost = O.refine_iter(P, o)
    assert np.array_equal(_np(g["ids"]), o.ids)
    assert np.array_equal(_np(g["dist"]), o.dist)
    assert np.array_equal(_np(g["flags"]), o.flags)
    assert st["join_pairs"] == ost["pairs"]
    # a second pass (only new entries join) stays identical too
    fg.refine_pass(inp, g)
    O.refine_iter(P, o)
    assert np.array_equal(_np(g["ids"]), o.ids)


def test_refine_pass_small_rev_cap(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    o, _, _ = O.stage_a(P, w.k)
    g = _to_dev(o)
    fg.refine_pass(inp, g, rev_cap=3)
    O.refine_iter(P, o, rev_cap=3)
    assert len(PR.lists_match(_np(g["ids"]), _np(g["dist"]), o.ids, o.dist)) == 0


def test_indegree_repair_exact(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    o, _, _ = O.stage_a(P, w.k)
    O.refine_iter(P, o)
    g = _to_dev(o)
    T, st = fg.indegree_repair(inp, g)
    To, ost = O.indegree_repair(P, o)
    assert ost["zero_before"] > 0
    assert st["zero_indegree"] == ost["zero_before"]
    assert st["repaired"] == ost["replaced"]
    assert np.array_equal(_np(T), To)
    assert np.array_equal(_np(g["ids"]), o.ids)
    assert np.array_equal(_np(g["dist"]), o.dist)
    assert np.array_equal(_np(g["flags"]), o.flags)


# --------------------------------------------------------------------------- stage (c)
def _refined(P, w, iters=2):
    o, _, _ = O.stage_a(P, w.k)
    T = None
    for _ in range(iters):
        O.refine_iter(P, o)
        T, _ = O.indegree_repair(P, o)
    return o, T


def test_prune_small(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    o, T = _refined(P, w)
    ei, ed, ec = fg.prune(inp, _to_dev(o), torch.from_numpy(T).to(_dev()), w.R, w.alpha)
    oi, od, oc, _ = O.prune(P, o, T, w.R, w.alpha)
    ei, ed, ec = _np(ei), _np(ed), _np(ec)
    diff = np.nonzero(~np.all(ei == oi, 1))[0]
    assert len(diff) <= max(2, w.N // 2000), len(diff)
    for u in diff:
        # a differing row must contain an occlusion test that ties within tolerance
        cand = o.ids[u][o.ids[u] >= 0]
        assert PR.prune_row_has_near_tie(w.X, u, cand, o.dist[u][:len(cand)], w.alpha), u
    same = np.all(ei == oi, 1)
    assert np.array_equal(ed[same], od[same]) and np.array_equal(ec[same], oc[same])


def test_prune_integer_bit_exact(sift_like):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    o, T = _refined(P, w, iters=1)
    ei, ed, ec = fg.prune(inp, _to_dev(o), torch.from_numpy(T).to(_dev()), w.R, w.alpha)
    oi, od, oc, _ = O.prune(P, o, T, w.R, w.alpha)
    assert np.array_equal(_np(ei), oi) and np.array_equal(_np(ed), od) and np.array_equal(_np(ec), oc)


@pytest.mark.parametrize("which", ["high_dim", "bf16_batch"])
def test_prune_wide_rows(which, request):
    """Rows wider than 128 (d = 960 L2, d = 768 cosine): the warp-cooperative prune keeps the
    oracle's lists except where an occlusion test ties within tolerance."""
    import paper_2603_21710_gb300 as fg
    if which == "high_dim":
        w, graphs, P, inp = request.getfixturevalue("high_dim")
    else:
        w, graphs, P = request.getfixturevalue("bf16_batch")[2]
        inp = _inp_bf16(w, graphs)
    assert w.d > 128
    o, T = _refined(P, w, iters=1)
    ei, ed, ec = fg.prune(inp, _to_dev(o), torch.from_numpy(T).to(_dev()), w.R, w.alpha)
    oi, od, oc, _ = O.prune(P, o, T, w.R, w.alpha)
    ei, ed, ec = _np(ei), _np(ed), _np(ec)
    diff = np.nonzero(~np.all(ei == oi, 1))[0]
    assert len(diff) <= max(2, w.N // 2000), len(diff)
    for u in diff:
        cand = o.ids[u][o.ids[u] >= 0]
        assert PR.prune_row_has_near_tie(w.X, u, cand, o.dist[u][:len(cand)], w.alpha, metric=w.metric), u
    same = np.all(ei == oi, 1)
    assert np.array_equal(ed[same], od[same]) and np.array_equal(ec[same], oc[same])


def test_reverse_insert_exact(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    o, T = _refined(P, w, iters=1)
    oi, od, oc, _ = O.prune(P, o, T, w.R, w.alpha)
    dev = _dev()
    out = fg.reverse_insert(torch.from_numpy(oi).to(dev), torch.from_numpy(od).to(dev), torch.from_numpy(oc).to(dev))
    ri, rd, rg = O.reverse_insert(oi, od, oc)
    assert np.array_equal(_np(out["ids"]), ri)
    assert np.array_equal(_np(out["dist"]), rd)
    assert np.array_equal(_np(out["deg"]), rg)


def test_reach_fix_small(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    o, T = _refined(P, w, iters=1)
    oi, od, oc, _ = O.prune(P, o, T, w.R, w.alpha)
    ri, rd, rg = O.reverse_insert(oi, od, oc)
    entry = O.merged_entry(P)
    assert not PR.bfs_reached(ri, entry).all(), "the small workload is disconnected before the fix"
    dev = _dev()
    g = {"ids": torch.from_numpy(ri.copy()).to(dev), "dist": torch.from_numpy(rd.copy()).to(dev),
         "deg": torch.from_numpy(rg.copy()).to(dev)}
    st = fg.reach_fix(inp, g, entry, k=w.k)
    ost = O.reach_fix(P, ri, rd, rg, entry)
    gi = _np(g["ids"])
    assert st["unreached"] == 0 and ost["unreached"] == 0
    assert PR.bfs_reached(gi, entry).all()
    assert st["attached"] == ost["attached"]
    assert np.all(gi == ri, 1).mean() >= 0.999
    PR.check_lists(gi, _np(g["dist"]), w.N)


# --------------------------------------------------------------------------- end to end
def test_merge_small_end_to_end(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    out = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=3, return_knng=True)
    ref = O.merge(P, w.k, w.R, w.alpha, iters=3)
    gi, gd, gdeg = _np(out["ids"]), _np(out["dist"]), _np(out["deg"])
    PR.check_lists(gi, gd, w.N)
    assert np.all(gdeg <= w.R) and np.array_equal(gdeg, (gi >= 0).sum(1))
    assert out["entry"] == ref.entry
    assert out["stats"]["unreached"] == 0 and PR.bfs_reached(gi, out["entry"]).all()
    # k-NNG recall against exact k-NN on a sample, and search recall@10 at beam 64
    rng = np.random.default_rng(9)
    samp = rng.choice(w.N, 1000, replace=False)
    tid, _ = O.knn_exact(w.X, w.X[samp], w.k, w.metric, exclude=samp)
    kg = _np(out["knng"]["ids"])
    assert abs(O.recall_at(kg[samp], tid, w.k) - O.recall_at(ref.knn_ids[samp], tid, w.k)) <= 0.005
    gt, _ = O.knn_exact(w.X, w.Q, 10, w.metric)
    sg, _ = fg.search(inp.X, out["ids"], out["entry"], torch.from_numpy(w.Q).to(_dev()), topk=10, beam=64)
    so, _, _ = O.search(w.X, ref.ids, ref.entry, w.Q, 64, 10, w.metric)
    assert abs(O.recall_at(_np(sg), gt, 10) - O.recall_at(so, gt, 10)) <= 0.005


def test_merge_integer_bit_exact(sift_like):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    out = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2, return_knng=True)
    ref = O.merge(P, w.k, w.R, w.alpha, iters=2)
    assert np.array_equal(_np(out["knng"]["ids"]), ref.knn_ids)
    assert np.array_equal(_np(out["ids"]), ref.ids)
    assert np.array_equal(_np(out["deg"]), ref.deg)


def test_search_parity(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    ref = O.merge(P, w.k, w.R, w.alpha, iters=1)
    dev = _dev()
    sg, sd = fg.search(inp.X, torch.from_numpy(ref.ids).to(dev), ref.entry, torch.from_numpy(w.Q).to(dev), 10, 64)
    so, sdo, _ = O.search(w.X, ref.ids, ref.entry, w.Q, 64, 10, w.metric)
    sg = _np(sg)
    assert np.all(sg == so, 1).mean() >= 0.99
    gt, _ = O.knn_exact(w.X, w.Q, 10, w.metric)
    assert abs(O.recall_at(sg, gt, 10) - O.recall_at(so, gt, 10)) <= 0.005


def test_merge_host_matches_device(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    X = torch.from_numpy(w.X).pin_memory()
    adj = torch.from_numpy(np.concatenate([g[0] for g in graphs])).pin_memory()
    h = fg.merge_host(X, adj, w.shard_sizes, [g[1] for g in graphs], k=w.k, R=w.R, alpha=w.alpha, iters=1)
    d = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=1)
    assert np.array_equal(h["ids"].numpy(), _np(d["ids"]))
    assert h["entry"] == d["entry"]


def test_deterministic_repeat(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    a = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2)
    b = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2)
    assert torch.equal(a["ids"], b["ids"]) and torch.equal(a["dist"], b["dist"])


# --------------------------------------------------------------------------- edge cases
def _tiny(seed, sizes, d, M, metric=0):
    from synth import pgbuild
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((sum(sizes), d)).astype(np.float32)
    if metric == 1:
        X /= np.linalg.norm(X, axis=1, keepdims=True)
    gs, o = [], 0
    for n in sizes:
        gs.append(pgbuild.build_pg(X[o:o + n], M, 32, metric))
        o += n
    return X, gs


@pytest.mark.parametrize("sizes,d,M,k,R,metric", [
    ([3, 5], 8, 4, 6, 4, 0),            # shards smaller than k: padded lists
    ([700, 300, 257], 36, 40, 12, 10, 0),  # ragged K tail (d=36), two adjacency chunks (M=40), h=3
    ([500, 500], 96, 16, 48, 32, 1),    # inner product, k=48
    ([1, 400], 16, 8, 8, 8, 0),         # a one-point shard
])
def test_edge_cases_match_oracle(sizes, d, M, k, R, metric):
    import paper_2603_21710_gb300 as fg
    X, gs = _tiny(sum(sizes) + d, sizes, d, M, metric)
    P = O.Problem(X, sizes, np.concatenate([g[0] for g in gs]), np.array([g[1] for g in gs], np.int32), metric)
    dev = _dev()
    inp = fg.MergeInput.from_flat(torch.from_numpy(X).to(dev), sizes,
                                  torch.from_numpy(np.concatenate([g[0] for g in gs])).to(dev),
                                  [g[1] for g in gs], metric=metric)
    ga = fg.cross_query(inp, k)
    oa, _, _ = O.stage_a(P, k)
    assert np.all(_np(ga["ids"]) == oa.ids, 1).mean() >= 0.98
    g = _to_dev(oa)
    fg.refine_pass(inp, g)
    O.refine_iter(P, oa)
    assert len(PR.lists_match(_np(g["ids"]), _np(g["dist"]), oa.ids, oa.dist)) == 0
    out = fg.merge(inp, k=k, R=R, alpha=1.0, iters=2)
    gi = _np(out["ids"])
    PR.check_lists(gi, _np(out["dist"]), sum(sizes))
    assert PR.bfs_reached(gi, out["entry"]).all()


def test_reach_fix_victim_rule():
    """Every search candidate is full: the farthest neighbour with indegree > 1 is replaced (as in the oracle)."""
    import json
    import os
    import paper_2603_21710_gb300 as fg
    gd = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "reach_victim.json")))
    pos = np.asarray(gd["pos"], np.float32)
    X = np.zeros((len(pos), 4), np.float32)
    X[:, 0] = pos
    R = gd["R"]
    ids = np.asarray(gd["lists"], np.int32)
    deg = (ids >= 0).sum(1).astype(np.int32)
    dist = np.full(ids.shape, np.inf, np.float32)
    for u in range(len(pos)):
        for t in range(deg[u]):
            dist[u, t] = (pos[u] - pos[ids[u, t]]) ** 2
    dev = _dev()
    adj = torch.full((len(pos), 2), -1, dtype=torch.int32, device=dev)
    inp = fg.MergeInput.from_flat(torch.from_numpy(X).to(dev), [2, 2], adj, [0, 0])
    g = {"ids": torch.from_numpy(ids.copy()).to(dev), "dist": torch.from_numpy(dist).to(dev),
         "deg": torch.from_numpy(deg).to(dev)}
    st = fg.reach_fix(inp, g, gd["entry"], k=2)
    assert _np(g["ids"]).tolist() == gd["expected_lists"]
    assert _np(g["dist"])[2].tolist() == gd["expected_dist_row2"]
    assert st["attached"] == 1 and st["unreached"] == 0


@pytest.mark.parametrize("which", ["small", "sift_like"])
def test_join_filters_agree(which, request):
    """The BF16 tensor-core filter and the FP32 SIMT filter re-rank exactly: identical lists."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = request.getfixturevalue(which)
    o, _, _ = O.stage_a(P, w.k)
    a, b = _to_dev(o), _to_dev(o)
    sa = fg.refine_pass(inp, a, join_filter="tc")
    sb = fg.refine_pass(inp, b, join_filter="fp32")
    assert torch.equal(a["ids"], b["ids"]) and torch.equal(a["dist"], b["dist"]) and torch.equal(a["flags"], b["flags"])
    assert sa["join_pairs"] == sb["join_pairs"]
    ma = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2, join_filter="tc")
    mb = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2, join_filter="fp32")
    assert torch.equal(ma["ids"], mb["ids"])


def test_byte_rows_equal_fp32_rows(sift_like):
    """Integer data in [0, 255]: the byte-row stages (searches, join re-rank, prune) give the
    FP32-row results bit for bit, stage by stage and for the whole merge."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    ka = fg.cross_query(inp, w.k, rows="auto")
    kb = fg.cross_query(inp, w.k, rows="fp32")
    for key in ("ids", "dist", "flags"):
        assert torch.equal(ka[key], kb[key]), key
    assert ka["stats"]["ndc"] == kb["stats"]["ndc"]
    fg.refine_pass(inp, ka, rows="auto")
    fg.refine_pass(inp, kb, rows="fp32")
    for key in ("ids", "dist", "flags"):
        assert torch.equal(ka[key], kb[key]), key
    T, _ = fg.indegree_repair(inp, ka)
    ea = fg.prune(inp, ka, T, w.R, w.alpha, rows="auto")
    eb = fg.prune(inp, ka, T, w.R, w.alpha, rows="fp32")
    for x, y in zip(ea, eb):
        assert torch.equal(x, y)
    ma = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2, rows="auto")
    mb = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2, rows="fp32", join_filter="fp32")
    assert torch.equal(ma["ids"], mb["ids"]) and torch.equal(ma["deg"], mb["deg"])
    assert ma["entry"] == mb["entry"]


@pytest.mark.parametrize("join_filter", ["tc", "fp32"])
def test_refine_pass_high_dim(high_dim, join_filter):
    """d = 960: the tensor-core filter over eight K chunks, and the FP32 tile reading its rows
    from global memory (they do not fit shared memory), keep the oracle's lists."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = high_dim
    assert w.d == 960
    o, _, _ = O.stage_a(P, w.k)
    g = _to_dev(o)
    st = fg.refine_pass(inp, g, join_filter=join_filter)
    O.refine_iter(P, o)
    bad = PR.lists_match(_np(g["ids"]), _np(g["dist"]), o.ids, o.dist)
    assert len(bad) == 0, bad[:10]
    assert st["join_pairs"] > 0


def test_merge_high_dim(high_dim):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = high_dim
    out = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2)
    gi = _np(out["ids"])
    PR.check_lists(gi, _np(out["dist"]), w.N)
    assert PR.bfs_reached(gi, out["entry"]).all()


# --------------------------------------------------------------------------- BF16 storage, batches
@pytest.fixture(scope="module")
def bf16_batch():
    """Three merges of the batched form (d = 768, cosine, BF16 storage) at 2,000..4,000 points."""
    from synth import gen, pgbuild
    out = []
    for w in gen.batched(n_merges=3, n_lo=2_000, n_hi=4_000, nq=1000):
        graphs = pgbuild.build_all(w)
        out.append((w, graphs, O.Problem.from_workload(w, graphs)))
    return out


def _inp_bf16(w, graphs):
    import paper_2603_21710_gb300 as fg
    dev = _dev()
    Xb = torch.from_numpy(w.bits().view(np.int16)).to(dev).view(torch.bfloat16)
    adj = torch.from_numpy(np.concatenate([g[0] for g in graphs])).to(dev)
    return fg.MergeInput.from_flat(Xb, w.shard_sizes, adj, [g[1] for g in graphs], metric="cos")


def test_bf16_storage_decodes_exactly(bf16_batch):
    """BF16 storage is decoded to the FP32 values it encodes: the merge equals the FP32 merge of
    those values bit for bit, and its k-NNG stages keep the oracle's lists on them."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P = bf16_batch[0]
    ib = _inp_bf16(w, graphs)
    assert ib.X.dtype == torch.bfloat16
    i32 = _inp(w, graphs)
    a = fg.merge(ib, k=w.k, R=w.R, alpha=w.alpha, iters=2, return_knng=True)
    b = fg.merge(i32, k=w.k, R=w.R, alpha=w.alpha, iters=2, return_knng=True)
    assert torch.equal(a["ids"], b["ids"]) and torch.equal(a["dist"], b["dist"])
    assert torch.equal(a["knng"]["ids"], b["knng"]["ids"]) and a["entry"] == b["entry"]
    # stage (b) on the BF16 input against the oracle on the decoded values
    o, _, _ = O.stage_a(P, w.k)
    g = _to_dev(o)
    fg.refine_pass(ib, g)
    O.refine_iter(P, o)
    bad = PR.lists_match(_np(g["ids"]), _np(g["dist"]), o.ids, o.dist)
    assert len(bad) == 0, bad[:10]
    # search over BF16 base and queries equals search over their FP32 values
    Qb = torch.from_numpy((w.Q.view(np.uint32) >> 16).astype(np.uint16).view(np.int16)).to(_dev()).view(torch.bfloat16)
    sa, da = fg.search(ib.X, a["ids"], a["entry"], Qb, topk=10, beam=64, metric="cos")
    sb, db = fg.search(i32.X, a["ids"], a["entry"], torch.from_numpy(w.Q).to(_dev()), topk=10, beam=64, metric="cos")
    assert torch.equal(sa, sb) and torch.equal(da, db)


def test_merge_bf16_end_to_end(bf16_batch):
    """The whole merge on BF16 cosine input: valid lists, every vertex reachable, k-NNG and
    search recall within 0.5 point of the oracle's merge."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P = bf16_batch[1]
    ib = _inp_bf16(w, graphs)
    out = fg.merge(ib, k=w.k, R=w.R, alpha=w.alpha, iters=3, return_knng=True)
    ref = O.merge(P, w.k, w.R, w.alpha, iters=3)
    gi = _np(out["ids"])
    PR.check_lists(gi, _np(out["dist"]), w.N)
    assert PR.bfs_reached(gi, out["entry"]).all()
    assert out["entry"] == ref.entry
    samp = np.random.default_rng(5).choice(w.N, 500, replace=False)
    tid, _ = O.knn_exact(w.X, w.X[samp], w.k, w.metric, exclude=samp)
    kg = _np(out["knng"]["ids"])
    assert abs(O.recall_at(kg[samp], tid, w.k) - O.recall_at(ref.knn_ids[samp], tid, w.k)) <= 0.005
    gt, _ = O.knn_exact(w.X, w.Q, 10, w.metric)
    sg, _ = fg.search(_inp(w, graphs).X, out["ids"], out["entry"], torch.from_numpy(w.Q).to(_dev()), topk=10,
                      beam=64, metric="cos")
    so, _, _ = O.search(w.X, ref.ids, ref.entry, w.Q, 64, 10, w.metric)
    assert w.Q.shape[0] >= 1000
    assert abs(O.recall_at(_np(sg), gt, 10) - O.recall_at(so, gt, 10)) <= 0.005


def test_merge_batch_equals_single_merges(bf16_batch):
    """fgim_merge_batch gives each merge exactly what a call of its own gives."""
    import paper_2603_21710_gb300 as fg
    inps = [_inp_bf16(w, graphs) for w, graphs, _ in bf16_batch]
    w0 = bf16_batch[0][0]
    outs = fg.merge_batch(inps, k=w0.k, R=w0.R, alpha=w0.alpha, iters=2)
    assert len(outs) == len(inps)
    for inp, o in zip(inps, outs):
        s = fg.merge(inp, k=w0.k, R=w0.R, alpha=w0.alpha, iters=2)
        assert torch.equal(o["ids"], s["ids"]) and torch.equal(o["dist"], s["dist"])
        assert torch.equal(o["deg"], s["deg"]) and o["entry"] == s["entry"]
    assert fg.merge_batch([], k=w0.k, R=w0.R) == []


# --------------------------------------------------------------------------- validity (phi, Sec. 4.1.3)
def _masks(w, seed=11, frac=0.75):
    """About frac of the vertices valid; the entry of the largest shard invalid (the merged
    entry then falls back to that shard's first valid vertex)."""
    rng = np.random.default_rng(seed)
    valid = rng.random(w.N) < frac
    off = np.cumsum([0] + list(w.shard_sizes))
    return valid, off


def _masked_inputs(w, graphs, valid):
    import paper_2603_21710_gb300 as fg
    dev = _dev()
    X = torch.from_numpy(w.X).to(dev)
    adj = torch.from_numpy(np.concatenate([g[0] for g in graphs])).to(dev)
    inp = fg.MergeInput.from_flat(X, w.shard_sizes, adj, [g[1] for g in graphs],
                                  metric={0: "l2", 1: "ip", 2: "cos"}[w.metric],
                                  valid=torch.from_numpy(valid).to(dev))
    P = O.Problem.from_workload(w, graphs)
    Pv = O.Problem(P.X, P.sizes, P.adj, P.entry, P.metric, valid=valid)
    return inp, Pv


def test_masked_cross_query_bit_exact(sift_like):
    """Integer data: with invalid vertices the cross query equals the oracle's bit for bit."""
    import paper_2603_21710_gb300 as fg
    w, graphs, _, _ = sift_like
    valid, off = _masks(w)
    inp, Pv = _masked_inputs(w, graphs, valid)
    assert inp.N_out == int(valid.sum())
    g = fg.cross_query(inp, w.k)
    o, _, _ = O.stage_a(Pv, w.k)
    assert np.array_equal(_np(g["ids"]), o.ids)
    assert np.array_equal(_np(g["dist"]), o.dist)


def test_masked_merge_bit_exact(sift_like):
    """The whole merge with invalid vertices (one of them a shard entry) equals the oracle's."""
    import paper_2603_21710_gb300 as fg
    w, graphs, _, _ = sift_like
    valid, off = _masks(w, seed=12)
    big = int(np.argmax(w.shard_sizes))
    valid[off[big] + graphs[big][1]] = False
    inp, Pv = _masked_inputs(w, graphs, valid)
    out = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2, return_knng=True)
    ref = O.merge(Pv, w.k, w.R, w.alpha, iters=2)
    assert out["ids"].shape[0] == int(valid.sum())
    assert np.array_equal(_np(out["knng"]["ids"]), ref.knn_ids)
    assert np.array_equal(_np(out["ids"]), ref.ids)
    assert np.array_equal(_np(out["deg"]), ref.deg)
    assert out["entry"] == ref.entry
    assert PR.bfs_reached(_np(out["ids"]), out["entry"]).all()


def test_fully_invalid_shard_equals_merge_without_it(sift_like):
    """A shard with no valid vertex changes nothing: with the same L the merge equals the merge
    of the other shards (GPU against GPU, and against the oracle, bit for bit on integer data)."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    dev = _dev()
    n3 = int(sum(w.shard_sizes[:3]))
    valid = np.ones(w.N, bool)
    valid[n3:] = False
    masked, Pv = _masked_inputs(w, graphs, valid)
    a = fg.merge(masked, k=w.k, R=w.R, alpha=w.alpha, L=22, iters=2, return_knng=True)
    X = torch.from_numpy(w.X[:n3]).to(dev)
    adj = torch.from_numpy(np.concatenate([g[0] for g in graphs[:3]])).to(dev)
    three = fg.MergeInput.from_flat(X, w.shard_sizes[:3], adj, [g[1] for g in graphs[:3]])
    b = fg.merge(three, k=w.k, R=w.R, alpha=w.alpha, L=22, iters=2, return_knng=True)
    assert a["ids"].shape[0] == n3
    assert torch.equal(a["knng"]["ids"], b["knng"]["ids"]) and torch.equal(a["ids"], b["ids"])
    assert a["entry"] == b["entry"]
    ref = O.merge(Pv, w.k, w.R, w.alpha, L=22, iters=2)
    assert np.array_equal(_np(a["ids"]), ref.ids) and a["entry"] == ref.entry


def test_masks_rejected_where_not_honoured(small):
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    dev = _dev()
    X = torch.from_numpy(w.X).to(dev)
    adj = torch.from_numpy(np.concatenate([g[0] for g in graphs])).to(dev)
    none = fg.MergeInput.from_flat(X, w.shard_sizes, adj, [g[1] for g in graphs],
                                   valid=torch.zeros(w.N, dtype=torch.bool, device=dev))
    with pytest.raises(fg.FgimError) as e:
        fg.merge(none, k=w.k, R=w.R)
    assert e.value.status == -1
    some = fg.MergeInput.from_flat(X, w.shard_sizes, adj, [g[1] for g in graphs],
                                   valid=torch.ones(w.N, dtype=torch.bool, device=dev))
    o, _, _ = O.stage_a(P, w.k)
    with pytest.raises(fg.FgimError) as e:
        fg.refine_pass(some, _to_dev(o))
    assert e.value.status == -5


# --------------------------------------------------------------------------- HNSW-adaptive merging
def test_hnsw_levels_match_oracle():
    import paper_2603_21710_gb300 as fg
    _dev()
    lv, counts = fg.hnsw_levels(20_000, 8, seed=1234)
    ref = O.hnsw_levels(20_000, 8, seed=1234)
    assert np.array_equal(_np(lv), ref)
    assert counts[:5] == [int((ref >= l).sum()) for l in range(5)]


def test_hnsw_layers_bit_exact(sift_like):
    """Integer data: every upper layer (members, neighbour positions, degrees) equals the oracle's."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    X = torch.from_numpy(w.X).to(_dev())
    built = fg.build_layers(X, M=8, ef=32, seed=7)
    levels = O.hnsw_levels(w.N, 8, seed=7)
    assert np.array_equal(_np(built["levels"]), levels)
    assert len(built["layers"]) >= 3
    for l, ly in enumerate(built["layers"], start=1):
        members, adj, deg = O.hnsw_layer(w.X, w.metric, levels, l, 8, 32)
        assert np.array_equal(_np(ly["members"]), members), l
        assert np.array_equal(_np(ly["deg"]), deg), l
        assert np.array_equal(_np(ly["adj"]), adj), l
    assert built["entry"] == O.hnsw_entry(levels)


def test_search_hnsw_matches_oracle(sift_like):
    """The layered search: the same descent end points and results as the oracle's."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    dev = _dev()
    out = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=1)
    gi = _np(out["ids"])
    X = torch.from_numpy(w.X).to(dev)
    built = fg.build_layers(X, M=8, ef=32, seed=7)
    Q = w.Q[:200]
    layers = [(_np(ly["members"]), _np(ly["adj"])) for ly in built["layers"]]
    for ef_up in (1, 8):
        ids, dist, start = fg.search_hnsw(X, out["ids"], built["layers"], built["entry"], torch.from_numpy(Q).to(dev),
                                          topk=10, beam=32, ef_up=ef_up)
        oi, od, ost = O.hnsw_search(w.X, w.metric, gi, layers, built["entry"], Q, 32, 10, ef_up=ef_up)
        assert np.array_equal(_np(start), ost), ef_up
        assert np.array_equal(_np(ids), oi), ef_up
    # the descent's start is never farther from the query than the entry
    gt, _ = O.knn_exact(w.X, Q, 10, w.metric)
    assert O.recall_at(_np(ids), gt, 10) >= O.recall_at(
        _np(fg.search(X, out["ids"], out["entry"], torch.from_numpy(Q).to(dev), topk=10, beam=32)[0]), gt, 10) - 0.02


def test_hnsw_layer_cosine_bf16(bf16_batch):
    """768-d cosine, BF16 storage: layer 1 keeps the oracle's members and nearly all its rows."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P = bf16_batch[0]
    Xb = torch.from_numpy(w.bits().view(np.int16)).to(_dev()).view(torch.bfloat16)
    lv, counts = fg.hnsw_levels(w.N, 4, seed=3)
    ly = fg.hnsw_layer(Xb, lv, 1, counts[1], M=4, ef=16, metric="cos")
    members, adj, deg = O.hnsw_layer(w.X, w.metric, O.hnsw_levels(w.N, 4, seed=3), 1, 4, 16)
    assert np.array_equal(_np(ly["members"]), members)
    same = np.all(_np(ly["adj"]) == adj, 1).mean()
    assert same >= 0.98, same


def test_merge_host_bf16_matches_device(bf16_batch):
    """BF16 vectors through the host-buffer entry point: the same graph as the device call."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P = bf16_batch[2]
    Xh = torch.from_numpy(w.bits().view(np.int16)).view(torch.bfloat16).pin_memory()
    adj = torch.from_numpy(np.concatenate([g[0] for g in graphs])).pin_memory()
    h = fg.merge_host(Xh, adj, w.shard_sizes, [g[1] for g in graphs], k=w.k, R=w.R, alpha=w.alpha, iters=1,
                      metric="cos")
    d = fg.merge(_inp_bf16(w, graphs), k=w.k, R=w.R, alpha=w.alpha, iters=1)
    assert np.array_equal(h["ids"].numpy(), _np(d["ids"])) and h["entry"] == d["entry"]


def test_build_pg_bit_exact_and_merges(sift_like):
    """Input PGs built on the GPU by batch-incremental insertion equal the host builder's
    (synth/pgbuild.c, the same recipe) bit for bit on integer data, entry (the medoid) included,
    and a merge of them equals the oracle's merge of the same PGs."""
    import paper_2603_21710_gb300 as fg
    from synth import pgbuild
    w, _, _, _ = sift_like
    dev = _dev()
    graphs = []
    for i in range(w.h):
        Xs = np.ascontiguousarray(w.shard(i))
        adj, entry = fg.build_pg(torch.from_numpy(Xs).to(dev), M=16, ef=32)
        ref, ref_entry = pgbuild.build_pg(Xs, 16, 32, w.metric)
        assert entry == ref_entry, i
        assert np.array_equal(_np(adj), ref), (i, int(np.sum(np.any(_np(adj) != ref, 1))))
        graphs.append((ref, entry))
    P = O.Problem.from_workload(w, graphs)
    inp = _inp(w, graphs)
    out = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=1)
    ref = O.merge(P, w.k, w.R, w.alpha, iters=1)
    assert np.array_equal(_np(out["ids"]), ref.ids) and out["entry"] == ref.entry


# --------------------------------------------------------------------------- the precision recipe
@pytest.fixture(scope="module")
def deep_like():
    """The precision recipe (unit-norm d = 96, inner product, 2 shards, k = 48) at N = 40,000
    with the cluster count scaled like the points (80 centers)."""
    from synth import gen, pgbuild
    w = gen.make("precision", N=40_000, nq=1000, n_centers=80)
    graphs = pgbuild.build_all(w)
    P = O.Problem.from_workload(w, graphs)
    return w, graphs, P, _inp(w, graphs)


def test_precision_recipe_refine_pass_and_merge(deep_like):
    """IP on unit vectors with the BF16 tensor-core filter: a refinement pass keeps the oracle's
    lists; the whole merge's k-NNG recall and search recall@10 (1,000 queries, beam 64) are
    within 0.5 point of the oracle-merged graph's."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = deep_like
    assert w.metric == 1 and w.d == 96 and w.k == 48
    o, _, _ = O.stage_a(P, w.k)
    g = _to_dev(o)
    st = fg.refine_pass(inp, g, join_filter="tc")
    O.refine_iter(P, o)
    bad = PR.lists_match(_np(g["ids"]), _np(g["dist"]), o.ids, o.dist)
    assert len(bad) == 0, bad[:10]
    assert sum(st["join_class"][:3]) > 0 and st["join_class"][3] == 0, st["join_class"]
    out = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=3, return_knng=True)
    ref = O.merge(P, w.k, w.R, w.alpha, iters=3)
    gi = _np(out["ids"])
    PR.check_lists(gi, _np(out["dist"]), w.N)
    assert PR.bfs_reached(gi, out["entry"]).all() and out["entry"] == ref.entry
    samp = np.random.default_rng(8).choice(w.N, 2000, replace=False)
    tid, _ = O.knn_exact(w.X, w.X[samp], w.k, w.metric, exclude=samp)
    kg = _np(out["knng"]["ids"])
    assert abs(O.recall_at(kg[samp], tid, w.k) - O.recall_at(ref.knn_ids[samp], tid, w.k)) <= 0.005
    gt, _ = O.knn_exact(w.X, w.Q, 10, w.metric)
    sg, _ = fg.search(inp.X, out["ids"], out["entry"], torch.from_numpy(w.Q).to(_dev()), topk=10, beam=64,
                      metric="ip")
    so, _, _ = O.search(w.X, ref.ids, ref.entry, w.Q, 64, 10, w.metric)
    assert abs(O.recall_at(_np(sg), gt, 10) - O.recall_at(so, gt, 10)) <= 0.005


# --------------------------------------------------------------------------- join forms reached
def test_parity_inputs_reach_every_join_form(sift_like, small):
    """Update's forms on the parity inputs: the Sift-like merge passes reach the two smaller
    tensor-core size classes and the warp-per-vertex form (few new candidates); a k-NNG with mixed flags reaches the third (|C| > 128); k = 96
    (candidate sets above the tile's limits) takes the FP32 tile; every one keeps the oracle's
    lists."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    o, _, _ = O.stage_a(P, w.k)
    g = _to_dev(o)
    seen = [0, 0, 0, 0, 0]
    for _ in range(3):
        st = fg.refine_pass(inp, g)
        seen = [a + b for a, b in zip(seen, st["join_class"])]
        fg.indegree_repair(inp, g)
    assert seen[0] > 0 and seen[1] > 0 and seen[4] > 0, seen
    # a k-NNG with half of its entries old (the state of a later pass on larger data) gives sets
    # of new and old candidates above 128: the third class, bit for bit against the oracle
    o, _, _ = O.stage_a(P, w.k)
    o.flags[np.random.default_rng(4).random(o.flags.shape) < 0.5] = 0
    g = _to_dev(o)
    st = fg.refine_pass(inp, g)
    O.refine_iter(P, o)
    assert st["join_class"][2] > 0, st["join_class"]
    assert np.array_equal(_np(g["ids"]), o.ids) and np.array_equal(_np(g["flags"]), o.flags)
    ws, gs, Ps, inps = small
    os_, _, _ = O.stage_a(Ps, 96)
    g = _to_dev(os_)
    st = fg.refine_pass(inps, g, join_filter="tc")
    O.refine_iter(Ps, os_)
    assert st["join_class"][3] > 0, st["join_class"]
    bad = PR.lists_match(_np(g["ids"]), _np(g["dist"]), os_.ids, os_.dist)
    assert len(bad) == 0, bad[:10]


# --------------------------------------------------------------------------- rarely taken paths (test hooks)
@pytest.fixture
def hooks():
    import paper_2603_21710_gb300 as fg
    fg.load()
    yield fg._lib
    for knob, off in (("prop_cap", 0), ("hop_budget", 0), ("fail_alloc_after", -1), ("batch_union", 1),
                      ("join_sparse_nn", -1)):
        fg._lib.test_set(knob, off)


@pytest.mark.parametrize("join_filter", ["tc", "fp32"])
def test_proposal_overflow_rerun_bit_exact(sift_like, hooks, join_filter):
    """A proposal buffer far too small for one pass: the vertices whose proposals did not fit
    are re-run against the merged lists, and the pass still equals the oracle's bit for bit."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    o, _, _ = O.stage_a(P, w.k)
    g = _to_dev(o)
    hooks.test_set("prop_cap", 1)   # raised to what one vertex can propose
    st = fg.refine_pass(inp, g, join_filter=join_filter)
    hooks.test_set("prop_cap", 0)
    O.refine_iter(P, o)
    assert st["join_reruns"] > 0
    assert np.array_equal(_np(g["ids"]), o.ids)
    assert np.array_equal(_np(g["dist"]), o.dist)
    assert np.array_equal(_np(g["flags"]), o.flags)


def test_hop_budget_runs_out_cleanly(small, hooks):
    """A beam search whose expansion budget runs out stops, the call returns FGIM_ETIMEOUT, and
    the next call on the same context works."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    out = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=1)
    Q = torch.from_numpy(w.Q[:64]).to(_dev())
    hooks.test_set("hop_budget", 2)
    with pytest.raises(fg.FgimError) as e:
        fg.cross_query(inp, w.k)
    assert e.value.status == -4
    with pytest.raises(fg.FgimError) as e:
        fg.search(inp.X, out["ids"], out["entry"], Q, topk=10, beam=64)
    assert e.value.status == -4
    hooks.test_set("hop_budget", 0)
    g = fg.cross_query(inp, w.k)
    o, _, _ = O.stage_a(P, w.k)
    assert np.all(_np(g["ids"]) == o.ids, 1).mean() >= 0.99


def test_alloc_failure_is_enomem_and_leaks_nothing(small, hooks):
    """A scratch allocation that fails at any point of a merge returns FGIM_ENOMEM, every byte the
    call had taken goes back to the pool, and the next merge equals an undisturbed one."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    ref = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=1)
    n = hooks.test_get("scratch_allocs")
    assert n > 10
    torch.cuda.synchronize()
    assert hooks.test_get("pool_used_bytes") == 0
    for after in sorted({0, 1, n // 4, n // 2, n - 1}):
        hooks.test_set("fail_alloc_after", after)
        with pytest.raises(fg.FgimError) as e:
            fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=1)
        hooks.test_set("fail_alloc_after", -1)
        torch.cuda.synchronize()
        assert e.value.status == -2, after
        assert hooks.test_get("pool_used_bytes") == 0, after
    again = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=1)
    assert torch.equal(again["ids"], ref["ids"]) and again["entry"] == ref["entry"]


# --------------------------------------------------------------------------- input-PG builder, float data
@pytest.mark.parametrize("metric", ["l2", "cos"])
def test_build_pg_float_data(metric):
    """Float data (the small recipe; the same rows under cosine): the GPU builder's graph and the
    host builder's have the same entry and the same search quality (recall@10 of Alg. 1 at beam 32
    within one point; insertion is incremental, so a near tie early on changes later lists)."""
    import paper_2603_21710_gb300 as fg
    from synth import gen, pgbuild
    w = gen.make("small", N=6000, nq=500)
    Xs = np.ascontiguousarray(w.X)
    m = {"l2": 0, "cos": 2}[metric]
    adj, entry = fg.build_pg(torch.from_numpy(Xs).to(_dev()), M=12, ef=32, metric=metric)
    ref, ref_entry = pgbuild.build_pg(Xs, 12, 32, m)
    assert entry == ref_entry
    ga = _np(adj)
    assert np.all((ga >= -1) & (ga < Xs.shape[0])) and np.all(ga != np.arange(Xs.shape[0])[:, None])
    gt, _ = O.knn_exact(Xs, w.Q, 10, m)
    rg = O.recall_at(O.search(Xs, ga, entry, w.Q, 32, 10, m)[0], gt, 10)
    rr = O.recall_at(O.search(Xs, ref, ref_entry, w.Q, 32, 10, m)[0], gt, 10)
    assert abs(rg - rr) <= 0.01, (rg, rr)


# --------------------------------------------------------------------------- alternative neighbour selection
RULES = [("mrng", 0.0), ("tmng", 10.0), ("tmng", 60.0)]


@pytest.mark.parametrize("rule,tau", RULES)
def test_prune_rules_integer_bit_exact(sift_like, rule, tau):
    """MRNG and tau-MNG (Sec. 4.3.1) on integer data: the byte-row and FP32-row prunes equal the
    oracle's lists bit for bit, and so does the whole merge pruned with the rule."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    o, T = _refined(P, w, iters=1)
    oi, od, oc, _ = O.prune(P, o, T, w.R, 1.0, rule, tau)
    for rows in ("auto", "fp32"):
        ei, ed, ec = fg.prune(inp, _to_dev(o), torch.from_numpy(T).to(_dev()), w.R, 1.0, rows=rows, rule=rule, tau=tau)
        assert np.array_equal(_np(ei), oi) and np.array_equal(_np(ed), od) and np.array_equal(_np(ec), oc), rows
    out = fg.merge(inp, k=w.k, R=w.R, alpha=1.0, iters=1, rule=rule, tau=tau)
    ref = O.merge(P, w.k, w.R, 1.0, iters=1, rule=rule, tau=tau)
    assert np.array_equal(_np(out["ids"]), ref.ids) and out["entry"] == ref.entry
    assert PR.bfs_reached(_np(out["ids"]), out["entry"]).all()


@pytest.mark.parametrize("which", ["small", "high_dim"])
@pytest.mark.parametrize("rule,tau", [("mrng", 0.0), ("tmng", 0.5)])
def test_prune_rules_float_data(which, rule, tau, request):
    """Float data (the FP32 filter with re-check at d = 32, the warp-wide form at d = 960): the
    oracle's lists except where an occlusion test of the rule ties within tolerance."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = request.getfixturevalue(which)
    if which == "high_dim":
        tau = tau / 4
    o, T = _refined(P, w, iters=1)
    ei, ed, ec = fg.prune(inp, _to_dev(o), torch.from_numpy(T).to(_dev()), w.R, 1.0, rule=rule, tau=tau)
    oi, od, oc, _ = O.prune(P, o, T, w.R, 1.0, rule, tau)
    ei, ed, ec = _np(ei), _np(ed), _np(ec)
    diff = np.nonzero(~np.all(ei == oi, 1))[0]
    assert len(diff) <= max(2, w.N // 2000), len(diff)
    for u in diff:
        cand = o.ids[u][o.ids[u] >= 0]
        assert PR.prune_row_has_near_tie(w.X, u, cand, o.dist[u][:len(cand)], 1.0, metric=w.metric, rule=rule,
                                         tau=tau), u
    same = np.all(ei == oi, 1)
    assert np.array_equal(ed[same], od[same]) and np.array_equal(ec[same], oc[same])


def test_library_owned_graph(small):
    """fgim_graph_alloc / fgim_graph_free: a merge into library-owned buffers equals the merge into
    caller-owned ones; the graph is zeroed after the free."""
    import ctypes
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = small
    L = fg.load()
    ref = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=1)
    g = fg.Graph()
    assert L.fgim_graph_alloc(w.N, w.R, ctypes.byref(g)) == 0
    assert g.n == w.N and g.R == w.R and g.ids
    p = inp.params(w.k, w.R, w.alpha, 0, 1)
    fg.check(L.fgim_merge(inp._shards, inp.h, ctypes.byref(p), None, ctypes.byref(g),
                          torch.cuda.current_stream().cuda_stream))
    class _View:   # the library's block seen as a tensor (no copy)
        def __init__(self, ptr, shape):
            self.__cuda_array_interface__ = {"data": (ptr, False), "shape": shape, "typestr": "<i4", "version": 2}
    ids = torch.as_tensor(_View(g.ids, (w.N, w.R)), device=_dev())
    assert torch.equal(ids, ref["ids"]) and g.entry == ref["entry"]
    del ids
    L.fgim_graph_free(ctypes.byref(g))
    assert not g.ids and g.n == 0


# --------------------------------------------------------------------------- the batch as one problem
@pytest.fixture(scope="module")
def int_batch():
    """Four Sift-like merges of uneven size and shard count (h = 2, 3, 5, 4): integer data, so the
    batch must equal the oracle's merges bit for bit."""
    from synth import gen, pgbuild
    out = []
    for i, (n, h) in enumerate(((3000, 2), (9000, 3), (5000, 5), (12000, 4))):
        w = gen.make("medium", N=n, h=h, nq=10, n_centers=12, seed=gen.MASTER_SEED + 100 + i)
        graphs = pgbuild.build_all(w)
        out.append((w, graphs, O.Problem.from_workload(w, graphs)))
    return out


def test_batch_as_one_problem_equals_oracle_merges(int_batch, hooks):
    """fgim_merge_batch runs the merges as one problem over their disjoint union; each output
    equals the oracle's merge of that input alone (its own L = ceil(k / (h - 1)), its own entry),
    and the one-after-another form gives the same graphs."""
    import paper_2603_21710_gb300 as fg
    inps = [_inp(w, graphs) for w, graphs, _ in int_batch]
    w0 = int_batch[0][0]
    outs = fg.merge_batch(inps, k=w0.k, R=w0.R, alpha=w0.alpha, iters=2)
    for (w, graphs, P), o in zip(int_batch, outs):
        ref = O.merge(P, w0.k, w0.R, w0.alpha, iters=2)
        assert np.array_equal(_np(o["ids"]), ref.ids) and np.array_equal(_np(o["deg"]), ref.deg)
        assert o["entry"] == ref.entry
        assert PR.bfs_reached(_np(o["ids"]), o["entry"]).all()
    hooks.test_set("batch_union", 0)
    seq = fg.merge_batch(inps, k=w0.k, R=w0.R, alpha=w0.alpha, iters=2)
    hooks.test_set("batch_union", 1)
    for a, b in zip(outs, seq):
        assert torch.equal(a["ids"], b["ids"]) and torch.equal(a["dist"], b["dist"]) and a["entry"] == b["entry"]


# --------------------------------------------------------------------------- FP8 E4M3 candidate distances
@pytest.mark.parametrize("which", ["high_dim", "deep_like", "small"])
def test_fp8_join_filter_keeps_the_fp32_lists(which, request):
    """Update with E4M3 rows and per-vector scales on the tensor cores (filter only; survivors
    re-ranked in exact FP32): the refined lists, distances and flags equal the FP32 SIMT form's
    and the BF16 form's, and it evaluates the same pairs."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = request.getfixturevalue(which)
    assert w.d % 32 == 0
    o, _, _ = O.stage_a(P, w.k)
    outs = {}
    for jf in ("fp8", "tc", "fp32"):
        g = _to_dev(o)
        st = fg.refine_pass(inp, g, join_filter=jf)
        outs[jf] = (g, st)
    a, sa = outs["fp8"]
    for jf in ("tc", "fp32"):
        b, sb = outs[jf]
        assert torch.equal(a["ids"], b["ids"]) and torch.equal(a["dist"], b["dist"]), jf
        assert torch.equal(a["flags"], b["flags"]), jf
        assert sa["join_pairs"] == sb["join_pairs"], jf
    assert sum(sa["join_class"][:3]) > 0 and sa["join_class"][3] == 0, sa["join_class"]


def test_fp8_merge_equals_fp32_merge(high_dim):
    """The whole d = 960 merge with the FP8 filter builds the FP32 form's graph."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = high_dim
    a = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2, join_filter="fp8")
    b = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=2, join_filter="fp32", rows="fp32")
    assert torch.equal(a["ids"], b["ids"]) and torch.equal(a["dist"], b["dist"]) and a["entry"] == b["entry"]


# --------------------------------------------------------------------------- autotuned launch shapes
def test_autotune_changes_no_result(sift_like, tmp_path):
    """The autotuner picks a beam-search launch shape for the workload and writes it to its cache;
    merges with the tuned shape, and with the smallest visited table and two warps per block
    forced through a cache file, build the default shape's graph bit for bit."""
    import json
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    fg.autotune_clear()
    ref = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=1)
    cache = tmp_path / "tune.jsonl"
    r = fg.autotune(inp, w.k, cache_path=str(cache))
    assert r["wpb"] in (2, 4) and 6 <= r["ht_bits"] <= 13 and r["ms"] > 0
    a = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=1)
    assert torch.equal(a["ids"], ref["ids"]) and torch.equal(a["dist"], ref["dist"])
    rec = json.loads(cache.read_text().strip().splitlines()[-1])
    assert rec["wpb"] == r["wpb"] and rec["ht_bits"] == r["ht_bits"] and rec["L"] == 22 and rec["row_bytes"] == 1
    forced = tmp_path / "forced.jsonl"
    forced.write_text(json.dumps({"key": rec["key"], "wpb": 2, "ht_bits": 6}) + "\n")
    fg.autotune_clear()
    fg.autotune_load(str(forced))
    b = fg.merge(inp, k=w.k, R=w.R, alpha=w.alpha, iters=1)
    fg.autotune_clear()
    assert torch.equal(b["ids"], ref["ids"]) and torch.equal(b["dist"], ref["dist"])
    assert b["stats"]["ndc"] >= ref["stats"]["ndc"]   # a smaller table may only re-evaluate


# --------------------------------------------------------------------------- warp-per-vertex Update
def test_sparse_join_form_overflow_rerun(sift_like, hooks):
    """The warp-per-vertex form with a proposal buffer far too small: its vertices whose
    proposals did not fit are re-run by the tile form against the merged lists, and the pass
    still equals the oracle's bit for bit."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    o, _, _ = O.stage_a(P, w.k)
    g = _to_dev(o)
    hooks.test_set("join_sparse_nn", 1 << 20)   # every vertex with |C| <= 128
    hooks.test_set("prop_cap", 1)
    st = fg.refine_pass(inp, g)
    O.refine_iter(P, o)
    assert st["join_reruns"] > 0 and st["join_class"][4] > 0, st
    for key, ref in (("ids", o.ids), ("dist", o.dist), ("flags", o.flags)):
        assert np.array_equal(_np(g[key]), ref), key


@pytest.mark.parametrize("cut", [0, 1 << 20])
def test_sparse_join_form_bit_exact(sift_like, hooks, cut):
    """Update with every eligible vertex (|C| <= 128) joined one warp per vertex, and with none:
    three passes from the oracle's state (the later ones have few new candidates per vertex)
    each equal the oracle's pass bit for bit, pair count included."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    o, _, _ = O.stage_a(P, w.k)
    hooks.test_set("join_sparse_nn", cut)
    sparse = 0
    for _ in range(3):
        g = _to_dev(o)
        st = fg.refine_pass(inp, g)
        ost = O.refine_iter(P, o)
        sparse += st["join_class"][4]
        assert np.array_equal(_np(g["ids"]), o.ids)
        assert np.array_equal(_np(g["dist"]), o.dist)
        assert np.array_equal(_np(g["flags"]), o.flags)
        assert st["join_pairs"] == ost["pairs"]
    assert (sparse > 0) == (cut > 0), sparse


def _int_tiny(seed, sizes, d, M, metric):
    from synth import pgbuild
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0, 255, (20, d))
    X = np.rint(np.clip(centers[rng.integers(0, 20, sum(sizes))] + rng.normal(0, 25, (sum(sizes), d)), 0, 255))
    X = X.astype(np.float32)
    gs, o = [], 0
    for n in sizes:
        gs.append(pgbuild.build_pg(X[o:o + n], M, 32, metric))
        o += n
    return X, gs


@pytest.mark.parametrize("metric", [0, 1, 2])
def test_sparse_join_form_metrics(hooks, metric):
    """Integer rows under each metric (squared L2, inner product, cosine): the warp-per-vertex
    form and the tensor-core tile give the same lists, flags and pair counts, and both keep
    the oracle's lists."""
    import paper_2603_21710_gb300 as fg
    sizes, d, M, k = [700, 500, 300], 48, 16, 16
    X, gs = _int_tiny(40 + metric, sizes, d, M, metric)
    P = O.Problem(X, sizes, np.concatenate([g[0] for g in gs]), np.array([g[1] for g in gs], np.int32), metric)
    dev = _dev()
    inp = fg.MergeInput.from_flat(torch.from_numpy(X).to(dev), sizes,
                                  torch.from_numpy(np.concatenate([g[0] for g in gs])).to(dev),
                                  [g[1] for g in gs], metric=metric)
    o, _, _ = O.stage_a(P, k)
    for _ in range(2):
        outs = []
        for cut in (0, 1 << 20):
            hooks.test_set("join_sparse_nn", cut)
            g = _to_dev(o)
            st = fg.refine_pass(inp, g)
            outs.append((g, st))
        (a, sa), (b, sb) = outs
        assert sa["join_class"][4] == 0 and sb["join_class"][4] > 0, (sa["join_class"], sb["join_class"])
        for key in ("ids", "dist", "flags"):
            assert torch.equal(a[key], b[key]), key
        assert sa["join_pairs"] == sb["join_pairs"]
        O.refine_iter(P, o)
        assert len(PR.lists_match(_np(b["ids"]), _np(b["dist"]), o.ids, o.dist)) == 0


def test_cross_query_adjacency_with_repeated_ids(sift_like):
    """Input graphs whose rows list a neighbour twice (within one 32-entry chunk): the searches
    evaluate each neighbour once, as Alg. 1's visited set does, so stage a still equals the
    oracle's bit for bit; the same graphs without repeats give the same result."""
    import paper_2603_21710_gb300 as fg
    w, graphs, P, inp = sift_like
    rng = np.random.default_rng(21)
    gs = []
    for adj, ent in graphs:
        a = adj.copy()
        rows = rng.choice(a.shape[0], a.shape[0] // 3, replace=False)
        for r in rows:   # replace the last valid entry by a copy of the first (same chunk)
            nv = int((a[r] >= 0).sum())
            if nv >= 2 and nv <= 32:
                a[r, nv - 1] = a[r, 0]
        gs.append((a, ent))
    Pd = O.Problem.from_workload(w, gs)
    dev = _dev()
    inpd = fg.MergeInput.from_flat(inp.X, w.shard_sizes, torch.from_numpy(np.concatenate([g[0] for g in gs])).to(dev),
                                   [g[1] for g in gs])
    ga = fg.cross_query(inpd, w.k)
    oa, _, _ = O.stage_a(Pd, w.k)
    assert np.array_equal(_np(ga["ids"]), oa.ids)
    assert np.array_equal(_np(ga["dist"]), oa.dist)
