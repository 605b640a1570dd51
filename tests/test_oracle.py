"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Each test ties one oracle function to something other than itself: a hand-derived
trace (tests/golden), a closed form, a special case that reduces to exact k-NN, or
an invariant the algorithm guarantees.
"""
import json
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _line_problem(pos, sizes=None, adj=None, M=1):
    """1-D points (d=1) as a problem; adjacency defaults to empty lists."""
    X = np.asarray(pos, np.float32).reshape(-1, 1)
    N = X.shape[0]
    sizes = sizes or [N]
    if adj is None:
        adj = np.full((N, M), -1, np.int32)
    return O.Problem(X, sizes, adj, np.zeros(len(sizes), np.int32), O_METRIC_L2)


O_METRIC_L2, O_METRIC_IP, O_METRIC_COS = 0, 1, 2


def _knng_from_lists(P, lists, flags=0):
    N = len(lists)
    k = len(lists[0])
    g = O.KNNG(N, k)
    for u, row in enumerate(lists):
        for t, v in enumerate(row):
            g.ids[u, t] = v
            g.dist[u, t] = O.delta(P.X[u], P.X[v], P.metric)
    g.flags[:] = flags
    return g


def _check_lists(ids, dist, N):
    for u in range(ids.shape[0]):
        row = ids[u]
        valid = row[row >= 0]
        n = len(valid)
        assert np.all(row[n:] == -1), "empty slots must be last"
        assert len(set(valid.tolist())) == n, "duplicate id"
        assert u not in set(valid.tolist()), "self loop"
        d = dist[u, :n]
        keys = list(zip(d.tolist(), valid.tolist()))
        assert keys == sorted(keys), "row not sorted by (dist, id)"
        assert np.all(valid < N)


# --------------------------------------------------------------------------- delta
def test_delta_closed_forms():
    x = np.array([1, 2, 3, 0], np.float32)
    y = np.array([4, 6, 3, 0], np.float32)
    assert O.delta(x, y, O_METRIC_L2) == 25.0
    assert O.delta(y, x, O_METRIC_L2) == 25.0
    e1 = np.array([1, 0, 0, 0], np.float32)
    s = np.array([1, 1, 0, 0], np.float32) / np.float32(np.sqrt(2))
    assert abs(O.delta(e1, s, O_METRIC_IP) - (1 - 1 / np.sqrt(2))) < 1e-7
    # cosine ignores the norms
    assert abs(O.delta(e1 * 3, np.array([2, 2, 0, 0], np.float32), O_METRIC_COS) - (1 - 1 / np.sqrt(2))) < 1e-7
    # 1 - x.y on unit vectors equals half the squared L2 distance
    a = np.random.default_rng(1).standard_normal(16).astype(np.float32)
    b = np.random.default_rng(2).standard_normal(16).astype(np.float32)
    a /= np.linalg.norm(a)
    b /= np.linalg.norm(b)
    assert abs(O.delta(a, b, O_METRIC_IP) - 0.5 * O.delta(a, b, O_METRIC_L2)) < 1e-6


# --------------------------------------------------------------------------- Alg. 1
def test_beam_chain_golden():
    g = _golden("beam_chain.json")
    n = g["n"]
    X = np.arange(n, dtype=np.float32).reshape(-1, 1)
    adj = np.full((n, 2), -1, np.int32)
    for i in range(n):
        if i > 0:
            adj[i, 0] = i - 1
        if i + 1 < n:
            adj[i, 1] = i + 1
    q = np.array([g["query"]], np.float32)
    ids, dist, st = O.knn_search(X, adj, g["entry"], q, g["L"], g["k"], O_METRIC_L2)
    assert ids.tolist() == g["expected_ids"]
    np.testing.assert_allclose(dist, g["expected_dist"], rtol=1e-5)
    assert st["hops"] == g["expected_hops"]
    assert st["ndc"] == g["expected_ndc"]


def test_beam_exhaustive_equals_bruteforce():
    """If the graph is connected from ep and L >= n, Alg. 1 evaluates every vertex: exact top-k."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((300, 8)).astype(np.float32)
    # a ring (connected) plus random chords
    adj = np.concatenate([((np.arange(300) + 1) % 300)[:, None], ((np.arange(300) - 1) % 300)[:, None],
                          rng.integers(0, 300, (300, 6))], axis=1).astype(np.int32)
    ep = 17
    Q = rng.standard_normal((20, 8)).astype(np.float32)
    gt, gd = O.knn_exact(X, Q, 10, O_METRIC_L2)
    for qi in range(20):
        ids, dist, st = O.knn_search(X, adj, ep, Q[qi], 300, 10, O_METRIC_L2)
        assert ids.tolist() == gt[qi].tolist()
        assert st["ndc"] == 300


def test_beam_invariants(small_problem):
    w, graphs, P = small_problem
    X0 = w.shard(0)
    adj, ep = graphs[0]
    for qi in range(50):
        ids, dist, st = O.knn_search(X0, adj, ep, w.Q[qi], 16, 16, w.metric)
        assert len(ids) == 16 and len(set(ids.tolist())) == 16
        keys = list(zip(dist.tolist(), ids.tolist()))
        assert keys == sorted(keys)
        assert st["hops"] >= 1 and st["ndc"] >= 16


# --------------------------------------------------------------------------- Alg. 2
def _complete_problem(X, sizes, metric=O_METRIC_L2):
    N = X.shape[0]
    M = max(sizes) - 1
    adj = np.full((N, M), -1, np.int32)
    off = np.cumsum([0] + sizes)
    for i, s in enumerate(sizes):
        for u in range(s):
            others = [v for v in range(s) if v != u]
            adj[off[i] + u, :len(others)] = others
    return O.Problem(X, sizes, adj, np.zeros(len(sizes), np.int32), metric)


@pytest.mark.parametrize("sizes,k,L", [([60, 60], 8, 0), ([40, 50, 30], 6, 6)])
def test_stage_a_complete_graphs_is_exact(sizes, k, L):
    """Complete input graphs make C+ exact and one expansion of ep exact, so Alg. 2 yields the exact k-NNG."""
    rng = np.random.default_rng(7)
    X = rng.standard_normal((sum(sizes), 6)).astype(np.float32)
    P = _complete_problem(X, sizes)
    g, Lu, st = O.stage_a(P, k, L)
    gt, gd = O.knn_exact(X, X, k, O_METRIC_L2, exclude=np.arange(X.shape[0]))
    assert np.array_equal(g.ids, gt)
    np.testing.assert_allclose(g.dist, gd, rtol=1e-6)
    assert np.all(g.flags == O.FLAG_NEW)


@pytest.mark.parametrize("k,h,L", [(16, 2, 16), (64, 4, 22), (48, 2, 48), (64, 8, 10), (32, 6, 7), (32, 3, 16)])
def test_minimum_querying_L(k, h, L):
    """Sec. 4.1.2 worst case: L = ceil(k / (h - 1))."""
    rng = np.random.default_rng(0)
    sizes = [12] * h
    X = rng.standard_normal((12 * h, 4)).astype(np.float32)
    P = _complete_problem(X, sizes)
    _, Lu, _ = O.stage_a(P, k, 0)
    assert Lu == L


def test_stage_a_rows_valid(small_problem):
    w, graphs, P = small_problem
    g, Lu, st = O.stage_a(P, w.k)
    assert Lu == 16
    _check_lists(g.ids, g.dist, w.N)
    assert np.all(g.ids >= 0), "every vertex gets k candidates (L >= k / (h-1))"


# --------------------------------------------------------------------------- Alg. 3
def _two_shard_uniform(N=600, d=4, seed=11):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (N, d)).astype(np.float32)
    return X, [N // 2, N - N // 2]


def test_refine_exact_knng_is_fixed_point():
    X, sizes = _two_shard_uniform()
    P = _complete_problem(X, sizes)
    k = 8
    gt, gd = O.knn_exact(X, X, k, O_METRIC_L2, exclude=np.arange(X.shape[0]))
    g = O.KNNG(X.shape[0], k)
    g.ids[:], g.dist[:], g.flags[:] = gt, gd, O.FLAG_NEW
    st = O.refine_iter(P, g)
    assert st["updates"] == 0
    assert st["pairs"] > 0
    assert np.array_equal(g.ids, gt) and np.array_equal(g.dist, gd)
    assert np.all(g.flags == 0), "visited entries are old after the pass"


def test_refine_monotone_cross_only(small_problem):
    w, graphs, P = small_problem
    g, _, _ = O.stage_a(P, w.k)
    shard = np.repeat(np.arange(w.h), w.shard_sizes)
    for _ in range(2):
        before = g.copy()
        st = O.refine_iter(P, g)
        assert st["updates"] > 0
        _check_lists(g.ids, g.dist, w.N)
        # the j-th distance of a list never increases
        assert np.all(g.dist <= before.dist)
        # every entry inserted by Update is a cross-graph pair (Alg. 3: v1, v2 from different G_i)
        new = (g.flags & O.FLAG_NEW) > 0
        rows = np.nonzero(new)[0]
        assert np.all(shard[g.ids[new]] != shard[rows])
        # entries that were already present keep their distance
        for u in range(0, w.N, 997):
            old = dict(zip(before.ids[u].tolist(), before.dist[u].tolist()))
            for v, dv in zip(g.ids[u].tolist(), g.dist[u].tolist()):
                if v in old:
                    assert old[v] == dv


def test_refine_converges_to_exact_with_complete_local_graphs():
    """Complete local graphs make the intra-shard part exact; refinement must complete the cross part."""
    X, sizes = _two_shard_uniform(N=800, d=3, seed=3)
    P = _complete_problem(X, sizes)
    k = 8
    g, _, _ = O.stage_a(P, k, 2)          # deliberately few cross candidates
    gt, _ = O.knn_exact(X, X, k, O_METRIC_L2, exclude=np.arange(X.shape[0]))
    r0 = O.recall_at(g.ids, gt, k)
    for _ in range(6):
        O.refine_iter(P, g)
    r1 = O.recall_at(g.ids, gt, k)
    assert r0 < 0.95 and r1 >= 0.99, (r0, r1)


def test_refine_rev_cap_limits_pairs(small_problem):
    w, graphs, P = small_problem
    g, _, _ = O.stage_a(P, w.k)
    g2 = g.copy()
    s_full = O.refine_iter(P, g, rev_cap=w.k)
    s_cap = O.refine_iter(P, g2, rev_cap=2)
    assert s_cap["pairs"] < s_full["pairs"]


# --------------------------------------------------------------------------- Alg. 4
def test_repair_golden():
    gd = _golden("repair_10v.json")
    P = _line_problem(gd["pos"])
    g = _knng_from_lists(P, gd["lists"], flags=0)
    T, st = O.indegree_repair(P, g)
    assert g.ids.tolist() == gd["expected_lists"]
    np.testing.assert_array_equal(g.dist, np.asarray(gd["expected_dist"], np.float32))
    assert g.flags.tolist() == gd["expected_flags"]
    assert T.tolist() == gd["expected_T"]
    assert st["zero_before"] == 4 and st["zero_after"] == 0 and st["replaced"] == 4


def test_repair_invariants(small_problem):
    w, graphs, P = small_problem
    g, _, _ = O.stage_a(P, w.k)
    O.refine_iter(P, g)
    T0 = O.indegree(g.ids)
    outdeg0 = (g.ids >= 0).sum(1)
    T, st = O.indegree_repair(P, g)
    assert np.array_equal(T, O.indegree(g.ids)), "returned recorder equals the recomputed indegree"
    assert T.sum() == (g.ids >= 0).sum()
    assert np.array_equal((g.ids >= 0).sum(1), outdeg0), "outdegree unchanged"
    assert st["zero_before"] == (T0 == 0).sum()
    assert st["zero_after"] <= st["zero_before"]
    assert np.all(T[T0 > 0] > 0), "no vertex driven to zero indegree"
    _check_lists(g.ids, g.dist, w.N)


# --------------------------------------------------------------------------- Alg. 5
def test_prune_golden():
    gd = _golden("prune_line.json")
    P = _line_problem(gd["pos"])
    N = len(gd["pos"])
    lists = [[1, 2, 3, 4, 5]] + [[-1] * 5 for _ in range(N - 1)]
    g = O.KNNG(N, 5)
    for t, v in enumerate(lists[0]):
        g.ids[0, t] = v
        g.dist[0, t] = O.delta(P.X[0], P.X[v], 0)
    for case in gd["cases"]:
        T = np.full(N, 2, np.int32)
        for v in case["T1"]:
            T[v] = 1
        e_ids, e_dist, e_cnt, _ = O.prune(P, g, T, case["R"], case["alpha"])
        assert e_ids[0, :e_cnt[0]].tolist() == case["kept"], case


def test_prune_exact_tie_is_pruned():
    gd = _golden("prune_line.json")["tie_case"]
    X = np.asarray(gd["pts"], np.float32)
    P = O.Problem(X, [3], np.full((3, 1), -1, np.int32), np.zeros(1, np.int32), 0)
    g = O.KNNG(3, 2)
    g.ids[0] = [1, 2]
    g.dist[0] = [O.delta(X[0], X[1], 0), O.delta(X[0], X[2], 0)]
    assert g.dist[0].tolist() == [1.0, 1.25]
    for case in gd["cases"]:
        T = np.full(3, 2, np.int32)
        for v in case["T1"]:
            T[v] = 1
        e_ids, _, e_cnt, _ = O.prune(P, g, T, case["R"], case["alpha"])
        assert e_ids[0, :e_cnt[0]].tolist() == case["kept"]


def test_prune_line_keeps_one_per_side():
    """alpha=1 on a line: only the nearest neighbour on each side survives (all T > 1)."""
    rng = np.random.default_rng(4)
    pos = np.concatenate([[0.0], rng.uniform(-10, 10, 30)])
    P = _line_problem(pos)
    N = len(pos)
    d = (pos[1:] - pos[0]) ** 2
    order = np.lexsort((np.arange(1, N), d)) + 1
    g = O.KNNG(N, N - 1)
    for t, v in enumerate(order):
        g.ids[0, t] = v
        g.dist[0, t] = O.delta(P.X[0], P.X[v], 0)
    T = np.full(N, 2, np.int32)
    e_ids, _, e_cnt, _ = O.prune(P, g, T, 8, 1.0)
    kept = e_ids[0, :e_cnt[0]]
    right = [v for v in range(1, N) if pos[v] > 0]
    left = [v for v in range(1, N) if pos[v] < 0]
    expect = {min(right, key=lambda v: pos[v]), max(left, key=lambda v: pos[v])}
    assert set(kept.tolist()) == expect


def test_prune_invariants(small_problem):
    w, graphs, P = small_problem
    g, _, _ = O.stage_a(P, w.k)
    T = O.indegree(g.ids)
    e_ids, e_dist, e_cnt, _ = O.prune(P, g, T, w.R, w.alpha)
    a2 = np.float32(w.alpha) ** 2
    for u in range(0, w.N, 331):
        kept = e_ids[u, :e_cnt[u]].tolist()
        row = g.ids[u].tolist()
        assert kept == [v for v in row if v in set(kept)], "kept in list order"
        assert e_cnt[u] <= w.R
        # no kept, unprotected v is occluded by a kept w that precedes it
        for j, v in enumerate(kept):
            if T[v] == 1:
                continue
            for wv in kept[:j]:
                assert e_dist[u, j] < np.float32(a2 * np.float32(O.delta(P.X[wv], P.X[v], 0)))


def test_reverse_insert_invariants(small_problem):
    w, graphs, P = small_problem
    g, _, _ = O.stage_a(P, w.k)
    T = O.indegree(g.ids)
    e_ids, e_dist, e_cnt, _ = O.prune(P, g, T, w.R, w.alpha)
    o_ids, o_dist, o_deg = O.reverse_insert(e_ids, e_dist, e_cnt)
    _check_lists(o_ids, o_dist, w.N)
    assert np.all(o_deg <= w.R)
    E = {(u, int(v)) for u in range(w.N) for v in e_ids[u, :e_cnt[u]]}
    out = {(u, int(v)) for u in range(w.N) for v in o_ids[u, :o_deg[u]]}
    assert out <= (E | {(v, u) for (u, v) in E})
    for (u, v) in list(E)[::50]:
        if (v, u) not in out:
            # v's list is full of entries no worse than (delta(u,v), u)
            assert o_deg[v] == w.R
            duv = e_dist[u, list(e_ids[u]).index(v)]
            assert (o_dist[v, -1], o_ids[v, -1]) <= (duv, u)


# --------------------------------------------------------------------------- reachability fix
def test_reach_fix_attaches_one_rep_per_component():
    # three far-apart clusters of 1-D points; each cluster a clique
    pos = [0, 1, 2, 100, 101, 102, 103, 200, 201]
    P = _line_problem(pos)
    clusters = [[0, 1, 2], [3, 4, 5, 6], [7, 8]]
    R = 6
    N = len(pos)
    ids = np.full((N, R), -1, np.int32)
    dist = np.full((N, R), np.inf, np.float32)
    deg = np.zeros(N, np.int32)
    for c in clusters:
        for u in c:
            nb = sorted((O.delta(P.X[u], P.X[v], 0), v) for v in c if v != u)
            for t, (dv, v) in enumerate(nb):
                ids[u, t], dist[u, t] = v, dv
            deg[u] = len(nb)
    st = O.reach_fix(P, ids, dist, deg, 0)
    assert st["attached"] == 2 and st["unreached"] == 0
    # cluster [3..6] is represented by 3 and hangs under the nearest reached vertex (2)
    assert 3 in ids[2, :deg[2]].tolist()
    # in the same round, cluster [7, 8] is represented by 7 and searched over the round-start graph:
    # its nearest reached vertex is 2 again
    assert 7 in ids[2, :deg[2]].tolist()
    _check_lists(ids, dist, N)


def test_reach_fix_victim_golden():
    gd = _golden("reach_victim.json")
    P = _line_problem(gd["pos"])
    R = gd["R"]
    N = len(gd["pos"])
    ids = np.asarray(gd["lists"], np.int32)
    dist = np.full((N, R), np.inf, np.float32)
    deg = (ids >= 0).sum(1).astype(np.int32)
    for u in range(N):
        for t in range(deg[u]):
            dist[u, t] = O.delta(P.X[u], P.X[ids[u, t]], 0)
    st = O.reach_fix(P, ids, dist, deg, gd["entry"])
    assert ids.tolist() == gd["expected_lists"]
    assert dist[2].tolist() == gd["expected_dist_row2"]
    assert st["attached"] == gd["expected_attached"] and st["unreached"] == 0


# --------------------------------------------------------------------------- end to end
def test_merge_small_invariants(small_problem):
    w, graphs, P = small_problem
    r = O.merge(P, w.k, w.R, w.alpha)
    _check_lists(r.ids, r.dist, w.N)
    _check_lists(r.knn_ids, r.knn_dist, w.N)
    assert np.all(r.deg <= w.R)
    assert r.stats["unreached"] == 0
    assert r.entry == O.merged_entry(P) == graphs[0][1]   # equal shards: the first shard's entry


def test_merge_uniform_recall_and_exhaustive_search():
    rng = np.random.default_rng(21)
    from synth import pgbuild
    X = rng.uniform(0, 1, (4000, 8)).astype(np.float32)
    Q = rng.uniform(0, 1, (200, 8)).astype(np.float32)
    sizes = [2000, 2000]
    graphs = [pgbuild.build_pg(X[:2000], 16, 64, 0), pgbuild.build_pg(X[2000:], 16, 64, 0)]
    P = O.Problem(X, sizes, np.concatenate([graphs[0][0], graphs[1][0]]),
                  np.array([graphs[0][1], graphs[1][1]], np.int32), 0)
    r = O.merge(P, 16, 32, 1.2)
    gt, _ = O.knn_exact(X, Q, 10, 0)
    ids, _, _ = O.search(X, r.ids, r.entry, Q, 64, 10, 0)
    assert O.recall_at(ids, gt, 10) >= 0.95
    # beam >= N on a graph where everything is reachable is exhaustive
    ids_all, _, st = O.search(X, r.ids, r.entry, Q[:5], 4000, 10, 0)
    assert np.array_equal(ids_all, gt[:5])


def test_merge_thread_count_independent(small_problem):
    w, graphs, _ = small_problem
    P1 = O.Problem.from_workload(w, graphs, nthreads=1)
    a = O.merge(P1, w.k, w.R, w.alpha, iters=1)
    P4 = O.Problem.from_workload(w, graphs, nthreads=4)
    b = O.merge(P4, w.k, w.R, w.alpha, iters=1)
    assert np.array_equal(a.ids, b.ids) and np.array_equal(a.dist, b.dist)
    assert np.array_equal(a.knn_ids, b.knn_ids)


def test_batched_recipe_bf16_storage():
    """The batched recipe's storage step is BF16 round-to-nearest-even (torch's conversion) and
    its vectors are unit-norm up to that rounding."""
    import torch
    from synth import gen
    x = np.random.default_rng(1).standard_normal(50_000).astype(np.float32) * 3
    assert np.array_equal(gen.bf16_round(x), torch.from_numpy(x).to(torch.bfloat16).float().numpy())
    assert gen.bf16_round(np.array([1.0 + 2.0 ** -8], np.float32))[0] == 1.0          # tie -> even
    assert gen.bf16_round(np.array([1.0 + 3 * 2.0 ** -8], np.float32))[0] == 1.0 + 2.0 ** -6  # tie -> even (up)
    w = gen.batched_one(N=500, h=4, d=64, nq=10)
    assert w.dtype == "bf16" and w.metric == gen.METRIC_COS and w.shard_sizes == [125] * 4
    assert np.array_equal(gen.bf16_round(w.X), w.X)
    assert np.abs(np.linalg.norm(w.X.astype(np.float64), axis=1) - 1).max() < 4 * 2.0 ** -8
    hs = [wk.h for wk in gen.batched(n_merges=12, n_lo=100, n_hi=400, d=16, nq=4)]
    assert min(hs) >= 2 and max(hs) <= 6


# --------------------------------------------------------------------------- phi with invalid vertices
def _small_problem(N=900, h=3, seed=7):
    from synth import gen, pgbuild
    w = gen.small(seed=seed, N=N, d=8, h=h, nq=4)
    graphs = pgbuild.build_all(w)
    return w, O.Problem.from_workload(w, graphs)


def _with_valid(P, valid):
    return O.Problem(P.X, P.sizes, P.adj, P.entry, P.metric, valid=valid)


def test_phi_numbers_valid_vertices_in_shard_order():
    """Sec. 4.1.3: phi gives the valid vertices consecutive ids in (shard, local id) order."""
    w, P = _small_problem()
    valid = np.random.default_rng(1).random(P.N) < 0.7
    phi = _with_valid(P, valid).phi()
    assert np.array_equal(phi[~valid], np.full((~valid).sum(), -1))
    assert np.array_equal(phi[valid], np.arange(valid.sum()))
    assert np.array_equal(_with_valid(P, None).phi(), np.arange(P.N))


def test_all_valid_mask_is_the_plain_merge():
    w, P = _small_problem()
    a = O.merge(P, w.k, w.R, w.alpha, iters=2)
    b = O.merge(_with_valid(P, np.ones(P.N, np.uint8)), w.k, w.R, w.alpha, iters=2)
    assert np.array_equal(a.ids, b.ids) and np.array_equal(a.dist, b.dist)
    assert np.array_equal(a.knn_ids, b.knn_ids) and a.entry == b.entry


def test_fully_invalid_shard_equals_merge_without_it():
    """A shard whose every vertex is invalid contributes nothing: with the same L the merge
    equals the merge of the other shards (its searches return only vertices phi drops)."""
    w, P = _small_problem(N=900, h=3)
    valid = np.ones(P.N, np.uint8)
    valid[P.off[2]:] = 0
    a = O.merge(_with_valid(P, valid), w.k, w.R, w.alpha, L=8, iters=2)
    n2 = int(P.off[2])
    P2 = O.Problem(P.X[:n2], P.sizes[:2], P.adj[:n2], P.entry[:2], P.metric)
    b = O.merge(P2, w.k, w.R, w.alpha, L=8, iters=2)
    assert a.ids.shape == (n2, w.R)
    assert np.array_equal(a.knn_ids, b.knn_ids) and np.array_equal(a.knn_dist, b.knn_dist)
    assert np.array_equal(a.ids, b.ids) and np.array_equal(a.deg, b.deg) and a.entry == b.entry


def test_masked_cross_query_filters_the_unmasked_candidates():
    """With k >= M + (h - 1) L nothing is cut by the top-k, so the masked k-NNG row of a valid
    vertex is its unmasked row with the invalid ids removed and the rest renumbered by phi."""
    w, P = _small_problem(N=600, h=3)
    L = 4
    k = P.adj.shape[1] + (P.h - 1) * L
    valid = np.random.default_rng(3).random(P.N) < 0.6
    Pv = _with_valid(P, valid)
    phi = Pv.phi()
    full, _, _ = O.stage_a(P, k, L)
    part, _, _ = O.stage_a(Pv, k, L)
    assert part.ids.shape == (int(valid.sum()), k)
    for g in np.nonzero(valid)[0]:
        ids, dist = full.ids[g], full.dist[g]
        keep = (ids >= 0) & valid[np.maximum(ids, 0)]
        want = phi[ids[keep]]
        row = part.ids[phi[g]]
        assert np.array_equal(row[:len(want)], want), g
        assert np.all(row[len(want):] == -1)
        assert np.array_equal(part.dist[phi[g]][:len(want)], dist[keep])
    assert np.all(part.ids < valid.sum())


def test_merged_entry_with_invalid_entry():
    """The entry is the entry of the shard with the most valid vertices (lowest index on ties)
    if valid, else that shard's first valid vertex."""
    w, P = _small_problem(N=901, h=3)          # shard sizes 301, 300, 300
    assert list(P.sizes) == [301, 300, 300]
    valid = np.ones(P.N, np.uint8)
    valid[P.off[0] + P.entry[0]] = 0           # shard 0 keeps 300 valid vertices: still first on the tie
    Pv = _with_valid(P, valid)
    phi = Pv.phi()
    first_valid = phi[P.off[0]:P.off[1]][phi[P.off[0]:P.off[1]] >= 0][0]
    assert O.merged_entry(Pv) == first_valid == 0
    valid2 = np.ones(P.N, np.uint8)
    valid2[P.off[0]:P.off[0] + 200] = 0        # shard 0 now has the fewest valid vertices
    valid2[P.off[2]:P.off[2] + 10] = 0         # and shard 1 the most
    Pv2 = _with_valid(P, valid2)
    assert O.merged_entry(Pv2) == Pv2.phi()[P.off[1] + P.entry[1]]


# --------------------------------------------------------------------------- HNSW-adaptive merging
def test_splitmix64_known_outputs():
    """SplitMix64 from state 0: its first three published outputs."""
    assert O.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert O.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert O.splitmix64(0, 2) == 0x06C45D188009454F


def test_hnsw_level_distribution():
    """P(level >= l) = M^-l: thresholds are exact integer quotients; counts within 5 sigma."""
    M = 8
    T = O.level_thresholds(M)
    assert T[0] == ((1 << 64) - 1) // 8 and T[1] == ((1 << 64) - 1) // 64
    assert all(a > b for a, b in zip(T, T[1:]))
    n = 40_000
    lv = O.hnsw_levels(n, M, seed=5)
    for l in (1, 2, 3):
        p = M ** -l
        got = int((lv >= l).sum())
        assert abs(got - n * p) <= 5 * np.sqrt(n * p * (1 - p)) + 1, (l, got)
    assert np.array_equal(O.hnsw_levels(1000, M, seed=5), lv[:1000])   # counter-based: prefix-stable


def test_hnsw_layer_collinear():
    """Three points on a line a - b - c: the heuristic drops c from a's list (b is nearer to c
    than a is) and a from c's; b keeps both; reverse edges add nothing new."""
    X = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [3, 0, 0, 0]], np.float32)
    levels = np.array([1, 1, 1], np.int32)
    members, adj, deg = O.hnsw_layer(X, 0, levels, 1, M=4, ef=4)
    assert list(members) == [0, 1, 2]
    assert list(adj[0][:deg[0]]) == [1]
    assert list(adj[1][:deg[1]]) == [0, 2]
    assert list(adj[2][:deg[2]]) == [1]


def test_hnsw_layer_invariants():
    """Rows sorted by distance, no self or duplicate, degree <= M, every kept pair obeys the
    RNG rule, and a layer holds exactly the vertices of that level or higher."""
    from synth import gen
    w = gen.small(seed=3, N=3000, d=8, h=2, nq=4)
    levels = O.hnsw_levels(w.N, 8, seed=11)
    members, adj, deg = O.hnsw_layer(w.X, 0, levels, 1, M=8, ef=32)
    assert np.array_equal(members, np.nonzero(levels >= 1)[0])
    Xl = w.X[members].astype(np.float64)
    for u in range(len(members)):
        row = adj[u][:deg[u]]
        assert deg[u] <= 8 and len(set(row)) == len(row) and u not in row and np.all(adj[u][deg[u]:] == -1)
        du = [np.sum((Xl[u] - Xl[v]) ** 2) for v in row]
        assert all(a <= b for a, b in zip(du, du[1:]))
        for j in range(len(row)):
            for i in range(j):
                assert du[j] < np.sum((Xl[row[i]] - Xl[row[j]]) ** 2) * (1 + 1e-5)


def test_hnsw_search_descends_to_the_nearest_member():
    """On a path graph layer over points on a line, the descent ends at the member nearest to
    the query, and the base search starts there; with a pool (ef_up > 1) the layer search
    passes a vertex that greedy stops at."""
    X = np.array([[float(i), 0, 0, 0] for i in range(10)], np.float32)
    members = np.array([0, 3, 6, 9], np.int32)
    adj = np.array([[1, -1], [0, 2], [1, 3], [2, -1]], np.int32)
    base = np.array([[(i + 1) % 10, (i + 9) % 10] for i in range(10)], np.int32)
    Q = np.array([[7.2, 0, 0, 0], [1.4, 0, 0, 0]], np.float32)
    for ef_up in (1, 4):   # greedy, and a pool over the whole path
        ids, dist, starts = O.hnsw_search(X, 0, base, [(members, adj)], 0, Q, beam=4, topk=2, ef_up=ef_up)
        assert list(starts) == [6, 0]
        assert list(ids[0]) == [7, 8] and list(ids[1]) == [1, 2]
    # a layer where greedy stops early: 0 - 3 - 9 - 6; the query at 5 is nearest to 6, but from
    # 3 every neighbour (0, 9) is farther than 3 itself
    adj2 = np.array([[1, -1], [0, 3], [3, -1], [1, 2]], np.int32)   # positions: 0:0, 1:3, 2:6, 3:9
    Q2 = np.array([[5.0, 0, 0, 0]], np.float32)
    _, _, s1 = O.hnsw_search(X, 0, base, [(members, adj2)], 0, Q2, beam=4, topk=2, ef_up=1)
    _, _, s4 = O.hnsw_search(X, 0, base, [(members, adj2)], 0, Q2, beam=4, topk=2, ef_up=4)
    assert s1[0] == 3 and s4[0] == 6


def test_hnsw_layer_links_across_clusters():
    """Two far clusters with interleaved ids: a member links to its nearest among the members
    inserted before it, so early members link across the gap and the layer stays connected
    (nearest neighbours over all members, ef = 8, would split it in two)."""
    rng = np.random.default_rng(4)
    a = rng.normal(0, 0.1, (20, 4))
    b = rng.normal(0, 0.1, (20, 4)) + 100.0
    X = np.empty((40, 4), np.float32)
    X[0::2], X[1::2] = a, b
    members, adj, deg = O.hnsw_layer(X, 0, np.ones(40, np.int32), 1, M=4, ef=8)
    seen, todo = {0}, [0]
    while todo:
        u = todo.pop()
        for v in list(adj[u][:deg[u]]) + [x for x in range(40) if u in adj[x][:deg[x]]]:
            if v not in seen:
                seen.add(int(v))
                todo.append(int(v))
    assert len(seen) == 40


def test_synchronous_refinement_matches_the_literal_dfs_form_in_quality():
    """Alg. 3 as printed (DFS order, streamlined Visit + Update) against the synchronous form
    the GPU runs: both raise the k-NNG recall of stage (a), and the synchronous form stays
    within one point of the literal one after three iterations; the literal form's lists are
    valid k-NN lists."""
    from synth import gen, pgbuild
    from tests import _parity as PR
    w = gen.make("small", N=20_000, nq=10)
    graphs = pgbuild.build_all(w)
    P = O.Problem.from_workload(w, graphs)
    g0, _, _ = O.stage_a(P, w.k)
    samp = np.random.default_rng(9).choice(w.N, 1000, replace=False)
    tid, _ = O.knn_exact(w.X, w.X[samp], w.k, w.metric, exclude=samp)
    gs = g0.copy()
    for _ in range(3):
        O.refine_iter(P, gs)
        O.indegree_repair(P, gs)
    gd = g0.copy()
    O.refine_dfs(P, gd, 3)
    PR.check_lists(gd.ids, gd.dist, w.N)
    r0, rs, rd = (O.recall_at(g.ids[samp], tid, w.k) for g in (g0, gs, gd))
    assert rs > r0 + 0.01 and rd > r0 + 0.01
    assert abs(rs - rd) <= 0.01, (rs, rd)


def test_refine_dfs_pins():
    """The literal DFS form: the exact k-NNG is a fixed point (no update is accepted and the
    repair finds nothing to change), and on complete local graphs it completes the cross part."""
    X, sizes = _two_shard_uniform()
    P = _complete_problem(X, sizes)
    k = 8
    gt, gd = O.knn_exact(X, X, k, O_METRIC_L2, exclude=np.arange(X.shape[0]))
    g = O.KNNG(X.shape[0], k)
    g.ids[:], g.dist[:], g.flags[:] = gt, gd, O.FLAG_NEW
    T, st = O.refine_dfs(P, g, 1)
    assert st["updates"] == 0 and st["pairs"] > 0
    assert np.array_equal(g.ids, gt) and np.array_equal(g.dist, gd)
    X2, sizes2 = _two_shard_uniform(N=800, d=3, seed=3)
    P2 = _complete_problem(X2, sizes2)
    g2, _, _ = O.stage_a(P2, k, 2)
    gt2, _ = O.knn_exact(X2, X2, k, O_METRIC_L2, exclude=np.arange(X2.shape[0]))
    r0 = O.recall_at(g2.ids, gt2, k)
    O.refine_dfs(P2, g2, 6)
    assert r0 < 0.95 and O.recall_at(g2.ids, gt2, k) >= 0.99


def test_knn_prefix_is_brute_force_over_earlier_rows():
    """or_knn_prefix: row i's k nearest among rows 0 .. i - 1, by (distance, id)."""
    rng = np.random.default_rng(2)
    X = np.round(rng.random((60, 4)) * 8).astype(np.float32)   # integer coordinates: ties by id
    k = 5
    ids = np.empty((60, k), np.int32)
    dist = np.empty((60, k), np.float32)
    O.lib().or_knn_prefix(X.ctypes.data, 60, 4, 0, k, 0, ids.ctypes.data, dist.ctypes.data)
    for i in range(60):
        d = ((X[:i].astype(np.float64) - X[i]) ** 2).sum(1)
        order = sorted(range(i), key=lambda j: (d[j], j))[:k]
        want = order + [-1] * (k - len(order))
        assert list(ids[i]) == want, i


# --------------------------------------------------------------------------- alternative neighbour selection
# Sec. 4.3.1: RNG, MRNG and tau-MNG are interchangeable neighbour-selection rules. Expected lists
# below are derived by hand from each rule's definition (all distances exact in FP32).
def _rule_case(points, lists, T=None):
    X = np.zeros((len(points), 4), np.float32)
    for i, p in enumerate(points):
        X[i, :len(p)] = p
    P = O.Problem(X, [len(points)], np.full((len(points), 1), -1, np.int32), np.zeros(1, np.int32), O_METRIC_L2)
    g = _knng_from_lists(P, lists)
    return P, g, np.full(len(points), 2, np.int32) if T is None else np.asarray(T, np.int32)


def test_prune_rules_line_golden():
    """u = 0, w = 1, v' = -2, v = 3 on a line. delta(u,.) = 1, 4, 9; delta(w,v') = 9, delta(w,v) = 4,
    delta(v',v) = 25. alpha-RNG (alpha 1) and MRNG: w occludes v (4 < 9), v' survives. tau-MNG
    with tau = 0.25: sqrt(9) - 0.75 = 2.25, 4 < 2.25^2 = 5.0625, so w occludes v; with tau = 0.4:
    3 - 1.2 = 1.8, 4 > 3.24 and 25 > 3.24, v is kept; with tau = 1 no edge is pruned (t <= 0)."""
    P, g, T = _rule_case([[0.], [1.], [-2.], [3.]], [[1, 2, 3], [0, 2, 3], [0, 1, 3], [1, 0, 2]])
    expect = {("arng", 0.0): [1, 2], ("mrng", 0.0): [1, 2], ("tmng", 0.25): [1, 2], ("tmng", 0.4): [1, 2, 3],
              ("tmng", 1.0): [1, 2, 3]}
    for (rule, tau), want in expect.items():
        e_ids, e_dist, e_cnt, _ = O.prune(P, g, T, 3, 1.0, rule, tau)
        assert e_ids[0, :e_cnt[0]].tolist() == want, (rule, tau)
        assert e_dist[0, :e_cnt[0]].tolist() == [{1: 1.0, 2: 4.0, 3: 9.0}[x] for x in want]


def test_prune_mrng_keeps_the_equidistant_candidate():
    """u = (0,0), w = (2,0), v = (1,2): delta(u,w) = 4, delta(u,v) = delta(w,v) = 5. alpha-RNG with
    alpha = 1 prunes v (5 <= 1 * 5); MRNG keeps it (uv is not strictly the longest edge)."""
    P, g, T = _rule_case([[0., 0.], [2., 0.], [1., 2.]], [[1, 2], [0, 2], [0, 1]])
    a, _, ca, _ = O.prune(P, g, T, 2, 1.0, "arng")
    m, _, cm, _ = O.prune(P, g, T, 2, 1.0, "mrng")
    assert a[0, :ca[0]].tolist() == [1]
    assert m[0, :cm[0]].tolist() == [1, 2]


def test_prune_rules_keep_protected_vertices():
    """Alg. 5's indegree clause holds for every rule: a candidate with T = 1 is kept although an
    earlier kept neighbour occludes it."""
    P, g, T = _rule_case([[0.], [1.], [-2.], [3.]], [[1, 2, 3], [0, 2, 3], [0, 1, 3], [1, 0, 2]], T=[2, 2, 2, 1])
    for rule in ("arng", "mrng", "tmng"):
        e_ids, _, e_cnt, _ = O.prune(P, g, T, 3, 1.0, rule, 0.25)
        assert e_ids[0, :e_cnt[0]].tolist() == [1, 2, 3], rule


def test_prune_tmng_large_tau_is_top_r_truncation(small_problem):
    """With 3 tau above every distance, tau-MNG prunes nothing: E'(u) is the first R entries."""
    w, graphs, P = small_problem
    g, _, _ = O.stage_a(P, w.k)
    T = np.full(w.N, 2, np.int32)
    tau = float(np.sqrt(np.nanmax(g.dist[np.isfinite(g.dist)]))) + 1.0
    e_ids, e_dist, e_cnt, _ = O.prune(P, g, T, 8, 1.0, "tmng", tau)
    n = (g.ids >= 0).sum(1)
    assert np.array_equal(e_cnt, np.minimum(n, 8))
    assert np.array_equal(e_ids[:, :8][e_cnt == 8], g.ids[:, :8][e_cnt == 8])


def test_prune_rules_invariants(small_problem):
    """Every rule: degree <= R, the kept entries are a sorted subsequence of the list, and the
    MRNG and tau-MNG lists are never shorter than alpha-RNG's with alpha = 1 on the same input at
    the first candidate they disagree on (both keep the nearest candidate)."""
    w, graphs, P = small_problem
    g, _, _ = O.stage_a(P, w.k)
    T = O.indegree(g.ids)
    for rule, tau in (("arng", 0.0), ("mrng", 0.0), ("tmng", 0.5)):
        e_ids, e_dist, e_cnt, _ = O.prune(P, g, T, 8, 1.0, rule, tau)
        assert np.all(e_cnt <= 8) and np.all(e_cnt >= np.minimum(1, (g.ids >= 0).sum(1)))
        for u in range(0, w.N, 499):
            row = g.ids[u].tolist()
            kept = e_ids[u, :e_cnt[u]].tolist()
            pos = [row.index(x) for x in kept]
            assert pos == sorted(pos) and kept[0] == row[0]


# --------------------------------------------------------------------------- HNSW's sequential insertion
def test_hnsw_insert_golden():
    """Four points on a line, inserted in id order at x = 0, 10, 1, 11 (all level 1, M = 1, ef = 4),
    traced by hand: 1 links to 0 and 0 back to 1; 2 finds 0 and 1, keeps 0, and 0's overfull list
    {1, 2} is re-pruned to {2} (2 occludes 1: 81 <= 100); 3, searched from the entry 0, reaches 0
    and 2 only, keeps 2, and 2's list {0, 3} is cut to {0}."""
    X = np.zeros((4, 4), np.float32)
    X[:, 0] = [0, 10, 1, 11]
    layers, entry = O.hnsw_insert_layers(X, O_METRIC_L2, np.ones(4, np.int32), 1, 4)
    assert entry == 0 and len(layers) == 1
    members, adj, deg = layers[0]
    assert members.tolist() == [0, 1, 2, 3]
    assert adj[:, 0].tolist() == [2, 0, 0, 2]
    # the layer built at once from exact prefix candidates links 3 to 1 (its true nearest earlier
    # member), which the sequential search from the entry could not reach
    m2, adj2, _ = O.hnsw_layer(X, O_METRIC_L2, np.ones(4, np.int32), 1, 1, 4)
    assert adj2[3, 0] == 1


def test_hnsw_insert_layers_invariants(small_problem):
    w, graphs, P = small_problem
    levels = O.hnsw_levels(w.N, 8, seed=5)
    layers, entry = O.hnsw_insert_layers(w.X, w.metric, levels, 8, 32)
    assert levels[entry] == levels.max() and entry == int(np.argmax(levels))
    for l, (members, adj, deg) in enumerate(layers, start=1):
        assert np.array_equal(members, np.nonzero(levels >= l)[0])
        assert adj.shape == (len(members), 8) and np.all(deg <= 8)
        for r in range(len(members)):
            row = adj[r][adj[r] >= 0]
            assert len(set(row.tolist())) == len(row) and r not in set(row.tolist())
            assert np.all(adj[r][len(row):] == -1)


def test_parallel_layers_match_the_sequential_insertion_in_quality(small_problem):
    """The layers built at once (every member's exact ef nearest earlier members) against HNSW's
    sequential insertion (Sec. 4.3.3 as printed): over the same merged base graph, the layered
    search's recall@10 (1,000 queries, beam 32, ef_up 8) stays within one point."""
    w, graphs, P = small_problem
    r = O.merge(P, w.k, w.R, w.alpha, iters=1)
    levels = O.hnsw_levels(w.N, 8, seed=5)
    seq, entry = O.hnsw_insert_layers(w.X, w.metric, levels, 8, 32)
    par = [O.hnsw_layer(w.X, w.metric, levels, l, 8, 32) for l in range(1, len(seq) + 1)]
    Q = w.Q[:1000]
    gt, _ = O.knn_exact(w.X, Q, 10, w.metric)
    rs = O.recall_at(O.hnsw_search(w.X, w.metric, r.ids, [(m, a) for m, a, _ in seq], entry, Q, 32, 10, 8)[0], gt, 10)
    rp = O.recall_at(O.hnsw_search(w.X, w.metric, r.ids, [(m, a) for m, a, _ in par], O.hnsw_entry(levels), Q, 32,
                                   10, 8)[0], gt, 10)
    assert rp >= rs - 0.01, (rp, rs)


# --------------------------------------------------------------------------- reachability fix, plain form
def test_reach_fix_rounds_against_the_plain_sequential_rule(small_problem):
    """The round-based reachability fix (the form the kernels follow) against the plain sequential
    rule (each unreached vertex in ascending id attached to the first reached vertex of its k-NNG
    list or search results with room, else with a neighbour of indegree > 1): both leave every
    vertex reachable from the entry and both lift the flat search's recall far above the graph
    without the fix (the two attach differently, so their recalls are reported, not equated)."""
    w, graphs, P = small_problem
    r = O.merge(P, w.k, w.R, w.alpha, iters=1, ensure_reachable=False)
    assert not _bfs_all(r.ids, r.entry)
    a_ids, a_dist, a_deg = r.ids.copy(), r.dist.copy(), r.deg.copy()
    b_ids, b_dist, b_deg = r.ids.copy(), r.dist.copy(), r.deg.copy()
    sa = O.reach_fix(P, a_ids, a_dist, a_deg, r.entry, 64)
    sb = O.reach_fix_seq(P, b_ids, b_dist, b_deg, r.entry, 64, knn_ids=r.knn_ids)
    assert sa["unreached"] == 0 and sb["unreached"] == 0
    assert _bfs_all(a_ids, r.entry) and _bfs_all(b_ids, r.entry)
    assert sa["attached"] > 0 and sb["attached"] > 0
    Q = w.Q[:1000]
    gt, _ = O.knn_exact(w.X, Q, 10, w.metric)
    r0 = O.recall_at(O.search(w.X, r.ids, r.entry, Q, 64, 10, w.metric)[0], gt, 10)
    ra = O.recall_at(O.search(w.X, a_ids, r.entry, Q, 64, 10, w.metric)[0], gt, 10)
    rb = O.recall_at(O.search(w.X, b_ids, r.entry, Q, 64, 10, w.metric)[0], gt, 10)
    assert ra > r0 + 0.2 and rb > r0 + 0.2, (r0, ra, rb)


def test_plain_reach_fix_can_cut_off_vertices_the_round_form_keeps():
    """Why the round-based form replaces only a neighbour that keeps another BFS parent: on the
    Sift-like recipe (12,000 points) the plain rule's 'indegree > 1' victim can lose its only
    reached in-edge, and vertices stay unreachable; the round-based form reaches every vertex
    with as many attachments."""
    from synth import gen, pgbuild
    w = gen.make("medium", N=12000, nq=10, n_centers=12)
    P = O.Problem.from_workload(w, pgbuild.build_all(w))
    r = O.merge(P, w.k, w.R, w.alpha, iters=2, ensure_reachable=False)
    a = (r.ids.copy(), r.dist.copy(), r.deg.copy())
    b = (r.ids.copy(), r.dist.copy(), r.deg.copy())
    sa = O.reach_fix(P, *a, r.entry, 64)
    sb = O.reach_fix_seq(P, *b, r.entry, 64, knn_ids=r.knn_ids)
    assert sa["unreached"] == 0 and _bfs_all(a[0], r.entry)
    assert sb["unreached"] > 0 and not _bfs_all(b[0], r.entry)


def _bfs_all(ids, entry):
    seen = np.zeros(ids.shape[0], bool)
    seen[entry] = True
    stack = [entry]
    while stack:
        x = stack.pop()
        for y in ids[x]:
            if y >= 0 and not seen[y]:
                seen[y] = True
                stack.append(int(y))
    return bool(seen.all())
