"""Brute-force pin of the oracle's refinement pass (Alg. 3, Sec. 4.2.1).

One synchronous Visit + Update pass is restated here from its definition, in plain Python
sets and sorts, and the oracle's ``or_refine_iter`` must give the same lists, distances and
flags entry for entry:

  Visit   forward entries split by their `new` flag; reverse lists Gbar_n(v), Gbar_o(v) built
          from the lists as they stand when the pass starts, each cut to the rev_cap smallest
          (distance, source id); C_n(v) = new forward U new reverse, C_o(v) = (old forward U
          old reverse) minus C_n(v); every forward entry is old afterwards.
  Update  every unordered pair {a, b} of C_n(v)^2 U C_n(v) x C_o(v) with a != b whose two
          vertices come from different input graphs proposes b to list(a) and a to list(b).
  merge   each list becomes the top-k by (distance, id) of its own entries and every
          proposal, duplicates by id removed; an inserted entry carries the `new` flag.

Integer coordinates make every squared distance exact, so the restatement and the oracle
agree bit for bit, and the many equal distances exercise the id tie-break.
"""
import numpy as np
import pytest

import oracle as O

L2 = 0


def _random_knng(X, k, rng, fill=0.85, p_new=0.5, p_replaced=0.1):
    """A valid k-NNG over X: rows of distinct non-self ids (some rows short, -1 padded),
    sorted by (distance, id), with random new / replaced flags."""
    N = X.shape[0]
    ids = np.full((N, k), -1, np.int32)
    dist = np.full((N, k), np.inf, np.float32)
    flags = np.zeros((N, k), np.uint8)
    for u in range(N):
        m = k if rng.random() < fill else int(rng.integers(0, k))
        cand = rng.choice(np.delete(np.arange(N), u), size=m, replace=False)
        ent = sorted(((float(((X[u] - X[v]) ** 2).sum()), int(v)) for v in cand))
        for t, (d, v) in enumerate(ent):
            ids[u, t] = v
            dist[u, t] = d
            flags[u, t] = (O.FLAG_NEW if rng.random() < p_new else 0) | \
                          (O.FLAG_REPLACED if rng.random() < p_replaced else 0)
    return ids, dist, flags


def brute_refine_pass(X, shard, ids, dist, flags, k, rev_cap, plant=None):
    """One synchronous Visit + Update pass, restated from the definition. Returns the new
    (ids, dist, flags) and the number of pair evaluations. `plant` (tests only) substitutes
    one plausible mistake: "largest" keeps the rev_cap largest reverse entries, "old_old"
    also joins C_o x C_o, "no_dedupe" leaves C_o overlapping C_n (its pairs counted twice),
    "flag_kept" leaves visited entries new."""
    N = X.shape[0]
    rev = {True: [[] for _ in range(N)], False: [[] for _ in range(N)]}
    for u in range(N):
        for t in range(k):
            v = int(ids[u, t])
            if v >= 0:
                rev[bool(flags[u, t] & O.FLAG_NEW)][v].append((float(dist[u, t]), u))
    pairs = set()
    n_eval = 0
    for v in range(N):
        fwd_new = {int(ids[v, t]) for t in range(k) if ids[v, t] >= 0 and flags[v, t] & O.FLAG_NEW}
        fwd_old = {int(ids[v, t]) for t in range(k) if ids[v, t] >= 0 and not flags[v, t] & O.FLAG_NEW}
        order = (lambda r: sorted(r, reverse=True)) if plant == "largest" else sorted
        rn = {u for _, u in order(rev[True][v])[:rev_cap]}
        ro = {u for _, u in order(rev[False][v])[:rev_cap]}
        cn = fwd_new | rn
        co = (fwd_old | ro) if plant == "no_dedupe" else (fwd_old | ro) - cn
        firsts = cn | co if plant == "old_old" else cn
        vpairs = set()
        for a in firsts:
            for b in cn | co:
                if a != b and shard[a] != shard[b]:
                    vpairs.add((min(a, b), max(a, b)))
        if plant == "no_dedupe":
            n_eval += sum(1 for a in cn for b in co & cn if a < b and shard[a] != shard[b])
        n_eval += len(vpairs)
        pairs |= vpairs
    proposals = [dict() for _ in range(N)]
    for a, b in pairs:
        d = np.float32(((X[a].astype(np.float64) - X[b]) ** 2).sum())
        proposals[a][b] = d
        proposals[b][a] = d
    out_i = np.full_like(ids, -1)
    out_d = np.full_like(dist, np.inf)
    out_f = np.zeros_like(flags)
    clear = 0 if plant == "flag_kept" else O.FLAG_NEW
    for a in range(N):
        ent = {}
        for t in range(k):
            if ids[a, t] >= 0:
                ent[int(ids[a, t])] = (float(dist[a, t]), int(flags[a, t]) & ~clear)
        for b, d in proposals[a].items():
            if b not in ent:
                ent[b] = (float(d), O.FLAG_NEW)
        top = sorted(ent.items(), key=lambda e: (e[1][0], e[0]))[:k]
        for t, (b, (d, f)) in enumerate(top):
            out_i[a, t], out_d[a, t], out_f[a, t] = b, d, f
    return out_i, out_d, out_f, n_eval


def _problem(N=300, sizes=(100, 120, 80), d=4, seed=5):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 12, (N, d)).astype(np.float32)
    P = O.Problem(X, list(sizes), np.full((N, 1), -1, np.int32), np.zeros(len(sizes), np.int32), L2)
    shard = np.repeat(np.arange(len(sizes)), sizes)
    return P, X, shard, rng


@pytest.mark.parametrize("rev_cap", [6, 2])
@pytest.mark.parametrize("seed", [5, 6])
def test_refine_pass_equals_brute_force(rev_cap, seed):
    P, X, shard, rng = _problem(seed=seed)
    k = 6
    ids, dist, flags = _random_knng(X, k, rng)
    ei, ed, ef, npairs = brute_refine_pass(X, shard, ids, dist, flags, k, rev_cap)
    g = O.KNNG(X.shape[0], k)
    g.ids[:], g.dist[:], g.flags[:] = ids, dist, flags
    st = O.refine_iter(P, g, rev_cap=rev_cap)
    assert st["pairs"] == npairs
    np.testing.assert_array_equal(g.ids, ei)
    np.testing.assert_array_equal(g.dist, ed)
    np.testing.assert_array_equal(g.flags, ef)


def test_refine_pass_after_stage_a_equals_brute_force():
    """The same check on the pass the merge actually runs first: stage (a) output (all new)
    over input graphs, then a second pass over its mixed new / old flags."""
    P, X, shard, rng = _problem(seed=9)
    N, k = X.shape[0], 6
    adj = np.full((N, 5), -1, np.int32)
    off = np.concatenate([[0], np.cumsum(P.sizes)])
    for s in range(P.h):
        n = P.sizes[s]
        for v in range(n):
            adj[off[s] + v] = rng.choice(np.delete(np.arange(n), v), size=5, replace=False)
    P = O.Problem(X, P.sizes, adj, np.zeros(P.h, np.int32), L2)
    g, _, _ = O.stage_a(P, k)
    for _ in range(2):
        ei, ed, ef, npairs = brute_refine_pass(X, shard, g.ids, g.dist, g.flags, k, k)
        st = O.refine_iter(P, g, rev_cap=k)
        assert st["pairs"] == npairs
        np.testing.assert_array_equal(g.ids, ei)
        np.testing.assert_array_equal(g.dist, ed)
        np.testing.assert_array_equal(g.flags, ef)


@pytest.mark.parametrize("plant", ["largest", "old_old", "no_dedupe", "flag_kept"])
def test_brute_force_restatement_catches_planted_mistakes(plant):
    """Each plausible mistake of a refinement pass, planted in the restatement, changes the
    lists, the flags or the number of pair evaluations on the test input, so a pass carrying
    it cannot satisfy the equalities above."""
    P, X, shard, rng = _problem(seed=5)
    k = 6
    ids, dist, flags = _random_knng(X, k, rng)
    ref = brute_refine_pass(X, shard, ids, dist, flags, k, 2)
    bad = brute_refine_pass(X, shard, ids, dist, flags, k, 2, plant=plant)
    same = (np.array_equal(ref[0], bad[0]) and np.array_equal(ref[1], bad[1])
            and np.array_equal(ref[2], bad[2]) and ref[3] == bad[3])
    assert not same
