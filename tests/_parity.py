"""Comparison rules shared by the GPU parity tests.

FP32 distances must match the oracle within RTOL relative (ATOL absolute for distances
near zero). Neighbour-id lists must be identical wherever the candidate distances are
further apart than that tolerance: ids may differ only inside a group of entries whose
oracle distances are within tolerance of each other, or at the list boundary where the
excluded and included candidates tie within tolerance.
"""
import numpy as np

RTOL = 1e-5
ATOL = 1e-6


def close(a, b, rtol=RTOL, atol=ATOL):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    both_inf = np.isinf(a) & np.isinf(b)
    with np.errstate(invalid="ignore"):  # inf - inf is covered by both_inf
        return both_inf | (np.abs(a - b) <= rtol * np.maximum(np.abs(a), np.abs(b)) + atol)


def row_matches(gi, gd, oi, od, rtol=RTOL, atol=ATOL) -> bool:
    """One list: GPU (gi, gd) against oracle (oi, od), both sorted by (dist, id)."""
    if np.array_equal(gi, oi):
        return bool(np.all(close(gd, od, rtol, atol)))
    gv, ov = gi >= 0, oi >= 0
    if gv.sum() != ov.sum():
        return False
    n = int(ov.sum())
    if n == 0:
        return True
    # position by position the distances agree
    if not np.all(close(gd[:n], od[:n], rtol, atol)):
        return False
    og = dict(zip(oi[:n].tolist(), od[:n].tolist()))
    gg = dict(zip(gi[:n].tolist(), gd[:n].tolist()))
    for t in range(n):
        if gi[t] == oi[t]:
            continue
        a = int(gi[t])
        if a in og:
            # a moved inside a tie group: its oracle distance ties the distance at position t
            if not close(og[a], od[t], rtol, atol):
                return False
        else:
            # a entered at the boundary: it ties the oracle's last kept distance
            if not close(gg[a], od[n - 1], rtol, atol):
                return False
    for b in set(oi[:n].tolist()) - set(gi[:n].tolist()):
        if not close(og[b], gd[n - 1], rtol, atol):
            return False
    return True


def lists_match(g_ids, g_dist, o_ids, o_dist, rtol=RTOL, atol=ATOL):
    """Indices of rows that violate the rule (empty array = parity)."""
    bad = []
    diff = np.nonzero(~(np.all(g_ids == o_ids, 1) & np.all(close(g_dist, o_dist, rtol, atol), 1)))[0]
    for u in diff:
        if not row_matches(g_ids[u], g_dist[u], o_ids[u], o_dist[u], rtol, atol):
            bad.append(int(u))
    return np.asarray(bad, dtype=np.int64)


def check_lists(ids, dist, N, allow_self=False):
    """Rows sorted by (dist, id), valid prefix, no duplicates, no self loops, ids in range."""
    valid = ids >= 0
    n = valid.sum(1)
    assert np.all(ids.max(1) < N)
    pref = np.arange(ids.shape[1])[None, :] < n[:, None]
    assert np.array_equal(valid, pref), "valid entries must form a prefix"
    if not allow_self:
        assert not np.any(ids == np.arange(ids.shape[0])[:, None]), "self loop"
    s = np.sort(np.where(valid, ids, -1 - np.arange(ids.shape[1])[None, :]), 1)
    assert not np.any((s[:, 1:] == s[:, :-1]) & (s[:, 1:] >= 0)), "duplicate id in a row"
    d = np.where(valid, dist, np.inf)
    with np.errstate(invalid="ignore"):  # inf - inf past the valid prefix; masked below
        dd = np.diff(d, axis=1)
    ii = np.diff(ids, axis=1)
    both = valid[:, 1:]
    ok = (dd > 0) | ((dd == 0) & (ii > 0)) | ~both
    assert np.all(ok), "row not sorted by (dist, id)"


def bfs_reached(ids, entry):
    from collections import deque
    N = ids.shape[0]
    seen = np.zeros(N, bool)
    seen[entry] = True
    q = deque([entry])
    while q:
        x = q.popleft()
        for y in ids[x]:
            if y >= 0 and not seen[y]:
                seen[y] = True
                q.append(int(y))
    return seen


def _delta64(a, b, metric):
    if metric == 0:
        return float(np.sum((a - b) ** 2))
    if metric == 1:
        return 1.0 - float(np.dot(a, b))
    return 1.0 - float(np.dot(a, b)) / (float(np.linalg.norm(a)) * float(np.linalg.norm(b)))


def prune_row_has_near_tie(X, u, cand, dist_u, alpha, rtol=RTOL, atol=ATOL, metric=0, rule="arng", tau=0.0):
    """True when some occlusion test of row u is within tolerance of equality (FP64 check): the
    compared quantities are alpha^2 delta(w,v) against delta(u,v) (alpha-RNG), delta(w,v) against
    delta(u,v) (MRNG) or delta(w,v) against (sqrt(delta(u,v)) - 3 tau)^2 (tau-MNG)."""
    a2 = float(np.float32(np.float64(alpha) ** 2))
    Xc = X[cand].astype(np.float64)
    for j in range(len(cand)):
        duv = float(dist_u[j])
        if rule == "tmng":
            t = np.sqrt(max(duv, 0.0)) - 3.0 * tau
            if t <= 0:
                continue
            thr = t * t
        for i in range(j):
            dwv = _delta64(Xc[i], Xc[j], metric)
            if rule == "arng":
                a, b = duv, a2 * dwv
            elif rule == "mrng":
                a, b = duv, dwv
            else:
                a, b = thr, dwv
            if abs(a - b) <= rtol * max(abs(a), abs(b)) + atol:
                return True
    return False
