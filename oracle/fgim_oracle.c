/*
 * FGIM merge oracle (see fgim_oracle.h). TEST INFRASTRUCTURE ONLY.
 *
 * Plain CPU restatement of the paper's steps, in the paper's order:
 *   Alg. 1  KNNSearch (beam search)                   -> or_knn_search
 *   Alg. 2  PGs -> k-NNG (cross querying, Sec. 4.1)   -> or_stage_a
 *   Alg. 3  k-NNG refinement, Visit + Update (4.2.1)  -> or_refine_iter (synchronous form)
 *   Alg. 4  indegree repair (Sec. 4.2.2)              -> or_indegree_repair
 *   Alg. 5  k-NNG -> PG: neighbour selection and
 *           connectivity enhancement (Sec. 4.3)       -> or_prune_rule (alpha-RNG, MRNG, tau-MNG),
 *                                                        or_reverse_insert
 *   added   reachability fix                          -> or_reach_fix
 *
 * Readings of the paper where it is silent (each one also listed in the design notes):
 *  - Alg. 1 keeps two marks: "seen" (distance evaluated; a vertex is evaluated at most once)
 *    and "expanded" (popped). One vertex is expanded per step: the first unexpanded pool entry.
 *  - Every ordering is by (distance, global id) ascending.
 *  - Alg. 3 runs synchronously: Visit builds C_n / C_o of every vertex from the snapshot at the
 *    start of the pass, then Update evaluates every pair; each list ends as the top-k of
 *    (its snapshot entries U all proposals), duplicates by id removed. Reverse lists are capped
 *    at rev_cap, keeping the smallest (distance, source id).
 *  - Alg. 4 takes the zero-indegree vertices in ascending id; `replaced` marks are cleared when
 *    a repair call starts; the new entry gets the marks {new, replaced}.
 *  - Alg. 5 keeps v when T(v) = 1 or delta(u,v) < alpha^2 * delta(w,v) for every kept w
 *    (alpha-RNG on squared-type distances), stops at R, and adds reverse edges taken from the
 *    pruned snapshot only.
 *  - phi with invalid vertices (Sec. 4.1.3): valid vertices are numbered consecutively in
 *    (shard, local id) order. Alg. 2 runs for valid u only; Alg. 1 searches the input PG
 *    unchanged (invalid vertices route and may fill the pool), and phi then drops invalid
 *    vertices from C_i^+(u) and from the search results before the top-k. The merged entry
 *    is the entry of the shard with the most valid vertices if valid, else that shard's
 *    first valid vertex.
 */
#include "fgim_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Distance delta (Sec. 2.1): squared L2, 1 - inner product, or 1 - cosine.    */
/* ------------------------------------------------------------------------- */
double or_delta64(const float* x, const float* y, int32_t d, int32_t metric) {
    if (metric == OR_METRIC_L2) {
        double s = 0.0;
        for (int32_t t = 0; t < d; ++t) {
            double z = (double)x[t] - (double)y[t];
            s += z * z;
        }
        return s;
    }
    double xy = 0.0, xx = 0.0, yy = 0.0;
    for (int32_t t = 0; t < d; ++t) {
        xy += (double)x[t] * (double)y[t];
        xx += (double)x[t] * (double)x[t];
        yy += (double)y[t] * (double)y[t];
    }
    if (metric == OR_METRIC_IP) return 1.0 - xy;
    return 1.0 - xy / (sqrt(xx) * sqrt(yy));
}

float or_delta(const float* x, const float* y, int32_t d, int32_t metric) {
    return (float)or_delta64(x, y, d, metric);
}

static inline const float* row(const or_input* in, int64_t g) { return in->X + g * (int64_t)in->d; }

static inline float dist_g(const or_input* in, int64_t a, int64_t b) {
    return or_delta(row(in, a), row(in, b), in->d, in->metric);
}

/* (distance, id) lexicographic order */
static inline int key_lt(float da, int32_t ia, float db, int32_t ib) {
    return da < db || (da == db && ia < ib);
}

typedef struct { float d; int32_t id; } ent_t;

static int ent_cmp(const void* pa, const void* pb) {
    const ent_t* a = (const ent_t*)pa;
    const ent_t* b = (const ent_t*)pb;
    if (key_lt(a->d, a->id, b->d, b->id)) return -1;
    if (key_lt(b->d, b->id, a->d, a->id)) return 1;
    return 0;
}

static int shard_of(const or_input* in, int64_t g) {
    int s = 0;
    while (s + 1 < in->h && g >= in->off[s + 1]) ++s;
    return s;
}

// n > 0: that many threads; n <= 0: the OpenMP default seen at the first call (an earlier
// call's count does not stick)
static void set_threads(int32_t n) {
#ifdef _OPENMP
    static int dflt = 0;
    if (dflt == 0) dflt = omp_get_max_threads();
    omp_set_num_threads(n > 0 ? n : dflt);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* Alg. 1 KNNSearch(q, G, L, k, ep)                                           */
/* ------------------------------------------------------------------------- */
static int32_t knn_search_tagged(const float* X, int32_t d, int32_t metric, const int32_t* adj, int32_t M,
                                 int32_t ep, const float* q, int32_t L, int32_t k, uint32_t* seen,
                                 uint32_t tag, int32_t* out_ids, float* out_dist, or_stats* st) {
    /* candidate pool C, sorted by (delta, id), at most L entries */
    float* cd = (float*)malloc(sizeof(float) * (L + 1));
    int32_t* ci = (int32_t*)malloc(sizeof(int32_t) * (L + 1));
    uint8_t* cx = (uint8_t*)malloc(L + 1);
    int32_t n = 0;
    int64_t ndc = 0, hops = 0;

    /* start: C <- {(ep, delta(ep, q))} */
    seen[ep] = tag;
    cd[0] = or_delta(q, X + (int64_t)ep * d, d, metric);
    ci[0] = ep;
    cx[0] = 0;
    n = 1;
    ndc++;
    for (;;) {
        /* i <- index of the first unexpanded vertex in C */
        int32_t i = 0;
        while (i < n && cx[i]) ++i;
        if (i >= n) break;                 /* no unexpanded vertex left */
        /* u <- C[i], mark u as visited (expanded) */
        cx[i] = 1;
        int32_t u = ci[i];
        hops++;
        /* insert every not-yet-seen neighbour v of u */
        for (int32_t t = 0; t < M; ++t) {
            int32_t v = adj[(int64_t)u * M + t];
            if (v < 0) continue;
            if (seen[v] == tag) continue;
            seen[v] = tag;
            float dv = or_delta(q, X + (int64_t)v * d, d, metric);
            ndc++;
            /* keep the top-L of C by (delta, id) */
            if (n == L && !key_lt(dv, v, cd[n - 1], ci[n - 1])) continue;
            int32_t pos = n < L ? n : L - 1;
            while (pos > 0 && key_lt(dv, v, cd[pos - 1], ci[pos - 1])) {
                cd[pos] = cd[pos - 1];
                ci[pos] = ci[pos - 1];
                cx[pos] = cx[pos - 1];
                --pos;
            }
            cd[pos] = dv;
            ci[pos] = v;
            cx[pos] = 0;
            if (n < L) ++n;
        }
    }
    /* result: the first k entries */
    int32_t r = n < k ? n : k;
    for (int32_t t = 0; t < r; ++t) {
        out_ids[t] = ci[t];
        out_dist[t] = cd[t];
    }
    free(cd);
    free(ci);
    free(cx);
    if (st) {
        st->ndc += ndc;
        st->hops += hops;
    }
    return r;
}

/* ------------------------------------------------------------------------- */
/* HNSW's upper layers by sequential insertion (Sec. 4.3.3, as HNSW builds)    */
/* ------------------------------------------------------------------------- */
/* The heuristic neighbour selection of HNSW (Alg. 5's rule with alpha = 1 and no indegree
 * clause): candidates (ids, dist to u) ascending; keep e unless a kept r has delta(e, r) <= delta(u, e);
 * at most M. Returns the number kept, written to keep_ids / keep_dist. */
static int32_t hnsw_heuristic(const float* X, int32_t d, int32_t metric, const int32_t* ids, const float* dist,
                              int32_t n, int32_t M, int32_t* keep_ids, float* keep_dist) {
    int32_t nk = 0;
    for (int32_t t = 0; t < n && nk < M; ++t) {
        int ok = 1;
        for (int32_t s = 0; s < nk && ok; ++s) {
            float der = or_delta(X + (int64_t)ids[t] * d, X + (int64_t)keep_ids[s] * d, d, metric);
            if (!(dist[t] < der)) ok = 0;
        }
        if (ok) {
            keep_ids[nk] = ids[t];
            keep_dist[nk] = dist[t];
            ++nk;
        }
    }
    return nk;
}

void or_hnsw_insert(const float* X, int64_t N, int32_t d, int32_t metric, const int32_t* levels, int32_t max_level,
                    int32_t M, int32_t ef, int32_t* adj, int32_t* entry_out, or_stats* st) {
    /* adj: [max_level, N, M] global ids, -1 padded; layer l (1 .. max_level) at adj + (l-1) N M. Every
     * vertex with level >= 1 is inserted in ascending id: greedy descent (Alg. 1 with a pool of
     * one) from the entry through the layers above its level, then on each of its layers Alg. 1
     * with pool ef from the vertex reached (HNSW hands all of W down as entry points; Alg. 1
     * starts from one vertex, so the nearest of W starts the next layer), HNSW's heuristic to M,
     * edges both ways, and the heuristic again over a neighbour's list that overflows M. The
     * entry is the first vertex that reached the highest level. Layer 0 (the merged base graph)
     * is not touched. */
    for (int64_t t = 0; t < (int64_t)max_level * N * M; ++t) adj[t] = -1;
    uint32_t* seen = (uint32_t*)calloc(N, sizeof(uint32_t));
    uint32_t tag = 0;
    int32_t* w_ids = (int32_t*)malloc(sizeof(int32_t) * (ef + 1));
    float* w_dist = (float*)malloc(sizeof(float) * (ef + 1));
    int32_t* k_ids = (int32_t*)malloc(sizeof(int32_t) * (M + 1));
    float* k_dist = (float*)malloc(sizeof(float) * (M + 1));
    ent_t* ov = (ent_t*)malloc(sizeof(ent_t) * (M + 1));
    int32_t* ov_ids = (int32_t*)malloc(sizeof(int32_t) * (M + 1));
    float* ov_dist = (float*)malloc(sizeof(float) * (M + 1));
    int32_t* rp_ids = (int32_t*)malloc(sizeof(int32_t) * M);
    float* rp_dist = (float*)malloc(sizeof(float) * M);
    int32_t entry = -1, top = 0;
    for (int64_t q = 0; q < N; ++q) {
        const int32_t lq = levels[q] < max_level ? levels[q] : max_level;
        if (lq < 1) continue;
        if (entry < 0) {
            entry = (int32_t)q;
            top = lq;
            continue;
        }
        const float* xq = X + q * d;
        int32_t ep = entry;
        /* greedy descent through the layers above lq */
        for (int32_t l = top; l > lq; --l) {
            int32_t* A = adj + (int64_t)(l - 1) * N * M;
            int32_t r = knn_search_tagged(X, d, metric, A, M, ep, xq, 1, 1, seen, ++tag, w_ids, w_dist, st);
            if (r > 0) ep = w_ids[0];
        }
        for (int32_t l = (lq < top ? lq : top); l >= 1; --l) {
            int32_t* A = adj + (int64_t)(l - 1) * N * M;
            int32_t r = knn_search_tagged(X, d, metric, A, M, ep, xq, ef, ef, seen, ++tag, w_ids, w_dist, st);
            int32_t nk = hnsw_heuristic(X, d, metric, w_ids, w_dist, r, M, k_ids, k_dist);
            for (int32_t s = 0; s < nk; ++s) A[q * M + s] = k_ids[s];
            /* reverse edges, re-pruning a list that overflows M (the new edge with its old ones) */
            for (int32_t s = 0; s < nk; ++s) {
                const int32_t e = k_ids[s];
                int32_t* row = A + (int64_t)e * M;
                int32_t n = 0;
                while (n < M && row[n] >= 0) ++n;
                if (n < M) {
                    row[n] = (int32_t)q;
                    continue;
                }
                for (int32_t t = 0; t < M; ++t) {
                    ov[t].id = row[t];
                    ov[t].d = or_delta(X + (int64_t)e * d, X + (int64_t)row[t] * d, d, metric);
                }
                ov[M].id = (int32_t)q;
                ov[M].d = k_dist[s];
                qsort(ov, M + 1, sizeof(ent_t), ent_cmp);
                for (int32_t t = 0; t <= M; ++t) {
                    ov_ids[t] = ov[t].id;
                    ov_dist[t] = ov[t].d;
                }
                int32_t kept = hnsw_heuristic(X, d, metric, ov_ids, ov_dist, M + 1, M, rp_ids, rp_dist);
                for (int32_t t = 0; t < M; ++t) row[t] = t < kept ? rp_ids[t] : -1;
            }
            ep = w_ids[0];
        }
        if (lq > top) {
            entry = (int32_t)q;
            top = lq;
        }
    }
    *entry_out = entry;
    free(seen); free(w_ids); free(w_dist); free(k_ids); free(k_dist); free(ov); free(ov_ids); free(ov_dist);
    free(rp_ids); free(rp_dist);
}

int32_t or_knn_search(const float* X_local, int64_t n, int32_t d, int32_t metric, const int32_t* adj_local,
                      int32_t M, int32_t ep, const float* q, int32_t L, int32_t k,
                      int32_t* out_ids, float* out_dist, or_stats* st) {
    uint32_t* seen = (uint32_t*)calloc(n, sizeof(uint32_t));
    int32_t r = knn_search_tagged(X_local, d, metric, adj_local, M, ep, q, L, k, seen, 1u, out_ids, out_dist, st);
    free(seen);
    return r;
}

/* ------------------------------------------------------------------------- */
/* Exact k-NN (Definition k-NNS), exhaustive                                  */
/* ------------------------------------------------------------------------- */
/* For every row i of X: its k nearest rows among rows 0 .. i - 1 (the vertices inserted before it
 * when rows are inserted in order), ascending (delta, id), -1 / +inf padded. */
void or_knn_prefix(const float* X, int64_t N, int32_t d, int32_t metric, int32_t k, int32_t nthreads,
                   int32_t* out_ids, float* out_dist) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t qi = 0; qi < N; ++qi) {
        const float* q = X + qi * (int64_t)d;
        float* bd = out_dist + qi * (int64_t)k;
        int32_t* bi = out_ids + qi * (int64_t)k;
        int32_t n = 0;
        for (int64_t g = 0; g < qi; ++g) {
            float dg = or_delta(q, X + g * (int64_t)d, d, metric);
            if (n == k && !key_lt(dg, (int32_t)g, bd[k - 1], bi[k - 1])) continue;
            int32_t pos = n < k ? n : k - 1;
            while (pos > 0 && key_lt(dg, (int32_t)g, bd[pos - 1], bi[pos - 1])) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = dg;
            bi[pos] = (int32_t)g;
            if (n < k) ++n;
        }
        for (int32_t t = n; t < k; ++t) {
            bi[t] = -1;
            bd[t] = INFINITY;
        }
    }
}

void or_knn_exact(const float* X, int64_t N, int32_t d, int32_t metric, const float* Q, int64_t nq,
                  const int64_t* exclude, int32_t k, int32_t nthreads, int32_t* out_ids, float* out_dist) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t qi = 0; qi < nq; ++qi) {
        const float* q = Q + qi * (int64_t)d;
        int64_t ex = exclude ? exclude[qi] : -1;
        float* bd = out_dist + qi * (int64_t)k;
        int32_t* bi = out_ids + qi * (int64_t)k;
        int32_t n = 0;
        for (int64_t g = 0; g < N; ++g) {
            if (g == ex) continue;
            float dg = or_delta(q, X + g * (int64_t)d, d, metric);
            if (n == k && !key_lt(dg, (int32_t)g, bd[k - 1], bi[k - 1])) continue;
            int32_t pos = n < k ? n : k - 1;
            while (pos > 0 && key_lt(dg, (int32_t)g, bd[pos - 1], bi[pos - 1])) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = dg;
            bi[pos] = (int32_t)g;
            if (n < k) ++n;
        }
        for (int32_t t = n; t < k; ++t) {
            bi[t] = -1;
            bd[t] = INFINITY;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Alg. 2 PGs -> k-NNG                                                        */
/* ------------------------------------------------------------------------- */
static int32_t minimum_L(int32_t k, int32_t h) {
    /* Sec. 4.1.2, worst case: L >= ceil(k / (|G| - 1)) */
    return (k + (h - 1) - 1) / (h - 1);
}

int64_t or_phi(const or_input* in, int32_t* phi) {
    int64_t n = 0;
    for (int64_t g = 0; g < in->off[in->h]; ++g) phi[g] = (!in->valid || in->valid[g]) ? (int32_t)n++ : -1;
    return n;
}

int32_t or_stage_a(const or_input* in, int32_t k, int32_t L, int32_t* ids, float* dist, uint8_t* flags,
                   or_stats* st) {
    const int32_t h = in->h;
    if (L <= 0) L = minimum_L(k, h);
    /* phi: identity when every vertex is valid */
    int32_t* phi = (int32_t*)malloc(sizeof(int32_t) * (in->off[h] > 0 ? in->off[h] : 1));
    or_phi(in, phi);
    int64_t max_n = 0;
    for (int s = 0; s < h; ++s)
        if (in->off[s + 1] - in->off[s] > max_n) max_n = in->off[s + 1] - in->off[s];
    set_threads(in->nthreads);
    int64_t ndc = 0, hops = 0;
#pragma omp parallel reduction(+ : ndc, hops)
    {
        uint32_t* seen = (uint32_t*)calloc(max_n, sizeof(uint32_t));
        uint32_t tag = 0;
        int32_t cap = in->M + (h - 1) * L;
        ent_t* C = (ent_t*)malloc(sizeof(ent_t) * cap);
        int32_t* rid = (int32_t*)malloc(sizeof(int32_t) * L);
        float* rd = (float*)malloc(sizeof(float) * L);
        or_stats ls;
        memset(&ls, 0, sizeof(ls));
#pragma omp for schedule(dynamic, 16)
        for (int64_t g = 0; g < in->off[h]; ++g) {
            if (phi[g] < 0) continue;   /* no row for an invalid vertex */
            const int64_t o = phi[g];   /* its row of the k-NNG */
            int i = shard_of(in, g);
            int64_t u = g - in->off[i];
            int32_t n = 0;
            /* local candidate neighbours C_i^+(u) from G_i, mapped by phi */
            for (int32_t t = 0; t < in->M; ++t) {
                int32_t v = in->adj[g * in->M + t];
                if (v < 0 || v == u) continue;
                int64_t gv = in->off[i] + v;
                if (phi[gv] < 0) continue;
                C[n].id = phi[gv];
                C[n].d = dist_g(in, g, gv);
                ls.ndc++;
                ++n;
            }
            /* cross querying, KNNSearch(x_u, G_j, L, L, ep_j) for every j != i */
            for (int j = 0; j < h; ++j) {
                if (j == i) continue;
                int64_t nj = in->off[j + 1] - in->off[j];
                if (nj <= 0) continue;
                ++tag;
                if (tag == 0) {
                    memset(seen, 0, sizeof(uint32_t) * max_n);
                    tag = 1;
                }
                int32_t r = knn_search_tagged(row(in, in->off[j]), in->d, in->metric,
                                              in->adj + in->off[j] * in->M, in->M, in->entry[j],
                                              row(in, g), L, L, seen, tag, rid, rd, &ls);
                for (int32_t t = 0; t < r; ++t) {
                    const int32_t mapped = phi[in->off[j] + rid[t]];
                    if (mapped < 0) continue;
                    C[n].id = mapped;
                    C[n].d = rd[t];
                    ++n;
                }
            }
            /* sort by distance, map ids (done above), resize(C, k) */
            qsort(C, n, sizeof(ent_t), ent_cmp);
            int32_t w = 0;
            for (int32_t t = 0; t < n && w < k; ++t) {
                int dup = 0;
                for (int32_t s = 0; s < w; ++s)
                    if (ids[o * k + s] == C[t].id) { dup = 1; break; }
                if (dup) continue;
                ids[o * k + w] = C[t].id;
                dist[o * k + w] = C[t].d;
                flags[o * k + w] = OR_FLAG_NEW;
                ++w;
            }
            for (; w < k; ++w) {
                ids[o * k + w] = -1;
                dist[o * k + w] = INFINITY;
                flags[o * k + w] = 0;
            }
        }
        ndc += ls.ndc;
        hops += ls.hops;
        free(seen);
        free(C);
        free(rid);
        free(rd);
    }
    if (st) {
        st->ndc += ndc;
        st->hops += hops;
    }
    free(phi);
    return L;
}

/* ------------------------------------------------------------------------- */
/* Bounded sorted list insertion used by Update: accept iff the id is absent   */
/* and the list has room or (delta, id) beats the current worst entry.         */
/* ------------------------------------------------------------------------- */
static int list_insert(int32_t* ids, float* dist, uint8_t* flags, int32_t k, int32_t id, float d) {
    int32_t n = 0;
    while (n < k && ids[n] >= 0) ++n;
    for (int32_t t = 0; t < n; ++t)
        if (ids[t] == id) return 0;
    if (n == k && !key_lt(d, id, dist[k - 1], ids[k - 1])) return 0;
    int32_t pos = n < k ? n : k - 1;
    while (pos > 0 && key_lt(d, id, dist[pos - 1], ids[pos - 1])) {
        ids[pos] = ids[pos - 1];
        dist[pos] = dist[pos - 1];
        flags[pos] = flags[pos - 1];
        --pos;
    }
    ids[pos] = id;
    dist[pos] = d;
    flags[pos] = OR_FLAG_NEW;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Alg. 3, one pass of Visit + Update (synchronous reading)                    */
/* ------------------------------------------------------------------------- */
typedef struct { float d; int32_t src; } rev_t;

static int rev_cmp(const void* pa, const void* pb) {
    const rev_t* a = (const rev_t*)pa;
    const rev_t* b = (const rev_t*)pb;
    if (key_lt(a->d, a->src, b->d, b->src)) return -1;
    if (key_lt(b->d, b->src, a->d, a->src)) return 1;
    return 0;
}

#define OR_NLOCKS 4096

void or_refine_iter(const or_input* in, int32_t k, int32_t rev_cap, int32_t* ids, float* dist,
                    uint8_t* flags, or_stats* st) {
    const int64_t N = in->off[in->h];
    if (rev_cap <= 0) rev_cap = k;
    set_threads(in->nthreads);

    /* --- Visit: reverse graphs G_n-bar and G_o-bar from the snapshot --- */
    int64_t* cnt_n = (int64_t*)calloc(N + 1, sizeof(int64_t));
    int64_t* cnt_o = (int64_t*)calloc(N + 1, sizeof(int64_t));
    for (int64_t u = 0; u < N; ++u)
        for (int32_t t = 0; t < k; ++t) {
            int32_t v = ids[u * k + t];
            if (v < 0) continue;
            if (flags[u * k + t] & OR_FLAG_NEW) cnt_n[v + 1]++;
            else cnt_o[v + 1]++;
        }
    for (int64_t v = 0; v < N; ++v) {
        cnt_n[v + 1] += cnt_n[v];
        cnt_o[v + 1] += cnt_o[v];
    }
    rev_t* rn = (rev_t*)malloc(sizeof(rev_t) * (cnt_n[N] + 1));
    rev_t* ro = (rev_t*)malloc(sizeof(rev_t) * (cnt_o[N] + 1));
    int64_t* fill_n = (int64_t*)calloc(N, sizeof(int64_t));
    int64_t* fill_o = (int64_t*)calloc(N, sizeof(int64_t));
    for (int64_t u = 0; u < N; ++u)
        for (int32_t t = 0; t < k; ++t) {
            int32_t v = ids[u * k + t];
            if (v < 0) continue;
            rev_t r = {dist[u * k + t], (int32_t)u};
            if (flags[u * k + t] & OR_FLAG_NEW) rn[cnt_n[v] + fill_n[v]++] = r;
            else ro[cnt_o[v] + fill_o[v]++] = r;
        }
    /* cap each reverse list at rev_cap, keeping the smallest (delta, source) */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t v = 0; v < N; ++v) {
        qsort(rn + cnt_n[v], cnt_n[v + 1] - cnt_n[v], sizeof(rev_t), rev_cmp);
        qsort(ro + cnt_o[v], cnt_o[v + 1] - cnt_o[v], sizeof(rev_t), rev_cmp);
    }
    /* C_n(v) = new forward U capped new reverse; C_o(v) = (old forward U capped old reverse) \ C_n(v) */
    const int32_t cmax = k + rev_cap;
    int32_t* Cn = (int32_t*)malloc(sizeof(int32_t) * N * cmax);
    int32_t* Co = (int32_t*)malloc(sizeof(int32_t) * N * cmax);
    int32_t* nn = (int32_t*)calloc(N, sizeof(int32_t));
    int32_t* no = (int32_t*)calloc(N, sizeof(int32_t));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t v = 0; v < N; ++v) {
        int32_t* cn = Cn + v * cmax;
        int32_t* co = Co + v * cmax;
        int32_t a = 0, b = 0;
        for (int32_t t = 0; t < k; ++t) {
            int32_t w = ids[v * k + t];
            if (w >= 0 && (flags[v * k + t] & OR_FLAG_NEW)) cn[a++] = w;
        }
        int64_t m = cnt_n[v + 1] - cnt_n[v];
        if (m > rev_cap) m = rev_cap;
        for (int64_t t = 0; t < m; ++t) {
            int32_t w = rn[cnt_n[v] + t].src;
            int dup = 0;
            for (int32_t s = 0; s < a; ++s) if (cn[s] == w) { dup = 1; break; }
            if (!dup) cn[a++] = w;
        }
        for (int32_t t = 0; t < k; ++t) {
            int32_t w = ids[v * k + t];
            if (w >= 0 && !(flags[v * k + t] & OR_FLAG_NEW)) co[b++] = w;
        }
        m = cnt_o[v + 1] - cnt_o[v];
        if (m > rev_cap) m = rev_cap;
        for (int64_t t = 0; t < m; ++t) {
            int32_t w = ro[cnt_o[v] + t].src;
            int dup = 0;
            for (int32_t s = 0; s < b; ++s) if (co[s] == w) { dup = 1; break; }
            if (!dup) co[b++] = w;
        }
        /* remove from C_o everything that is already in C_n */
        int32_t b2 = 0;
        for (int32_t t = 0; t < b; ++t) {
            int dup = 0;
            for (int32_t s = 0; s < a; ++s) if (cn[s] == co[t]) { dup = 1; break; }
            if (!dup) co[b2++] = co[t];
        }
        nn[v] = a;
        no[v] = b2;
    }
    /* new neighbours are old once visited */
    for (int64_t t = 0; t < N * k; ++t) flags[t] &= (uint8_t)~OR_FLAG_NEW;

    /* --- Update: every cross-graph pair of C_n^2 U (C_n x C_o) --- */
#ifdef _OPENMP
    omp_lock_t* locks = (omp_lock_t*)malloc(sizeof(omp_lock_t) * OR_NLOCKS);
    for (int t = 0; t < OR_NLOCKS; ++t) omp_init_lock(&locks[t]);
#endif
    int64_t pairs = 0, updates = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : pairs, updates)
    for (int64_t v = 0; v < N; ++v) {
        const int32_t* cn = Cn + v * cmax;
        const int32_t* co = Co + v * cmax;
        for (int32_t x = 0; x < nn[v]; ++x) {
            int32_t a = cn[x];
            int sa = shard_of(in, a);
            /* (a, b) with b later in C_n: each unordered pair once; then (a, b) in C_n x C_o */
            for (int32_t y = x + 1; y < nn[v] + no[v]; ++y) {
                int32_t b = y < nn[v] ? cn[y] : co[y - nn[v]];
                if (a == b || shard_of(in, b) == sa) continue;
                float dab = dist_g(in, a, b);
                ++pairs;
#ifdef _OPENMP
                omp_set_lock(&locks[a % OR_NLOCKS]);
#endif
                updates += list_insert(ids + (int64_t)a * k, dist + (int64_t)a * k, flags + (int64_t)a * k, k, b, dab);
#ifdef _OPENMP
                omp_unset_lock(&locks[a % OR_NLOCKS]);
                omp_set_lock(&locks[b % OR_NLOCKS]);
#endif
                updates += list_insert(ids + (int64_t)b * k, dist + (int64_t)b * k, flags + (int64_t)b * k, k, a, dab);
#ifdef _OPENMP
                omp_unset_lock(&locks[b % OR_NLOCKS]);
#endif
            }
        }
    }
#ifdef _OPENMP
    for (int t = 0; t < OR_NLOCKS; ++t) omp_destroy_lock(&locks[t]);
    free(locks);
#endif
    if (st) {
        st->pairs += pairs;
        st->ndc += pairs;
        st->updates += updates;
    }
    free(cnt_n); free(cnt_o); free(rn); free(ro); free(fill_n); free(fill_o);
    free(Cn); free(Co); free(nn); free(no);
}

/* ------------------------------------------------------------------------- */
/* Alg. 4 Indegree repair                                                      */
/* ------------------------------------------------------------------------- */
void or_indegree(const int32_t* ids, int64_t N, int32_t k, int32_t* T) {
    memset(T, 0, sizeof(int32_t) * N);
    for (int64_t t = 0; t < N * k; ++t)
        if (ids[t] >= 0) T[ids[t]]++;
}

/* move entry `pos` of a list to its sorted place by (delta, id) */
static void resort_entry(int32_t* ids, float* dist, uint8_t* flags, int32_t k, int32_t pos) {
    int32_t id = ids[pos];
    float d = dist[pos];
    uint8_t f = flags[pos];
    while (pos > 0 && ids[pos - 1] >= 0 && key_lt(d, id, dist[pos - 1], ids[pos - 1])) {
        ids[pos] = ids[pos - 1]; dist[pos] = dist[pos - 1]; flags[pos] = flags[pos - 1]; --pos;
    }
    while (pos + 1 < k && ids[pos + 1] >= 0 && key_lt(dist[pos + 1], ids[pos + 1], d, id)) {
        ids[pos] = ids[pos + 1]; dist[pos] = dist[pos + 1]; flags[pos] = flags[pos + 1]; ++pos;
    }
    ids[pos] = id; dist[pos] = d; flags[pos] = f;
}

void or_indegree_repair(const or_input* in, int32_t k, int32_t* ids, float* dist, uint8_t* flags,
                        int32_t* T, or_stats* st) {
    const int64_t N = in->off[in->h];
    /* T <- indegree of every vertex */
    or_indegree(ids, N, k, T);
    for (int64_t t = 0; t < N * k; ++t) flags[t] &= (uint8_t)~OR_FLAG_REPLACED;
    int64_t zero_before = 0, replaced = 0;
    /* every v* with T(v*) = 0, ascending id */
    for (int64_t vs = 0; vs < N; ++vs) {
        if (T[vs] != 0) continue;
        ++zero_before;
        int done = 0;
        /* neighbours v of v*, closest first, until T(v*) > 0 */
        for (int32_t a = 0; a < k && !done; ++a) {
            int32_t v = ids[vs * k + a];
            if (v < 0) break;
            int32_t* lv = ids + (int64_t)v * k;
            float* dv = dist + (int64_t)v * k;
            uint8_t* fv = flags + (int64_t)v * k;
            /* v' in N(v) in descending order of distance to x_v */
            for (int32_t b = k - 1; b >= 0; --b) {
                int32_t vp = lv[b];
                if (vp < 0) continue;
                /* not replaced and T(v') > 1. (Within one call a replaced entry holds a
                 * vertex whose indegree just became 1, so the T test alone would skip it too;
                 * the mark is kept because the paper states it.) */
                if ((fv[b] & OR_FLAG_REPLACED) || T[vp] <= 1) continue;
                /* replace v' by v*, mark it, update T */
                lv[b] = (int32_t)vs;
                dv[b] = dist_g(in, v, vs);
                fv[b] = OR_FLAG_NEW | OR_FLAG_REPLACED;
                resort_entry(lv, dv, fv, k, b);
                T[vp] -= 1;
                T[vs] += 1;
                ++replaced;
                done = 1;
                break;
            }
        }
    }
    if (st) {
        int64_t zero_after = 0;
        for (int64_t v = 0; v < N; ++v) zero_after += T[v] == 0;
        st->zero_before += zero_before;
        st->zero_after += zero_after;
        st->replaced += replaced;
    }
}

/* ------------------------------------------------------------------------- */
/* Alg. 5 k-NNG -> PG                                                          */
/* ------------------------------------------------------------------------- */
/* Occlusion test of the neighbour-selection rule (Sec. 4.3.1 names RNG, MRNG and tau-MNG as
 * interchangeable rules; the paper defines none of the last two, so each is restated from the
 * work it cites). u is the vertex, w an already kept neighbour, v the candidate:
 * duv = delta(u, v), duw = delta(u, w), dwv = delta(w, v), all squared-type distances.
 *  OR_PRUNE_ARNG  alpha-RNG (Alg. 5 with Vamana's alpha): w occludes v iff alpha^2 dwv <= duv.
 *  OR_PRUNE_MRNG  MRNG (NSG's edge selection, Fu et al.): w occludes v iff dwv < duv, i.e. uv is
 *                 strictly the longest edge of the triangle uwv (w precedes v, so duw <= duv).
 *  OR_PRUNE_TMNG  tau-MNG (Peng et al.): on the metric distances sqrt(delta), w occludes v iff
 *                 sqrt(duw) < sqrt(duv) and sqrt(dwv) < sqrt(duv) - 3 tau: edges shorter than
 *                 3 tau are never pruned. Decided in FP32, like every ordering decision here:
 *                 t = sqrtf(duv) - RN(3 tau); occluded iff t > 0, duw < duv and dwv < t * t. */
static int occludes(int32_t rule, float alpha2, float tau3, float duv, float duw, float dwv) {
    if (rule == OR_PRUNE_MRNG) return dwv < duv;
    if (rule == OR_PRUNE_TMNG) {
        float t = sqrtf(duv) - tau3;
        if (!(t > 0.f)) return 0;
        float t2 = t * t;
        return duw < duv && dwv < t2;
    }
    float bound = alpha2 * dwv;
    return !(duv < bound);
}

void or_prune_rule(const or_input* in, int32_t k, const int32_t* ids, const float* dist, const int32_t* T,
                   int32_t R, int32_t rule, float alpha, float tau, int32_t* e_ids, float* e_dist, int32_t* e_cnt,
                   or_stats* st) {
    const int64_t N = in->off[in->h];
    /* alpha^2 and 3 tau rounded once to FP32: the distances are squared-type */
    const float alpha2 = (float)((double)alpha * (double)alpha);
    const float tau3 = (float)(3.0 * (double)tau);
    set_threads(in->nthreads);
    int64_t evals = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : evals)
    for (int64_t u = 0; u < N; ++u) {
        int32_t nr = 0;
        /* v in N_G(u) in ascending order of delta(u, v) */
        for (int32_t t = 0; t < k; ++t) {
            int32_t v = ids[u * k + t];
            if (v < 0) break;
            float duv = dist[u * k + t];
            /* T(v) = 1 (Alg. 5 keeps a vertex whose only in-edge is u), else no kept w occludes v */
            int keep = T[v] == 1;
            if (!keep) {
                keep = 1;
                for (int32_t s = 0; s < nr; ++s) {
                    float dwv = dist_g(in, e_ids[u * R + s], v);
                    ++evals;
                    if (occludes(rule, alpha2, tau3, duv, e_dist[u * R + s], dwv)) { keep = 0; break; }
                }
            }
            if (keep) {
                e_ids[u * R + nr] = v;
                e_dist[u * R + nr] = duv;
                ++nr;
            }
            /* stop once |R| reaches the bound */
            if (nr == R) break;
        }
        e_cnt[u] = nr;
        for (int32_t s = nr; s < R; ++s) {
            e_ids[u * R + s] = -1;
            e_dist[u * R + s] = INFINITY;
        }
    }
    if (st) st->prune_dist += evals;
}

void or_prune(const or_input* in, int32_t k, const int32_t* ids, const float* dist, const int32_t* T,
              int32_t R, float alpha, int32_t* e_ids, float* e_dist, int32_t* e_cnt, or_stats* st) {
    or_prune_rule(in, k, ids, dist, T, R, OR_PRUNE_ARNG, alpha, 0.f, e_ids, e_dist, e_cnt, st);
}

void or_reverse_insert(int64_t N, int32_t R, const int32_t* e_ids, const float* e_dist, const int32_t* e_cnt,
                       int32_t* out_ids, float* out_dist, int32_t* out_deg) {
    /* reverse edges of the pruned snapshot E' */
    int64_t* cnt = (int64_t*)calloc(N + 1, sizeof(int64_t));
    for (int64_t u = 0; u < N; ++u)
        for (int32_t t = 0; t < e_cnt[u]; ++t) cnt[e_ids[u * R + t] + 1]++;
    for (int64_t v = 0; v < N; ++v) cnt[v + 1] += cnt[v];
    ent_t* rv = (ent_t*)malloc(sizeof(ent_t) * (cnt[N] + 1));
    int64_t* fill = (int64_t*)calloc(N, sizeof(int64_t));
    for (int64_t u = 0; u < N; ++u)
        for (int32_t t = 0; t < e_cnt[u]; ++t) {
            int32_t v = e_ids[u * R + t];
            ent_t e = {e_dist[u * R + t], (int32_t)u};
            rv[cnt[v] + fill[v]++] = e;
        }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t u = 0; u < N; ++u) {
        /* N(u) U {v : (v, u) in E'}, sorted by distance, resized to the bound */
        int64_t m = e_cnt[u] + (cnt[u + 1] - cnt[u]);
        ent_t* c = (ent_t*)malloc(sizeof(ent_t) * (m + 1));
        int64_t n = 0;
        for (int32_t t = 0; t < e_cnt[u]; ++t) {
            c[n].id = e_ids[u * R + t];
            c[n].d = e_dist[u * R + t];
            ++n;
        }
        for (int64_t t = cnt[u]; t < cnt[u + 1]; ++t) c[n++] = rv[t];
        qsort(c, n, sizeof(ent_t), ent_cmp);
        int32_t w = 0;
        for (int64_t t = 0; t < n && w < R; ++t) {
            int dup = 0;
            for (int32_t s = 0; s < w; ++s) if (out_ids[u * R + s] == c[t].id) { dup = 1; break; }
            if (dup) continue;
            out_ids[u * R + w] = c[t].id;
            out_dist[u * R + w] = c[t].d;
            ++w;
        }
        out_deg[u] = w;
        for (; w < R; ++w) {
            out_ids[u * R + w] = -1;
            out_dist[u * R + w] = INFINITY;
        }
        free(c);
    }
    free(cnt);
    free(rv);
    free(fill);
}

/* ------------------------------------------------------------------------- */
/* Reachability fix (added step; the paper only reduces SCCs, Sec. 4.2.2)      */
/* ------------------------------------------------------------------------- */
/* BFS over out-edges from src marking unmarked vertices; level[] (optional) gets 1 + hops from src */
static int64_t bfs_level(int64_t N, int32_t R, const int32_t* g, int32_t src, uint8_t* reached, int32_t* queue,
                         int32_t* level) {
    if (reached[src]) return 0;
    int64_t head = 0, tail = 0;
    reached[src] = 1;
    level[src] = 1;
    queue[tail++] = src;
    while (head < tail) {
        int32_t x = queue[head++];
        for (int32_t t = 0; t < R; ++t) {
            int32_t y = g[(int64_t)x * R + t];
            if (y < 0 || reached[y]) continue;
            reached[y] = 1;
            level[y] = level[x] + 1;
            queue[tail++] = y;
        }
    }
    (void)N;
    return tail;
}

static int64_t bfs_mark(int64_t N, int32_t R, const int32_t* g, int32_t src, uint8_t* reached, int32_t* queue) {
    if (reached[src]) return 0;
    int64_t head = 0, tail = 0, n = 0;
    reached[src] = 1;
    queue[tail++] = src;
    ++n;
    while (head < tail) {
        int32_t x = queue[head++];
        for (int32_t t = 0; t < R; ++t) {
            int32_t y = g[(int64_t)x * R + t];
            if (y < 0 || reached[y]) continue;
            reached[y] = 1;
            queue[tail++] = y;
            ++n;
        }
    }
    (void)N;
    return n;
}

static int32_t uf_find(int32_t* parent, int32_t x) {
    while (parent[x] != x) x = parent[x];
    return x;
}

/* union keeping the smaller id as the root, so each root is its component's minimum id */
static void uf_union(int32_t* parent, int32_t a, int32_t b) {
    int32_t ra = uf_find(parent, a), rb = uf_find(parent, b);
    if (ra == rb) return;
    if (ra < rb) parent[rb] = ra;
    else parent[ra] = rb;
}

#define OR_REACH_ROUNDS 16

/*
 * Rounds of: BFS from the entry (levels = 1 + hops); weak components of the subgraph
 * induced by the unreached vertices, each represented by its smallest id x; Alg. 1 for
 * x_x over the graph as it stands at the round start (pool `beam`, top `beam`); then,
 * for every representative in ascending id, one new edge p -> x:
 *   - p is the first search result (ascending (delta, id)) whose list has room
 *     (deg(p) < R): x is appended to p's list, kept sorted;
 *   - otherwise p is the first search result that has a replaceable neighbour: a
 *     reached y that keeps a BFS parent other than p (an in-neighbour at a smaller
 *     level), so y and all it reaches stay reachable; the farthest such y (by
 *     (delta, id)) is replaced by x and p's list is re-sorted.
 * Degrees and parent counts are updated after every attachment. Rounds repeat (at
 * most OR_REACH_ROUNDS) while unreached vertices remain.
 */
void or_reach_fix(const or_input* in, int32_t R, int32_t entry_g, int32_t beam,
                  int32_t* out_ids, float* out_dist, int32_t* out_deg, or_stats* st) {
    const int64_t N = in->off[in->h];
    uint8_t* reached = (uint8_t*)malloc(N);
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* reps = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* level = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* npar = (int32_t*)malloc(sizeof(int32_t) * N);
    int64_t attached = 0;
    set_threads(in->nthreads);
    for (int round = 0; round < OR_REACH_ROUNDS; ++round) {
        memset(reached, 0, N);
        memset(level, 0, sizeof(int32_t) * N);
        int64_t nr = bfs_level(N, R, out_ids, entry_g, reached, queue, level);
        if (nr == N) break;
        /* BFS parents: in-neighbours at a smaller level */
        memset(npar, 0, sizeof(int32_t) * N);
        for (int64_t x = 0; x < N; ++x) {
            if (!level[x]) continue;
            for (int32_t t = 0; t < R; ++t) {
                int32_t y = out_ids[x * R + t];
                if (y >= 0 && level[y] > level[x]) npar[y]++;
            }
        }
        for (int64_t x = 0; x < N; ++x) parent[x] = (int32_t)x;
        for (int64_t x = 0; x < N; ++x) {
            if (reached[x]) continue;
            for (int32_t t = 0; t < R; ++t) {
                int32_t y = out_ids[x * R + t];
                if (y >= 0 && !reached[y]) uf_union(parent, (int32_t)x, y);
            }
        }
        int64_t nreps = 0;
        for (int64_t x = 0; x < N; ++x)
            if (!reached[x] && uf_find(parent, (int32_t)x) == x) reps[nreps++] = (int32_t)x;
        int32_t* cid = (int32_t*)malloc(sizeof(int32_t) * nreps * beam);
        float* cdist = (float*)malloc(sizeof(float) * nreps * beam);
        int32_t* cn = (int32_t*)malloc(sizeof(int32_t) * nreps);
#pragma omp parallel
        {
            uint32_t* seen = (uint32_t*)calloc(N, sizeof(uint32_t));
            uint32_t tag = 0;
#pragma omp for schedule(dynamic, 1)
            for (int64_t r = 0; r < nreps; ++r) {
                ++tag;
                cn[r] = knn_search_tagged(in->X, in->d, in->metric, out_ids, R, entry_g, row(in, reps[r]), beam, beam,
                                          seen, tag, cid + r * beam, cdist + r * beam, NULL);
            }
            free(seen);
        }
        for (int64_t r = 0; r < nreps; ++r) {
            int32_t x = reps[r];
            int32_t p = -1, pos = -1;
            for (int32_t t = 0; t < cn[r] && p < 0; ++t)
                if (out_deg[cid[r * beam + t]] < R) { p = cid[r * beam + t]; pos = out_deg[p]; }
            for (int32_t t = 0; t < cn[r] && p < 0; ++t) {
                int32_t q = cid[r * beam + t];
                for (int32_t s = out_deg[q] - 1; s >= 0; --s) {
                    int32_t y = out_ids[(int64_t)q * R + s];
                    int32_t other = npar[y] - (level[q] < level[y] ? 1 : 0);
                    if (level[y] > 0 && other >= 1) { p = q; pos = s; break; }
                }
            }
            if (p < 0) continue;
            int32_t* li = out_ids + (int64_t)p * R;
            float* ld = out_dist + (int64_t)p * R;
            float d = dist_g(in, p, x);
            if (pos == out_deg[p]) out_deg[p] += 1;
            else if (level[p] < level[li[pos]]) npar[li[pos]] -= 1;
            /* place (d, x) at pos, then restore ascending (delta, id) */
            while (pos > 0 && key_lt(d, x, ld[pos - 1], li[pos - 1])) {
                li[pos] = li[pos - 1]; ld[pos] = ld[pos - 1]; --pos;
            }
            while (pos + 1 < out_deg[p] && key_lt(ld[pos + 1], li[pos + 1], d, x)) {
                li[pos] = li[pos + 1]; ld[pos] = ld[pos + 1]; ++pos;
            }
            li[pos] = x;
            ld[pos] = d;
            ++attached;
        }
        free(cid);
        free(cdist);
        free(cn);
    }
    if (st) {
        st->attached += attached;
        memset(reached, 0, N);
        st->unreached += N - bfs_mark(N, R, out_ids, entry_g, reached, queue);
    }
    free(reached);
    free(queue);
    free(parent);
    free(reps);
    free(level);
    free(npar);
}

/* ------------------------------------------------------------------------- */
/* The reachability fix as the plain sequential rule first proposed for it: the */
/* quality reference for the round-based form above (which the kernels follow). */
/* ------------------------------------------------------------------------- */
/* BFS from the entry; then for each vertex x in ascending id that is still unreached: the
 * candidates p are the reached vertices of x's k-NNG list (ascending (delta, id); none when
 * knn_ids is NULL), then the reached results of Alg. 1 for x over the current graph from the
 * entry (pool beam). The first p with fewer than R neighbours takes x at the end of its list;
 * else the first p having a neighbour of indegree > 1 has its farthest such neighbour (by
 * descending (delta, id)) replaced by x. p's list is re-sorted by (delta, id) and every vertex
 * reachable from x is marked reached. Sequential. */
void or_reach_fix_seq(const or_input* in, int32_t R, int32_t entry_g, int32_t beam, const int32_t* knn_ids,
                      int32_t k, int32_t* out_ids, float* out_dist, int32_t* out_deg, or_stats* st) {
    const int64_t N = in->off[in->h];
    uint8_t* reached = (uint8_t*)calloc(N, 1);
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* indeg = (int32_t*)calloc(N, sizeof(int32_t));
    uint32_t* seen = (uint32_t*)calloc(N, sizeof(uint32_t));
    int32_t* cid = (int32_t*)malloc(sizeof(int32_t) * (beam + k + 1));
    float* cdist = (float*)malloc(sizeof(float) * (beam + 1));
    uint32_t tag = 0;
    int64_t attached = 0;
    for (int64_t u = 0; u < N; ++u)
        for (int32_t t = 0; t < out_deg[u]; ++t) indeg[out_ids[u * R + t]]++;
    bfs_mark(N, R, out_ids, entry_g, reached, queue);
    for (int64_t x = 0; x < N; ++x) {
        if (reached[x]) continue;
        /* candidates: reached k-NNG neighbours, then reached search results */
        int32_t nc = 0;
        if (knn_ids)
            for (int32_t t = 0; t < k; ++t) {
                int32_t v = knn_ids[x * k + t];
                if (v >= 0 && reached[v]) cid[nc++] = v;
            }
        int32_t ns = knn_search_tagged(in->X, in->d, in->metric, out_ids, R, entry_g, row(in, x), beam, beam, seen,
                                       ++tag, cid + nc, cdist, NULL);
        int32_t w = nc;
        for (int32_t t = 0; t < ns; ++t)
            if (reached[cid[nc + t]]) cid[w++] = cid[nc + t];
        nc = w;
        int32_t p = -1, pos = -1;
        for (int32_t t = 0; t < nc && p < 0; ++t)
            if (out_deg[cid[t]] < R) { p = cid[t]; pos = out_deg[p]; }
        for (int32_t t = 0; t < nc && p < 0; ++t) {
            int32_t q = cid[t];
            for (int32_t s = out_deg[q] - 1; s >= 0; --s)
                if (indeg[out_ids[(int64_t)q * R + s]] > 1) { p = q; pos = s; break; }
        }
        if (p < 0) continue;
        int32_t* li = out_ids + (int64_t)p * R;
        float* ld = out_dist + (int64_t)p * R;
        float d = dist_g(in, p, x);
        if (pos == out_deg[p]) out_deg[p] += 1;
        else indeg[li[pos]]--;
        indeg[x]++;
        while (pos > 0 && key_lt(d, (int32_t)x, ld[pos - 1], li[pos - 1])) {
            li[pos] = li[pos - 1]; ld[pos] = ld[pos - 1]; --pos;
        }
        while (pos + 1 < out_deg[p] && key_lt(ld[pos + 1], li[pos + 1], d, (int32_t)x)) {
            li[pos] = li[pos + 1]; ld[pos] = ld[pos + 1]; ++pos;
        }
        li[pos] = (int32_t)x;
        ld[pos] = d;
        ++attached;
        bfs_mark(N, R, out_ids, (int32_t)x, reached, queue);
    }
    if (st) {
        st->attached += attached;
        memset(reached, 0, N);
        st->unreached += N - bfs_mark(N, R, out_ids, entry_g, reached, queue);
    }
    free(reached); free(queue); free(indeg); free(seen); free(cid); free(cdist);
}

/* ------------------------------------------------------------------------- */
/* Alg. 3 as printed: the streamlined (one pass per vertex) refinement in DFS   */
/* order, reverse graphs kept across iterations, lists updated at once (the     */
/* quality comparison for the synchronous form above). Sequential.              */
/* ------------------------------------------------------------------------- */
typedef struct { int32_t* v; int32_t n, cap; } ivec_t;

static void ivec_push(ivec_t* a, int32_t x) {
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 8;
        a->v = (int32_t*)realloc(a->v, sizeof(int32_t) * a->cap);
    }
    a->v[a->n++] = x;
}

static int ivec_has(const int32_t* v, int32_t n, int32_t x) {
    for (int32_t i = 0; i < n; ++i)
        if (v[i] == x) return 1;
    return 0;
}

void or_refine_dfs(const or_input* in, int32_t k, int32_t iters, int32_t* ids, float* dist, uint8_t* flags,
                   int32_t* T, or_stats* st) {
    const int64_t N = in->off[in->h];
    ivec_t* rn = (ivec_t*)calloc(N, sizeof(ivec_t));   /* reverse graph of new entries */
    ivec_t* ro = (ivec_t*)calloc(N, sizeof(ivec_t));   /* of old entries */
    uint8_t* seen = (uint8_t*)malloc(N);
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (N + 1));
    ivec_t cn = {0, 0, 0}, co = {0, 0, 0};
    for (int32_t it = 0; it < iters; ++it) {
        memset(seen, 0, N);
        for (int64_t u0 = 0; u0 < N; ++u0) {
            if (seen[u0]) continue;
            int64_t sp = 0;
            stack[sp++] = (int32_t)u0;
            seen[u0] = 1;
            while (sp > 0) {
                const int32_t v = stack[--sp];
                /* Visit v: its forward entries split new / old (new ones become old), each
                 * recorded in the partner's reverse graph */
                cn.n = co.n = 0;
                for (int32_t t = 0; t < k; ++t) {
                    const int32_t w = ids[(int64_t)v * k + t];
                    if (w < 0) continue;
                    if (flags[(int64_t)v * k + t] & OR_FLAG_NEW) {
                        ivec_push(&cn, w);
                        flags[(int64_t)v * k + t] &= (uint8_t)~OR_FLAG_NEW;
                        ivec_push(&rn[w], v);
                    } else {
                        ivec_push(&co, w);
                        ivec_push(&ro[w], v);
                    }
                }
                /* DFS: the neighbours of v next */
                for (int32_t t = k - 1; t >= 0; --t) {
                    const int32_t w = ids[(int64_t)v * k + t];
                    if (w >= 0 && !seen[w]) {
                        seen[w] = 1;
                        stack[sp++] = w;
                    }
                }
                /* move the reverse entries recorded for v into its candidate sets */
                for (int32_t i = 0; i < rn[v].n; ++i)
                    if (!ivec_has(cn.v, cn.n, rn[v].v[i])) ivec_push(&cn, rn[v].v[i]);
                for (int32_t i = 0; i < ro[v].n; ++i)
                    if (!ivec_has(cn.v, cn.n, ro[v].v[i]) && !ivec_has(co.v, co.n, ro[v].v[i]))
                        ivec_push(&co, ro[v].v[i]);
                rn[v].n = ro[v].n = 0;
                /* Update: C_n^2 and C_n x C_o, cross-graph pairs, lists changed at once */
                for (int32_t i = 0; i < cn.n; ++i) {
                    const int32_t a = cn.v[i];
                    for (int32_t j = 0; j < cn.n + co.n; ++j) {
                        if (j < cn.n && j <= i) continue;
                        const int32_t b = j < cn.n ? cn.v[j] : co.v[j - cn.n];
                        if (a == b || shard_of(in, a) == shard_of(in, b)) continue;
                        const float d = dist_g(in, a, b);
                        if (st) st->pairs++;
                        if (list_insert(ids + (int64_t)a * k, dist + (int64_t)a * k, flags + (int64_t)a * k, k, b, d) && st)
                            st->updates++;
                        if (list_insert(ids + (int64_t)b * k, dist + (int64_t)b * k, flags + (int64_t)b * k, k, a, d) && st)
                            st->updates++;
                    }
                }
            }
        }
        or_indegree_repair(in, k, ids, dist, flags, T, st);
    }
    for (int64_t v = 0; v < N; ++v) {
        free(rn[v].v);
        free(ro[v].v);
    }
    free(rn);
    free(ro);
    free(seen);
    free(stack);
    free(cn.v);
    free(co.v);
}

int32_t or_merged_entry(const or_input* in) {
    /* the shard with the most valid vertices (lowest index on ties) */
    int best = 0;
    int64_t best_n = -1;
    for (int s = 0; s < in->h; ++s) {
        int64_t nv = 0;
        for (int64_t g = in->off[s]; g < in->off[s + 1]; ++g) nv += (!in->valid || in->valid[g]) ? 1 : 0;
        if (nv > best_n) {
            best = s;
            best_n = nv;
        }
    }
    /* its entry mapped by phi, else its first valid vertex */
    int32_t* phi = (int32_t*)malloc(sizeof(int32_t) * (in->off[in->h] > 0 ? in->off[in->h] : 1));
    or_phi(in, phi);
    int32_t e = phi[in->off[best] + in->entry[best]];
    for (int64_t g = in->off[best]; e < 0 && g < in->off[best + 1]; ++g) e = phi[g];
    free(phi);
    return e;
}

int32_t or_merge(const or_input* in, int32_t k, int32_t L, int32_t iters, int32_t rev_cap, int32_t R,
                 float alpha, int32_t ensure_reachable, int32_t* out_ids, float* out_dist, int32_t* out_deg,
                 int32_t* out_entry, int32_t* knn_ids_out, float* knn_dist_out, or_stats* st) {
    return or_merge_rule(in, k, L, iters, rev_cap, R, OR_PRUNE_ARNG, alpha, 0.f, ensure_reachable, out_ids, out_dist,
                         out_deg, out_entry, knn_ids_out, knn_dist_out, st);
}

int32_t or_merge_rule(const or_input* in, int32_t k, int32_t L, int32_t iters, int32_t rev_cap, int32_t R,
                      int32_t rule, float alpha, float tau, int32_t ensure_reachable, int32_t* out_ids,
                      float* out_dist, int32_t* out_deg, int32_t* out_entry, int32_t* knn_ids_out,
                      float* knn_dist_out, or_stats* st) {
    const int64_t N = in->off[in->h];
    int32_t* ids = (int32_t*)malloc(sizeof(int32_t) * N * k);
    float* dist = (float*)malloc(sizeof(float) * N * k);
    uint8_t* flags = (uint8_t*)malloc(N * k);
    int32_t* T = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* e_ids = (int32_t*)malloc(sizeof(int32_t) * N * R);
    float* e_dist = (float*)malloc(sizeof(float) * N * R);
    int32_t* e_cnt = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t Lu = or_stage_a(in, k, L, ids, dist, flags, st);
    for (int32_t it = 0; it < iters; ++it) {
        or_refine_iter(in, k, rev_cap, ids, dist, flags, st);
        or_indegree_repair(in, k, ids, dist, flags, T, st);
    }
    if (iters <= 0) or_indegree(ids, N, k, T);
    or_prune_rule(in, k, ids, dist, T, R, rule, alpha, tau, e_ids, e_dist, e_cnt, st);
    or_reverse_insert(N, R, e_ids, e_dist, e_cnt, out_ids, out_dist, out_deg);
    int32_t entry = or_merged_entry(in);
    if (ensure_reachable) or_reach_fix(in, R, entry, 64, out_ids, out_dist, out_deg, st);
    *out_entry = entry;
    if (knn_ids_out) memcpy(knn_ids_out, ids, sizeof(int32_t) * N * k);
    if (knn_dist_out) memcpy(knn_dist_out, dist, sizeof(float) * N * k);
    free(ids); free(dist); free(flags); free(T); free(e_ids); free(e_dist); free(e_cnt);
    return Lu;
}

void or_search(const float* X, int64_t N, int32_t d, int32_t metric, const int32_t* g_ids, int32_t R,
               int32_t entry, const float* Q, int64_t nq, int32_t beam, int32_t topk, int32_t nthreads,
               int32_t* out_ids, float* out_dist, or_stats* st) {
    set_threads(nthreads);
    int64_t ndc = 0, hops = 0;
#pragma omp parallel reduction(+ : ndc, hops)
    {
        uint32_t* seen = (uint32_t*)calloc(N, sizeof(uint32_t));
        uint32_t tag = 0;
        or_stats ls;
        memset(&ls, 0, sizeof(ls));
#pragma omp for schedule(dynamic, 8)
        for (int64_t qi = 0; qi < nq; ++qi) {
            ++tag;
            int32_t r = knn_search_tagged(X, d, metric, g_ids, R, entry, Q + qi * (int64_t)d, beam, topk, seen, tag,
                                          out_ids + qi * topk, out_dist + qi * topk, &ls);
            for (int32_t t = r; t < topk; ++t) {
                out_ids[qi * topk + t] = -1;
                out_dist[qi * topk + t] = INFINITY;
            }
        }
        ndc += ls.ndc;
        hops += ls.hops;
        free(seen);
    }
    if (st) {
        st->ndc += ndc;
        st->hops += hops;
    }
}
