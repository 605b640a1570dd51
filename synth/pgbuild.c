/*
 * Input proximity-graph builder for the synthetic workloads.
 *
 * Input generation only: this builds the h pre-built indexes G_i that the
 * merge (Sec. 2.1, Definition "Merging Graph-based Indexes") takes as input.
 * It is a flat, HNSW-style incremental insertion graph: every new point runs
 * HNSW's best-first layer search (two heaps, stop when the closest open
 * candidate is farther than the farthest kept result) over the graph built so
 * far, keeps up to M neighbours with HNSW's diversity heuristic, and adds the
 * reverse edges, re-running the heuristic on lists that overflow M.
 *
 * Determinism: points are inserted in batches; every point of a batch searches
 * the graph frozen at the batch start (parallel over points), then the reverse
 * edges are applied per target vertex in ascending source id (parallel over
 * targets). The output depends only on the inputs, never on the thread count.
 * All comparisons order (distance, id) lexicographically.
 *
 * Shares no code with the merge oracle or the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { float d; int32_t id; } cand_t;

static inline int cand_lt(cand_t a, cand_t b) {
    return a.d < b.d || (a.d == b.d && a.id < b.id);
}

typedef struct {
    const float* X;
    const float* inv_norm;   /* cosine only */
    int64_t n;
    int d;
    int metric;              /* 0 squared L2, 1 inner product (1 - x.y), 2 cosine */
} space_t;

static inline float pg_dist(const space_t* s, int64_t a, int64_t b) {
    const float* x = s->X + a * s->d;
    const float* y = s->X + b * s->d;
    float acc = 0.f;
    if (s->metric == 0) {
        for (int t = 0; t < s->d; ++t) { float z = x[t] - y[t]; acc += z * z; }
        return acc;
    }
    for (int t = 0; t < s->d; ++t) acc += x[t] * y[t];
    if (s->metric == 2) acc *= s->inv_norm[a] * s->inv_norm[b];
    return 1.f - acc;
}

/* ---- binary heaps over cand_t ---- */
typedef struct { cand_t* a; int n; } heap_t;

static void heap_push_min(heap_t* h, cand_t c) {
    int i = h->n++;
    h->a[i] = c;
    while (i > 0) {
        int p = (i - 1) >> 1;
        if (!cand_lt(h->a[i], h->a[p])) break;
        cand_t t = h->a[i]; h->a[i] = h->a[p]; h->a[p] = t; i = p;
    }
}
static cand_t heap_pop_min(heap_t* h) {
    cand_t top = h->a[0];
    h->a[0] = h->a[--h->n];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->n && cand_lt(h->a[l], h->a[m])) m = l;
        if (r < h->n && cand_lt(h->a[r], h->a[m])) m = r;
        if (m == i) break;
        cand_t t = h->a[i]; h->a[i] = h->a[m]; h->a[m] = t; i = m;
    }
    return top;
}
static void heap_push_max(heap_t* h, cand_t c) {
    int i = h->n++;
    h->a[i] = c;
    while (i > 0) {
        int p = (i - 1) >> 1;
        if (!cand_lt(h->a[p], h->a[i])) break;
        cand_t t = h->a[i]; h->a[i] = h->a[p]; h->a[p] = t; i = p;
    }
}
static cand_t heap_pop_max(heap_t* h) {
    cand_t top = h->a[0];
    h->a[0] = h->a[--h->n];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->n && cand_lt(h->a[m], h->a[l])) m = l;
        if (r < h->n && cand_lt(h->a[m], h->a[r])) m = r;
        if (m == i) break;
        cand_t t = h->a[i]; h->a[i] = h->a[m]; h->a[m] = t; i = m;
    }
    return top;
}

static int cand_cmp(const void* pa, const void* pb) {
    cand_t a = *(const cand_t*)pa, b = *(const cand_t*)pb;
    if (cand_lt(a, b)) return -1;
    if (cand_lt(b, a)) return 1;
    return 0;
}

typedef struct {
    int32_t* nbr;   /* [n, M] */
    float* nd;      /* [n, M] distance of each neighbour to the list owner */
    int32_t* cnt;   /* [n] */
    int M;
} graph_t;

/* HNSW layer search over the frozen graph; returns the number of results, sorted ascending. */
static int layer_search(const space_t* s, const graph_t* g, int64_t q, int32_t ep, int ef,
                        uint32_t* tag, uint32_t epoch, cand_t* cbuf, cand_t* wbuf, cand_t* out) {
    heap_t C = {cbuf, 0}, W = {wbuf, 0};
    cand_t e0 = {pg_dist(s, q, ep), ep};
    tag[ep] = epoch;
    heap_push_min(&C, e0);
    heap_push_max(&W, e0);
    while (C.n > 0) {
        cand_t c = heap_pop_min(&C);
        if (cand_lt(W.a[0], c)) break;
        const int32_t* nb = g->nbr + (int64_t)c.id * g->M;
        for (int t = 0; t < g->cnt[c.id]; ++t) {
            int32_t v = nb[t];
            if (tag[v] == epoch) continue;
            tag[v] = epoch;
            cand_t e = {pg_dist(s, q, v), v};
            if (W.n < ef || cand_lt(e, W.a[0])) {
                heap_push_min(&C, e);
                heap_push_max(&W, e);
                if (W.n > ef) heap_pop_max(&W);
            }
        }
    }
    int m = W.n;
    for (int i = m - 1; i >= 0; --i) out[i] = heap_pop_max(&W);
    return m;
}

/* HNSW neighbour-selection heuristic over candidates sorted ascending by distance to the base. */
static int select_heuristic(const space_t* s, const cand_t* cand, int nc, int M, cand_t* keep) {
    int nk = 0;
    for (int i = 0; i < nc && nk < M; ++i) {
        int good = 1;
        for (int j = 0; j < nk; ++j) {
            if (pg_dist(s, cand[i].id, keep[j].id) < cand[i].d) { good = 0; break; }
        }
        if (good) keep[nk++] = cand[i];
    }
    return nk;
}

typedef struct { int32_t v, p; float d; } redge_t;

static int redge_cmp(const void* pa, const void* pb) {
    const redge_t* a = (const redge_t*)pa;
    const redge_t* b = (const redge_t*)pb;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    if (a->p != b->p) return a->p < b->p ? -1 : 1;
    return 0;
}

/*
 * X: [n, d] row-major float32. adj_out: [n, M] int32, -1 padded. entry_out: medoid.
 * Returns 0 on success, negative on allocation failure or bad arguments.
 */
int pg_build(const float* X, int64_t n, int d, int metric, int M, int ef, int max_batch,
             int nthreads, int32_t* adj_out, int32_t* entry_out) {
    if (n <= 0 || d <= 0 || M <= 0 || ef < 1 || max_batch < 1) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    int T = omp_get_max_threads();
#else
    int T = 1;
    (void)nthreads;
#endif
    space_t s = {X, NULL, n, d, metric};
    float* inv = NULL;
    if (metric == 2) {
        inv = (float*)malloc(sizeof(float) * n);
        if (!inv) return -2;
        for (int64_t i = 0; i < n; ++i) {
            double a = 0;
            for (int t = 0; t < d; ++t) a += (double)X[i * d + t] * X[i * d + t];
            inv[i] = (float)(1.0 / sqrt(a > 0 ? a : 1.0));
        }
        s.inv_norm = inv;
    }
    /* medoid: the point closest (squared L2) to the mean, ties to the lowest id */
    double* mean = (double*)calloc(d, sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int t = 0; t < d; ++t) mean[t] += X[i * d + t];
    for (int t = 0; t < d; ++t) mean[t] /= (double)n;
    int64_t medoid = 0;
    double best = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double a = 0;
        for (int t = 0; t < d; ++t) { double z = X[i * d + t] - mean[t]; a += z * z; }
        if (a < best) { best = a; medoid = i; }
    }
    free(mean);

    graph_t g;
    g.M = M;
    g.nbr = (int32_t*)malloc(sizeof(int32_t) * n * M);
    g.nd = (float*)malloc(sizeof(float) * n * M);
    g.cnt = (int32_t*)calloc(n, sizeof(int32_t));
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * n);
    uint32_t* tags = (uint32_t*)calloc((size_t)T * n, sizeof(uint32_t));
    /* per thread: open-candidate heap (bounded by n), result heap (ef + 1), list scratch */
    int64_t heap_cap = n + ef + 16;
    int64_t cap = (ef > M + max_batch ? ef : M + max_batch) + 8;
    cand_t* cbufs = (cand_t*)malloc(sizeof(cand_t) * (size_t)T * heap_cap);
    cand_t* outs = (cand_t*)malloc(sizeof(cand_t) * (size_t)T * cap);
    int32_t* bl_nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)max_batch * M);
    float* bl_nd = (float*)malloc(sizeof(float) * (size_t)max_batch * M);
    int32_t* bl_cnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)max_batch);
    redge_t* red = (redge_t*)malloc(sizeof(redge_t) * (size_t)max_batch * M);
    int64_t* vstart = (int64_t*)malloc(sizeof(int64_t) * ((size_t)max_batch * M + 1));
    if (!g.nbr || !g.nd || !g.cnt || !order || !tags || !cbufs || !outs || !bl_nbr || !bl_nd ||
        !bl_cnt || !red || !vstart) {
        free(g.nbr); free(g.nd); free(g.cnt); free(order); free(tags); free(cbufs); free(outs);
        free(bl_nbr); free(bl_nd); free(bl_cnt); free(red); free(vstart); free(inv);
        return -2;
    }
    order[0] = (int32_t)medoid;
    {
        int64_t w = 1;
        for (int64_t i = 0; i < n; ++i) if (i != medoid) order[w++] = (int32_t)i;
    }
    uint32_t* epochs = (uint32_t*)calloc((size_t)T * 16, sizeof(uint32_t));
    int64_t c = 1;
    while (c < n) {
        int64_t b = c / 2;
        if (b < 1) b = 1;
        if (b > max_batch) b = max_batch;
        if (b > n - c) b = n - c;
        /* 1. every point of the batch searches the frozen graph */
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t bi = 0; bi < b; ++bi) {
#ifdef _OPENMP
            int tid = omp_get_thread_num();
#else
            int tid = 0;
#endif
            int64_t p = order[c + bi];
            cand_t* cb = cbufs + (size_t)tid * heap_cap;
            cand_t* ob = outs + (size_t)tid * cap;
            uint32_t ep_tag = ++epochs[(size_t)tid * 16];
            int m = layer_search(&s, &g, p, (int32_t)medoid, ef, tags + (size_t)tid * n,
                                 ep_tag, cb + ef + 8, cb, ob);
            cand_t keep[256];
            int nk = select_heuristic(&s, ob, m, M < 256 ? M : 256, keep);
            bl_cnt[bi] = nk;
            for (int t = 0; t < nk; ++t) {
                bl_nbr[bi * M + t] = keep[t].id;
                bl_nd[bi * M + t] = keep[t].d;
            }
        }
        /* 2. install the new lists and gather reverse edges */
        int64_t ne = 0;
        for (int64_t bi = 0; bi < b; ++bi) {
            int64_t p = order[c + bi];
            g.cnt[p] = bl_cnt[bi];
            for (int t = 0; t < bl_cnt[bi]; ++t) {
                g.nbr[p * M + t] = bl_nbr[bi * M + t];
                g.nd[p * M + t] = bl_nd[bi * M + t];
                red[ne].v = bl_nbr[bi * M + t];
                red[ne].p = (int32_t)p;
                red[ne].d = bl_nd[bi * M + t];
                ++ne;
            }
        }
        qsort(red, ne, sizeof(redge_t), redge_cmp);
        int64_t nv = 0;
        for (int64_t e = 0; e < ne; ++e)
            if (e == 0 || red[e].v != red[e - 1].v) vstart[nv++] = e;
        vstart[nv] = ne;
        /* 3. reverse edges, independently per target vertex */
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t vi = 0; vi < nv; ++vi) {
#ifdef _OPENMP
            int tid = omp_get_thread_num();
#else
            int tid = 0;
#endif
            int32_t v = red[vstart[vi]].v;
            cand_t* cl = outs + (size_t)tid * cap;
            int nc = 0;
            for (int t = 0; t < g.cnt[v]; ++t) {
                cl[nc].id = g.nbr[(int64_t)v * M + t];
                cl[nc].d = g.nd[(int64_t)v * M + t];
                ++nc;
            }
            for (int64_t e = vstart[vi]; e < vstart[vi + 1]; ++e) {
                cl[nc].id = red[e].p;
                cl[nc].d = red[e].d;
                ++nc;
            }
            qsort(cl, nc, sizeof(cand_t), cand_cmp);
            cand_t keep[256];
            int nk;
            if (nc <= M) {
                nk = nc;
                memcpy(keep, cl, sizeof(cand_t) * nc);
            } else {
                nk = select_heuristic(&s, cl, nc, M < 256 ? M : 256, keep);
            }
            g.cnt[v] = nk;
            for (int t = 0; t < nk; ++t) {
                g.nbr[(int64_t)v * M + t] = keep[t].id;
                g.nd[(int64_t)v * M + t] = keep[t].d;
            }
        }
        c += b;
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int t = 0; t < M; ++t)
            adj_out[i * M + t] = t < g.cnt[i] ? g.nbr[i * M + t] : -1;
    }
    *entry_out = (int32_t)medoid;
    free(epochs);
    free(g.nbr); free(g.nd); free(g.cnt); free(order); free(tags); free(cbufs); free(outs);
    free(bl_nbr); free(bl_nd); free(bl_cnt); free(red); free(vstart); free(inv);
    return 0;
}
