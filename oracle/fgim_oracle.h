/*
 * FGIM merge oracle: plain, slow, obviously-correct CPU reference.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. The product path (the
 * CUDA library and its Python binding) never calls it and shares no code,
 * header, helper or table with it.
 *
 * Every distance is evaluated in FP64 from the stored FP32 inputs and rounded
 * once to FP32; every ordering decision (pool order, top-k, prune test) is then
 * taken on those FP32 values with the (distance, global id) lexicographic order.
 *
 * Layout conventions shared by all entry points (host arrays):
 *   X        [N, d] float32, global ids in phi order: shard i owns rows
 *            [off[i], off[i+1]) (Sec. 4.1.3, phi as offsets).
 *   adj      [N, M] int32: row g is the input-PG row of global vertex g and
 *            holds LOCAL ids of g's shard, -1 padded.
 *   entry    [h] local entry point of each input PG.
 *   k-NNG    ids [N, k] int32 (-1 empty), dist [N, k] float32 (+inf empty),
 *            flags [N, k] uint8 (bit0 new, bit1 replaced), each row sorted
 *            ascending by (dist, id) with the empty slots last.
 *   valid    optional [N] uint8 (NULL = every vertex valid): the boolean part of
 *            the ID mapping phi of Sec. 4.1.3. Valid vertices take consecutive
 *            global ids in (shard, local id) order; invalid ones get no row and
 *            never appear as a neighbour, but stay in their input PG for routing.
 */
#ifndef FGIM_ORACLE_H
#define FGIM_ORACLE_H
#include <stdint.h>

#define OR_FLAG_NEW 1u
#define OR_FLAG_REPLACED 2u

#define OR_METRIC_L2 0
#define OR_METRIC_IP 1
#define OR_METRIC_COS 2

typedef struct {
    const float* X;
    int64_t N;
    int32_t d;
    int32_t metric;
    int32_t h;
    const int64_t* off;    /* [h + 1] */
    const int32_t* adj;    /* [N, M] local ids */
    int32_t M;
    const int32_t* entry;  /* [h] local */
    int32_t nthreads;      /* 0 = OpenMP default */
    const uint8_t* valid;  /* [N] or NULL; honoured by or_stage_a and or_merged_entry */
} or_input;

typedef struct {
    int64_t ndc;           /* distance computations */
    int64_t hops;          /* beam-search expansions */
    int64_t pairs;         /* join pairs evaluated */
    int64_t updates;       /* list insertions accepted */
    int64_t zero_before;   /* zero-indegree vertices before repair */
    int64_t zero_after;
    int64_t replaced;      /* repair replacements */
    int64_t prune_dist;    /* delta(w, v) evaluations in the prune */
    int64_t unreached;     /* vertices left unreached after the reachability fix */
    int64_t attached;      /* vertices attached by the reachability fix */
} or_stats;

double or_delta64(const float* x, const float* y, int32_t d, int32_t metric);
float or_delta(const float* x, const float* y, int32_t d, int32_t metric);

/* Alg. 1 on one graph of n vertices whose rows are X_local[v] and adj_local[v]; returns #results. */
int32_t or_knn_search(const float* X_local, int64_t n, int32_t d, int32_t metric, const int32_t* adj_local,
                      int32_t M, int32_t ep, const float* q, int32_t L, int32_t k,
                      int32_t* out_ids, float* out_dist, or_stats* st);

/* Exact k-NN by exhaustive scan; exclude[q] (or -1) is skipped. */
void or_knn_exact(const float* X, int64_t N, int32_t d, int32_t metric, const float* Q, int64_t nq,
                  const int64_t* exclude, int32_t k, int32_t nthreads, int32_t* out_ids, float* out_dist);

/* Alg. 2: PGs -> k-NNG. L <= 0 selects ceil(k / (h - 1)). */
int32_t or_stage_a(const or_input* in, int32_t k, int32_t L, int32_t* ids, float* dist, uint8_t* flags,
                   or_stats* st);

/* One synchronous Visit + Update pass of Alg. 3 over the k-NNG (in place). */
void or_refine_iter(const or_input* in, int32_t k, int32_t rev_cap, int32_t* ids, float* dist,
                    uint8_t* flags, or_stats* st);

/* Alg. 4 (in place); T [N] receives the indegree recorder of the repaired graph. */
void or_indegree_repair(const or_input* in, int32_t k, int32_t* ids, float* dist, uint8_t* flags,
                        int32_t* T, or_stats* st);

/* Indegree of every vertex over the valid entries of a [N, k] list array. */
void or_indegree(const int32_t* ids, int64_t N, int32_t k, int32_t* T);

/* Alg. 5 neighbour selection: E' [N, R] (ids -1 padded, dist), cnt [N]. or_prune is the
 * alpha-RNG rule; or_prune_rule takes the rule (OR_PRUNE_*, see fgim_oracle.c) and tau of tau-MNG.
 * Every rule keeps a candidate whose indegree T is 1 (Alg. 5). */
#define OR_PRUNE_ARNG 0
#define OR_PRUNE_MRNG 1
#define OR_PRUNE_TMNG 2
void or_prune(const or_input* in, int32_t k, const int32_t* ids, const float* dist, const int32_t* T,
              int32_t R, float alpha, int32_t* e_ids, float* e_dist, int32_t* e_cnt, or_stats* st);
void or_prune_rule(const or_input* in, int32_t k, const int32_t* ids, const float* dist, const int32_t* T,
                   int32_t R, int32_t rule, float alpha, float tau, int32_t* e_ids, float* e_dist, int32_t* e_cnt,
                   or_stats* st);

/* Alg. 5 connectivity enhancement: out [N, R] from E' and its reverse edges. */
void or_reverse_insert(int64_t N, int32_t R, const int32_t* e_ids, const float* e_dist, const int32_t* e_cnt,
                       int32_t* out_ids, float* out_dist, int32_t* out_deg);

/* Reachability fix (added step, not in the paper): attach every vertex unreachable from entry. */
void or_reach_fix(const or_input* in, int32_t R, int32_t entry_g, int32_t beam,
                  int32_t* out_ids, float* out_dist, int32_t* out_deg, or_stats* st);

/* The reachability fix as the plain sequential rule (the quality reference for or_reach_fix): each
 * unreached vertex in ascending id is attached to the first reached vertex of its k-NNG list
 * (knn_ids [N, k] or NULL), else of its search results, that has room, else that has a neighbour
 * of indegree > 1 (the farthest such one is replaced); see fgim_oracle.c. */
void or_reach_fix_seq(const or_input* in, int32_t R, int32_t entry_g, int32_t beam, const int32_t* knn_ids,
                      int32_t k, int32_t* out_ids, float* out_dist, int32_t* out_deg, or_stats* st);

/* Global id of the merged entry point: phi(entry of the largest shard, lowest shard index on ties). */
int32_t or_merged_entry(const or_input* in);
/* Alg. 3 as printed (DFS order, Visit and Update in one pass per vertex, lists updated at once,
 * reverse graphs kept across iterations), `iters` iterations each followed by Alg. 4; T gets
 * the indegrees after the last repair. The quality comparison for or_refine_iter. */
void or_refine_dfs(const or_input* in, int32_t k, int32_t iters, int32_t* ids, float* dist, uint8_t* flags,
                   int32_t* T, or_stats* st);
void or_knn_prefix(const float* X, int64_t N, int32_t d, int32_t metric, int32_t k, int32_t nthreads,
                   int32_t* out_ids, float* out_dist);
/* phi of Sec. 4.1.3 from in->valid: phi[g] = global id of g in the merged index or -1.
 * Returns the number of valid vertices. */
int64_t or_phi(const or_input* in, int32_t* phi);

/* Full merge: stage a, iters x (refine + repair), prune, reverse insertion, reachability fix.
 * or_merge prunes with alpha-RNG; or_merge_rule with the given rule. */
int32_t or_merge(const or_input* in, int32_t k, int32_t L, int32_t iters, int32_t rev_cap, int32_t R,
                 float alpha, int32_t ensure_reachable, int32_t* out_ids, float* out_dist, int32_t* out_deg,
                 int32_t* out_entry, int32_t* knn_ids_out, float* knn_dist_out, or_stats* st);
int32_t or_merge_rule(const or_input* in, int32_t k, int32_t L, int32_t iters, int32_t rev_cap, int32_t R,
                      int32_t rule, float alpha, float tau, int32_t ensure_reachable, int32_t* out_ids,
                      float* out_dist, int32_t* out_deg, int32_t* out_entry, int32_t* knn_ids_out,
                      float* knn_dist_out, or_stats* st);

/* HNSW's upper layers built as HNSW builds them (Sec. 4.3.3): the vertices of level >= 1 inserted
 * one at a time in ascending id (greedy descent, Alg. 1 with pool ef per layer, HNSW's
 * heuristic to M, edges both ways, overflowing lists re-pruned). adj [max_level, N, M] global
 * ids, -1 padded (layer l at offset (l - 1) N M); entry_out: the top vertex. */
void or_hnsw_insert(const float* X, int64_t N, int32_t d, int32_t metric, const int32_t* levels, int32_t max_level,
                    int32_t M, int32_t ef, int32_t* adj, int32_t* entry_out, or_stats* st);

/* Alg. 1 over the merged graph (global ids, rows of R) for nq queries. */
void or_search(const float* X, int64_t N, int32_t d, int32_t metric, const int32_t* g_ids, int32_t R,
               int32_t entry, const float* Q, int64_t nq, int32_t beam, int32_t topk, int32_t nthreads,
               int32_t* out_ids, float* out_dist, or_stats* st);

#endif
