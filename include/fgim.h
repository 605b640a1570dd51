/*
 * fgim.h -- C ABI of the GB300 (sm_103a) implementation of the FGIM merge hot path.
 *
 * FGIM merges h proximity-graph (PG) ANNS indexes built over disjoint vector sets
 * into one PG over their union (Sec. 2.1, Definition "Merging Graph-based Indexes
 * for ANNS"). The merge has three stages (Sec. 3.3):
 *   (a) PGs -> k-NNG by cross querying (Sec. 4.1, Alg. 1 + Alg. 2),
 *   (b) k-NNG refinement: Visit + Update local join and indegree repair (Sec. 4.2, Alg. 3 + Alg. 4),
 *   (c) k-NNG -> PG: neighbour selection and reverse-edge insertion (Sec. 4.3, Alg. 5),
 * followed by an added reachability fix (not in the paper) that attaches vertices the
 * entry point cannot reach.
 *
 * Conventions shared by every entry point:
 *  - All array arguments are DEVICE pointers unless the name ends in _host. They are
 *    borrowed: fgim never frees them and never keeps them after the call returns.
 *    Inputs are never modified (except arguments documented as in/out).
 *  - Global ids follow the ID mapping phi of Sec. 4.1.3 as offsets: local id v of
 *    shard i is global id  n_0 + ... + n_{i-1} + v.
 *  - Lists are rows of fixed width, sorted ascending by (distance, global id), valid
 *    entries first, empty slots hold id -1 and distance +inf.
 *  - Distances are squared L2, 1 - x.y (IP), or 1 - cos(x, y), evaluated in FP32.
 *  - Every call is ordered on `stream` (0 = legacy default stream). Scratch memory comes
 *    from a stream-ordered memory pool that the library keeps per device: a call takes
 *    its scratch from the pool on `stream` and hands it back before it returns, and the
 *    pool keeps the device memory it has mapped for later calls (fgim_trim_memory returns
 *    the unused part to the device). Calls return after the stream has drained (they
 *    synchronize the stream), so results are ready and every error is reported by the
 *    call itself.
 *  - Errors: argument errors are detected on the host before any work is queued and
 *    return FGIM_EINVAL / FGIM_EUNSUPPORTED. CUDA errors return FGIM_ECUDA (the CUDA
 *    error string is available from fgim_last_error()). A scratch allocation that fails
 *    returns FGIM_ENOMEM after handing back what the call had taken. A device-side
 *    bounded loop that ran out returns FGIM_ETIMEOUT. No exception crosses the ABI.
 *  - Not thread-safe for concurrent calls that share a stream; concurrent calls on
 *    different streams are safe, except fgim_search_noalloc, whose calls share one fixed
 *    device array and must not overlap on the GPU (see its comment).
 */
#ifndef FGIM_H
#define FGIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FGIM_OK = 0,
    FGIM_EINVAL = -1,
    FGIM_ENOMEM = -2,
    FGIM_ECUDA = -3,
    FGIM_ETIMEOUT = -4,
    FGIM_EUNSUPPORTED = -5,
    FGIM_EINTERNAL = -6
} fgim_status;

typedef enum { FGIM_L2SQ = 0, FGIM_IP = 1, FGIM_COSINE = 2 } fgim_metric;

/* Storage of the input vectors. BF16 vectors (bfloat16, round-to-nearest-even encodings of
 * the values the caller means) are decoded once per call into an FP32 working copy on the
 * device; every distance is that of the decoded values. */
typedef enum { FGIM_F32 = 0, FGIM_BF16 = 1 } fgim_dtype;

/* Size limits of the library. */
#define FGIM_MAX_SHARDS 64
#define FGIM_MAX_K 128          /* k of the k-NNG */
#define FGIM_MAX_R 128          /* degree bound of the merged PG */
#define FGIM_MAX_L 128          /* search pool (beam width) */
#define FGIM_MAX_DEGREE 128     /* max degree of an input PG */
#define FGIM_MAX_DIM 2048       /* dim must also be a multiple of 4 */

/* List-entry flags of the k-NNG (Sec. 4.2.1 new/old, Alg. 4 `replaced`). */
#define FGIM_FLAG_NEW 1u
#define FGIM_FLAG_REPLACED 2u

/* One input index G_i (Sec. 2.1): its vectors X_i and its PG. */
typedef struct {
    const void* vectors;     /* [n, dim] row-major in the params' dtype; 16-byte aligned (FP32), 2-byte (BF16) */
    const int32_t* adj;      /* [n, max_degree] LOCAL ids, -1 padded */
    int32_t n;               /* n_i >= 1 */
    int32_t max_degree;      /* 1 .. FGIM_MAX_DEGREE */
    int32_t entry;           /* entry point ep_i (local id) */
    int32_t reserved;
    /* Optional [n] device bytes, NULL = every vertex valid: the boolean part of the ID mapping
     * phi (Sec. 4.1.3), for merges with deleted vertices or with copies that another shard
     * already holds. A vertex with valid[v] == 0 gets no row in the merged index and is never
     * anybody's neighbour, but stays in its input PG: the cross-query searches still route
     * through it. The valid vertices take consecutive global ids in (shard, local id) order.
     * Honoured by fgim_merge, fgim_merge_batch and fgim_cross_query, whose outputs then have
     * one row per valid vertex (n = their number); the other entry points reject it. */
    const uint8_t* valid;
} fgim_shard;

typedef struct {
    int32_t dim;             /* d, multiple of 4, <= FGIM_MAX_DIM */
    int32_t dtype;           /* fgim_dtype */
    int32_t metric;          /* fgim_metric */
    int32_t k;               /* k of the k-NNG (Alg. 2 outdegree bound) */
    int32_t R;               /* degree bound of the merged PG (Alg. 5) */
    float alpha;             /* alpha-RNG factor of the prune; 1 = Alg. 5 as printed */
    int32_t L;               /* cross-query pool; 0 = ceil(k / (h - 1)) (Sec. 4.1.2) */
    int32_t iters;           /* I_max of Alg. 3 (>= 0) */
    int32_t rev_cap;         /* cap of each reverse list in Visit; 0 = k */
    int32_t ensure_reachable;/* 1 = run the reachability fix after Alg. 5 */
    int32_t reach_beam;      /* pool of the searches of the reachability fix; 0 = 64 */
    int32_t join_filter;     /* fgim_precision of Update's candidate distances: 0 = BF16 tensor-core tile
                                (tcgen05), 1 = FP32 SIMT tile, 2 = FP8 E4M3 tensor-core tile with one
                                scale per vector. Every form re-ranks its survivors with the exact FP32
                                distance, so the lists are the same; only speed differs. Passes whose
                                shapes a tensor-core tile does not cover (BF16: dim % 16 != 0; FP8:
                                dim % 32 != 0; both: |C_n| > 128, |C| > 256) use the FP32 tile. */
    int32_t byte_rows;       /* 0 = auto: when every coordinate is an integer in [0, 255] and dim <= 128,
                                dim % 16 == 0, the searches, the join's re-rank and the prune read one
                                byte per coordinate and form the distances in exact integer arithmetic
                                (they equal the FP32 distances bit for bit); 1 = off (FP32 rows only) */
    int32_t prune_rule;      /* fgim_prune_rule of Alg. 5's neighbour selection (0 = alpha-RNG) */
    float tau;               /* tau of FGIM_PRUNE_TAU_MNG (>= 0, in units of sqrt(distance)) */
    int32_t reserved;
} fgim_params;

/* Neighbour-selection rules of Alg. 5 (Sec. 4.3.1 names RNG, MRNG and tau-MNG as interchangeable;
 * the paper defines none but alpha-RNG, so the others follow the works it cites). u is the
 * vertex, candidates v are visited in ascending (distance, id), w ranges over the neighbours
 * kept so far; every rule keeps v when T(v) = 1 (Alg. 5's indegree clause) and stops at R.
 *   FGIM_PRUNE_ALPHA_RNG  w occludes v iff alpha^2 delta(w,v) >= delta(u,v) (alpha = 1: Alg. 5).
 *   FGIM_PRUNE_MRNG       w occludes v iff delta(w,v) < delta(u,v) (NSG's edge selection).
 *   FGIM_PRUNE_TAU_MNG    on the metric distances sqrt(delta): w occludes v iff sqrt(delta(u,w)) <
 *                         sqrt(delta(u,v)) and sqrt(delta(w,v)) < sqrt(delta(u,v)) - 3 tau, so
 *                         edges shorter than 3 tau are never pruned (decided in FP32:
 *                         t = sqrt(delta(u,v)) - 3 tau, occluded iff t > 0 and delta(w,v) < t * t). */
typedef enum { FGIM_PRUNE_ALPHA_RNG = 0, FGIM_PRUNE_MRNG = 1, FGIM_PRUNE_TAU_MNG = 2 } fgim_prune_rule;

/* Precision of Update's candidate distances (fgim_params.join_filter). The reduced-precision forms
 * are filters: a pair is re-ranked with the exact FP32 distance unless a rigorous bound (Cauchy-
 * Schwarz on the rows' conversion errors plus the FP32 accumulation error of the tile) shows it
 * cannot enter the list, so the kept ids equal the FP32 form's. FP8: s = amax|x| / 448 per vector,
 * q = saturating round-to-nearest E4M3 of x / s, the tile forms sum q_a q_b, scaled by s_a s_b. */
typedef enum { FGIM_PREC_BF16 = 0, FGIM_PREC_FP32 = 1, FGIM_PREC_FP8E4M3 = 2 } fgim_precision;

/* k-NNG buffers, caller-owned device memory: [n, k] each. */
typedef struct {
    int32_t* ids;
    float* dist;
    uint8_t* flags;
    int64_t n;
    int32_t k;
    int32_t reserved;
} fgim_knng;

/* Merged PG buffers, caller-owned device memory. */
typedef struct {
    int32_t* ids;            /* [n, R] global ids, -1 padded */
    float* dist;             /* [n, R] */
    int32_t* deg;            /* [n] */
    int64_t n;
    int32_t R;
    int32_t entry;           /* out: global id of the merged entry point */
} fgim_graph;

/*
 * Library-owned graph buffers, for callers that let the library allocate the merged PG:
 * fgim_graph_alloc takes one device block (cudaMalloc on the current device) holding ids [n, R],
 * dist [n, R] and deg [n], sets g->ids, dist, deg, n, R (entry 0), and returns FGIM_ENOMEM (g
 * zeroed) when the device has no room. fgim_graph_free releases a graph made by fgim_graph_alloc
 * and zeroes *g; it must not be given buffers the caller allocated, and it synchronizes the
 * device (cudaFree does). Both are safe on a zeroed graph.
 */
fgim_status fgim_graph_alloc(int64_t n, int32_t R, fgim_graph* g);
void fgim_graph_free(fgim_graph* g);

/* Counters of the last call on this host thread (informational). */
typedef struct {
    int64_t ndc;             /* distance evaluations of the beam searches (stage a + reach fix) */
    int64_t hops;            /* beam-search expansions */
    int64_t join_pairs;      /* cross-graph pairs evaluated by Update */
    int64_t proposals;       /* list insertions proposed by Update (after filtering) */
    int64_t zero_indegree;   /* zero-indegree vertices met by the last indegree repair */
    int64_t repaired;        /* replacements made by the indegree repairs */
    int64_t attached;        /* vertices attached by the reachability fix */
    int64_t unreached;       /* vertices still unreached after the fix */
    int64_t join_reruns;     /* Update passes re-run after a proposal-buffer overflow */
    int64_t join_cands;      /* candidate-set sizes |C_n| + |C_o| summed over the vertices joined */
    int64_t join_class[5];   /* vertices joined per Update form: tensor-core tile for |C| <= 64, <= 128,
                                > 128, the FP32 SIMT tile, and one warp per vertex (few new
                                candidates, byte rows) */
} fgim_stats;

/*
 * Full merge (Sec. 3.3): stage a, then `iters` x (Visit + Update + indegree repair),
 * then Alg. 5 and, if params->ensure_reachable, the reachability fix.
 * shards: host array of h descriptors (2 <= h <= FGIM_MAX_SHARDS). The shards' vector
 *   arrays may live anywhere on the device; when they are consecutive in one buffer
 *   (shard i+1 starts right after shard i) no copy is made.
 * knng_out: optional (NULL = internal); receives the refined k-NNG (n = sum n_i, k).
 * out: receives the merged PG (n = sum n_i, R = params->R) and its entry point, the
 *   entry of the largest input shard (lowest shard index on ties) mapped by phi.
 */
fgim_status fgim_merge(const fgim_shard* shards, int32_t h, const fgim_params* params,
                       fgim_knng* knng_out, fgim_graph* out, void* stream);

/*
 * n_merges independent merges with the same params (the batched form of the measurement
 * plan: many small merges of uneven size, e.g. one per tenant or time window). Merge m takes
 * the h[m] shard descriptors shards[m] and writes outs[m] (n = sum of its shard sizes, R =
 * params->R); no k-NNG is returned. The batch runs as one problem over the disjoint union of
 * the merges' vertices: every stage's kernels run once for all merges (the cross query of a
 * vertex searches its own merge's other shards with its merge's L; the reachability fix works
 * from every merge's entry), and each output equals what fgim_merge gives that merge alone.
 * This needs at most 512 shards in all and no validity masks; otherwise the merges run one
 * after another on the stream (same results), stopping at the first failing merge (earlier
 * outputs complete, later ones untouched). Scratch is sized for the whole batch.
 * fgim_last_stats() holds the counters of the batch.
 */
fgim_status fgim_merge_batch(const fgim_shard* const* shards, const int32_t* h, int32_t n_merges,
                             const fgim_params* params, fgim_graph* outs, void* stream);

/*
 * Same merge from and to HOST memory: copies the vectors and graphs in, merges, copies
 * the merged PG back. vectors_host: [sum n_i, dim] (shards consecutive in phi order);
 * adj_host: [sum n_i, max_degree] local ids; sizes/entries: [h]. out_ids_host [N, R],
 * out_deg_host [N], out_entry_host [1]. Host buffers should be pinned for full speed.
 */
fgim_status fgim_merge_host(const void* vectors_host, const int32_t* adj_host, const int32_t* sizes,
                            const int32_t* entries, int32_t h, int32_t max_degree, const fgim_params* params,
                            int32_t* out_ids_host, int32_t* out_deg_host, int32_t* out_entry_host, void* stream);

/* Stage (a), Alg. 2: PGs -> k-NNG by cross querying. out: [N, k], all flags new. */
fgim_status fgim_cross_query(const fgim_shard* shards, int32_t h, const fgim_params* params,
                             fgim_knng* out, void* stream);

/*
 * One pass of Alg. 3's Visit + Update, in place on `knng` (synchronous form: every
 * candidate set is built from the lists as they stand when the pass starts, and each
 * list ends as the top-k of its entries and all proposals, duplicates by id removed).
 */
fgim_status fgim_refine_pass(const fgim_shard* shards, int32_t h, const fgim_params* params,
                             fgim_knng* knng, void* stream);

/* Alg. 4 in place on `knng`; T_out (optional, [N]) receives the indegree recorder. */
fgim_status fgim_indegree_repair(const fgim_shard* shards, int32_t h, const fgim_params* params,
                                 fgim_knng* knng, int32_t* T_out, void* stream);

/*
 * Alg. 5 neighbour selection: keep v when T(v) = 1 or no kept w occludes it under
 * params->prune_rule (alpha-RNG: delta(u,v) < alpha^2 delta(w,v) for every kept w); stop at R.
 * e_ids/e_dist [N, R] (-1 / +inf padded), e_cnt [N].
 */
fgim_status fgim_prune(const fgim_shard* shards, int32_t h, const fgim_params* params,
                       const fgim_knng* knng, const int32_t* T, int32_t* e_ids, float* e_dist,
                       int32_t* e_cnt, void* stream);

/* Alg. 5 connectivity enhancement: out(u) = top-R of E'(u) U {v : u in E'(v)}. */
fgim_status fgim_reverse_insert(int64_t n, int32_t R, const int32_t* e_ids, const float* e_dist,
                                const int32_t* e_cnt, fgim_graph* out, void* stream);

/* Reachability fix in place on `graph` (graph->entry is read, not written). */
fgim_status fgim_reach_fix(const fgim_shard* shards, int32_t h, const fgim_params* params,
                           fgim_graph* graph, void* stream);

/*
 * Alg. 1 over a merged graph for nq queries: pool `beam` (<= FGIM_MAX_L), returns the
 * first `topk` (<= beam) results. base: [n, dim] vectors in global-id order; base and
 * queries are both in `dtype` (BF16 ones are decoded into FP32 scratch first).
 */
fgim_status fgim_search(const void* base, int64_t n, int32_t dim, int32_t dtype, int32_t metric,
                        const int32_t* graph_ids, int32_t R, int32_t entry, const void* queries, int32_t nq,
                        int32_t topk, int32_t beam, int32_t* out_ids, float* out_dist, void* stream);

/*
 * fgim_search for callers that cannot allocate device memory while they run: processes
 * whose device memory belongs to a pool they do not control, latency-critical paths where
 * an allocation (and the synchronisation it may bring) is not allowed, plug-ins inside a
 * host that forbids allocator calls. Same arguments and results as fgim_search for FP32
 * vectors; dtype must be FGIM_F32 (BF16 storage would need a decoded copy, which is an
 * allocation: it returns FGIM_EUNSUPPORTED). The paper has no counterpart (this is a
 * deployment variant of the evaluation search).
 * Its scratch (status word, counters and, for cosine, the inverse norms of the base and of
 * the queries) lives in one fixed device array inside the library, kept on every device
 * that loads the library until the process exits. Limits: cosine search accepts at most
 * 1,048,576 base vectors and 65,536 queries (larger calls return FGIM_EINVAL); the other
 * metrics have no extra limit. The first call on a device looks the array's address up
 * (cudaGetSymbolAddress): make that first call before any stream capture. All calls share
 * the array, so calls that overlap on the GPU race and must be serialised by the caller.
 * Calls no allocator (no cudaMalloc, cudaMallocAsync, cudaFree, no host allocation) as long
 * as launch profiling is off; errors are returned as status codes only (fgim_last_error()
 * is not updated).
 */
fgim_status fgim_search_noalloc(const void* base, int64_t n, int32_t dim, int32_t dtype, int32_t metric,
                                const int32_t* graph_ids, int32_t R, int32_t entry, const void* queries, int32_t nq,
                                int32_t topk, int32_t beam, int32_t* out_ids, float* out_dist, void* stream);

/* ---- HNSW-adaptive merging (Sec. 4.3.3): upper layers over a merged base graph ----------
 * Every vertex v draws a level with P(level >= l) = M^-l (HNSW's mL = 1 / ln M): r_v = the
 * v-th output of SplitMix64 started from `seed`, level = #{l >= 1 : r_v < floor((2^64 - 1) /
 * M^l)}. Layer l holds the vertices of level >= l (ascending ids). Each layer is built from
 * its own vertices at once (the paper inserts them one at a time, which a GPU cannot do in a
 * fixed order in parallel): the exact `ef` nearest members among those with smaller ids
 * (the members inserted before it, in id order), the RNG heuristic down to M
 * (Alg. 5's rule with alpha = 1 and no indegree clause), bidirectional edges, and the
 * heuristic again over the union of a member's own and reverse edges (the 128 nearest of it
 * when larger). The search goes down from the entry (the first vertex of the highest level)
 * layer by layer, then runs Alg. 1 on the base graph from the vertex it reached. */
#define FGIM_MAX_LEVELS 16

typedef struct {
    const int32_t* members;  /* [n] ascending global ids of the layer's vertices */
    const int32_t* adj;      /* [n, M] neighbours as positions in members, -1 padded */
    int64_t n;
    int32_t M;
    int32_t reserved;
} fgim_layer;

/* levels: device [n] out. counts: HOST [FGIM_MAX_LEVELS + 1] out, counts[l] = #{v : level(v)
 * >= l} (counts[0] = n). M in [2, 128]. Synchronous. */
fgim_status fgim_hnsw_levels(int64_t n, int32_t M, uint64_t seed, int32_t* levels, int64_t* counts, void* stream);

/* One upper layer `level` (1 .. FGIM_MAX_LEVELS) over `vectors` ([n, dim], dtype, metric) and
 * `levels` (device [n]); n_layer = counts[level] of fgim_hnsw_levels. Outputs (device,
 * caller-owned): members [n_layer], adj [n_layer, M] (positions in members, -1 padded),
 * deg [n_layer]. M in [1, 64], ef in [1, 128]. Synchronous. */
fgim_status fgim_hnsw_layer(const void* vectors, int64_t n, int32_t dim, int32_t dtype, int32_t metric,
                            const int32_t* levels, int32_t level, int32_t M, int32_t ef, int32_t* members,
                            int32_t* adj, int32_t* deg, int64_t n_layer, void* stream);

/* fgim_search with the upper layers: layers[l - 1] is layer l (host array of n_layers
 * descriptors, device buffers); entry: the top vertex. From the top, each layer is searched
 * with Alg. 1 (pool ef_up in [1, 128]; 1 = HNSW's greedy descent) from the vertex the layer
 * above gave, and its nearest result starts the next; the base graph is then searched with
 * pool `beam`. out_start (optional, device [nq]): the base-graph vertex each query started from. */
fgim_status fgim_search_hnsw(const void* base, int64_t n, int32_t dim, int32_t dtype, int32_t metric,
                             const int32_t* graph_ids, int32_t R, const fgim_layer* layers, int32_t n_layers,
                             int32_t entry, const void* queries, int32_t nq, int32_t topk, int32_t beam, int32_t ef_up,
                             int32_t* out_ids, float* out_dist, int32_t* out_start, void* stream);

/* An input PG for one shard on the GPU (the input side of a merge; the recipe of the synthetic
 * workloads' input indexes): the medoid (the row nearest, in FP64 squared L2, to the FP64 mean of
 * the rows, lowest id on ties) first, then the other rows in id order, inserted in batches of
 * min(max(c / 2, 1), 1024) rows once c are in. Each row of a batch runs Alg. 1 (pool ef, from the
 * medoid) over the graph as it stood when the batch started and keeps up to M results with
 * HNSW's heuristic (drop a candidate when a kept one is strictly nearer to it than the row:
 * FGIM_PRUNE_MRNG without the indegree clause); then each vertex that received edges takes its
 * list and the new edges in ascending (distance, id), all of them when at most M, else the
 * heuristic's M. adj [n, M] (local ids, -1 padded) and deg [n]: device, caller-owned; entry_out
 * (host): the medoid. M in [1, 128], ef in [1, 128]. Synchronous. */
fgim_status fgim_build_pg(const void* vectors, int64_t n, int32_t dim, int32_t dtype, int32_t metric, int32_t M,
                          int32_t ef, int32_t* adj, int32_t* deg, int32_t* entry_out, void* stream);

/* Counters of the last merge/search call made by this host thread. */
void fgim_last_stats(fgim_stats* out);

/*
 * Scratch memory: every call takes its scratch from a stream-ordered pool the library keeps
 * per device, and the pool keeps what it has mapped for later calls (a merge of 1M vectors
 * uses about 10 GB). This returns the pool's unused memory to the device; call it when no
 * call of this library has work in flight.
 */
void fgim_trim_memory(void);

/*
 * Test hooks: knobs that let a test drive rarely taken paths on small inputs, without
 * faulting or hanging the GPU. They are process-wide, default to off, and are not meant
 * for production use. fgim_test_set returns 1 when the knob exists (and sets it), else 0.
 *   "prop_cap"          > 0: capacity of Update's proposal buffer, in proposals (raised to
 *                       what one vertex can propose), so that small inputs overflow it and
 *                       take the re-run path; 0 = the default size.
 *   "hop_budget"        > 0: expansions each beam search may take; a search that needs more
 *                       stops and the call returns FGIM_ETIMEOUT; 0 = unbounded (default).
 *   "batch_union"       0: fgim_merge_batch runs its merges one after another instead of as
 *                       one problem (same results; for comparing the two); 1 = default.
 *   "join_sparse_nn"    >= 0: Update joins the vertices with at most this many new candidates
 *                       (and at most 128 candidates) one warp per vertex on byte rows, the
 *                       rest in the tensor-core tile (same results; 0 = never, a large value =
 *                       every eligible vertex); -1 = the default cut-off (10).
 *   "fail_alloc_after"  >= 0: the scratch allocation of a call that comes after this many
 *                       successful ones fails as if the device were out of memory (the call
 *                       returns FGIM_ENOMEM); -1 = off (default).
 * fgim_test_get("pool_used_bytes"): bytes of the current device's scratch pool handed out
 * and not yet handed back (0 whenever no call is running); fgim_test_get("scratch_allocs"):
 * scratch allocations made by the last call on this host thread; -1 for an unknown name.
 */
int32_t fgim_test_set(const char* knob, int64_t value);
int64_t fgim_test_get(const char* what);

/*
 * Autotuner of the launch shapes that change no result: the warps per block of the beam-search
 * kernels (the cross query of stage (a), the evaluation and reachability searches) and the size
 * of their visited table (a bigger table costs shared memory per warp, and so resident warps,
 * and saves re-evaluations of forgotten ids). fgim_autotune times every candidate shape (1, 2 or
 * 4 warps per block; the default table size, two steps smaller and one larger) on this merge's cross query
 * with CUDA events (one warm-up, best of two), keeps the fastest for this workload's key (metric,
 * bytes per coordinate read, dim, pool L, SM count of the current device) for the rest of the
 * process, appends it as a JSON line to cache_path (NULL: no file), and returns it (out pointers
 * optional: warps per block, table bits, milliseconds). Call it when no other call of this
 * library is running. fgim_autotune_load reads such a file (a later line for a key wins;
 * FGIM_EINVAL when nothing could be read); fgim_autotune_clear forgets every tuned shape.
 */
fgim_status fgim_autotune(const fgim_shard* shards, int32_t h, const fgim_params* params, const char* cache_path,
                          int32_t* out_wpb, int32_t* out_ht_bits, float* out_ms, void* stream);
fgim_status fgim_autotune_load(const char* cache_path);
void fgim_autotune_clear(void);

/* Human-readable name of a status; message of the last CUDA error on this host thread. */
const char* fgim_strerror(fgim_status s);
const char* fgim_last_error(void);

/* Library version string. */
const char* fgim_version(void);

/*
 * Launch accounting: number of kernels this library has launched since load (all
 * threads). With profiling enabled, every launch is bracketed by CUDA events on its
 * stream and the per-kernel event times are accumulated (fgim_prof_query, milliseconds).
 */
int64_t fgim_launch_count(void);
void fgim_prof_enable(int32_t on);
void fgim_prof_reset(void);
int32_t fgim_prof_query(const char* kernel, int64_t* launches, double* total_ms);
/* Comma-separated names of the kernels timed since the last reset; returns the full length. */
int32_t fgim_prof_names(char* buf, int32_t buf_bytes);

#ifdef __cplusplus
}
#endif
#endif /* FGIM_H */
