// Host-side launchers of the FGIM kernels (one declaration per kernel family).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fgim_internal.cuh"

namespace fgim {

// ---- k_search.cu
// X: FP32 rows; X8: the same rows as bytes when every coordinate is an integer in [0, 255]
// (searches then read X8, with identical results), else nullptr
// phi / src (optional): the ID mapping with invalid vertices; nq = the number of output rows
// (valid vertices), src[r] = the input row of output row r, phi maps input rows to output ids
// (-1 = dropped)
cudaError_t launch_cross_query(const ShardTable& t, const float* X, const uint8_t* X8, const float* inv_norm,
                               long long N, int metric, int k, int L, fgim_knng* out, unsigned long long* counters,
                               int* status, cudaStream_t s, const int32_t* phi = nullptr,
                               const int32_t* src = nullptr, long long nq = -1, const uint16_t* Xh = nullptr);
cudaError_t launch_search(const float* X, const uint8_t* X8, const float* inv_norm, long long n, int d, int metric,
                          const int32_t* graph, int R, int entry, const float* Q, const float* q_inv,
                          const int32_t* qids, long long nq, int topk, int L, int32_t* out_ids, float* out_dist,
                          unsigned long long* counters, int* status, cudaStream_t s, const uint16_t* Xh = nullptr,
                          const int32_t* qentry = nullptr);
// X8[i] = X[i] as a byte; *flag |= 1 unless every X[i] is an integer in [0, 255] (n_elems % 4 == 0)
cudaError_t launch_narrow_u8(const float* X, long long n_elems, uint8_t* X8, int* flag, cudaStream_t s);

// ---- k_util.cu
// exclusive scan of n int32 counts into n + 1 int64 offsets (out[n] = total)
cudaError_t scan_counts(const int32_t* in, long long n, long long* out, void* scratch, size_t scratch_bytes,
                        cudaStream_t s);
size_t scan_scratch_bytes(long long n);
cudaError_t launch_inv_norms(const float* X, long long n, int d, float* inv, cudaStream_t s);
// out[i] = the FP32 value of the bfloat16 encoding in[i]
cudaError_t launch_bf16_to_f32(const uint16_t* in, long long n, float* out, cudaStream_t s);
// flag[i] = (mask == nullptr || mask[i] != 0)
cudaError_t launch_valid_flags(const uint8_t* mask, long long n, int32_t* flag, cudaStream_t s);
// phi[i] = flag[i] ? off[i] : -1 (off = exclusive prefix sums of flag)
cudaError_t launch_phi(const int32_t* flag, const long long* off, long long n, int32_t* phi, cudaStream_t s);
// out[r] = X[src[r]] for r < nv (rows of d floats)
cudaError_t launch_gather_rows(const float* X, const int32_t* src, long long nv, int d, float* out, cudaStream_t s);
cudaError_t launch_fill_i32(int32_t* p, long long n, int32_t v, cudaStream_t s);
// indices i (ascending) with flag[i] != 0, written to out; count to *count (device)
cudaError_t compact_flags(const int32_t* flag, long long n, int32_t* out, long long* offsets_scratch,
                          void* scan_scratch, size_t scan_bytes, cudaStream_t s);

// ---- k_refine.cu
struct RefineBuffers {
    // reverse lists
    int32_t* cntN;
    int32_t* cntO;
    long long* offN;
    long long* offO;
    int32_t* fillN;
    int32_t* fillO;
    uint64_t* revN;
    uint64_t* revO;
    long long rev_capacity;   // entries of revN / revO (N * k each)
    int32_t* topN;            // [N, rev_cap]
    int32_t* topO;
    int32_t* ntopN;
    int32_t* ntopO;
    // candidate sets
    int32_t* cand;            // [N, cmax]
    int32_t* nn;
    int32_t* no;
    int cmax;
    // proposals
    int32_t* prop_tgt;
    uint64_t* prop_key;
    long long prop_cap;
    unsigned long long* prop_count;   // device counter
    uint64_t* prop_sorted;
    int32_t* pcnt;
    long long* poff;
    int32_t* pfill;
    uint8_t* pending;
    int32_t* pend_flag;
    int32_t* pend_list;
    long long* pend_off;
    // scan scratch
    void* scan_tmp;
    size_t scan_bytes;
    // largest candidate set and C_n of a pass and the three launch lists' sizes and largest
    // sets (device, 8 ints), a pinned host slot to read them, and the launch lists (3 x cap)
    int32_t* max_nc;
    int32_t* host_i32;
    long long class_count[5];   // out of refine_join: vertices per form (TC <= 64, <= 128, > 128; FP32 tile;
                                // warp per vertex)
    uint64_t* wk;               // worst key of every list (filled by refine_join for the Update launches)
    int sparse_nn;              // vertices with |C_n| <= sparse_nn (and |C| <= 128) join one warp each
                                // (byte rows; 0: never)
    bool fp8;                   // Xb holds E4M3 rows with per-vector scales (tcm.w) instead of BF16 rows
    int32_t* blist;
    long long blist_cap;
    // tensor-core filter inputs: BF16 copy of the vectors and per row (|x|^2, bound on |x|,
    // bound on the BF16 conversion error |bf(x) - x|, unused)
    int join_filter;
    void* Xb;
    float4* tcm;
    // the vectors as bytes when every coordinate is an integer in [0, 255], else nullptr
    const uint8_t* X8;
};

cudaError_t refine_visit(const fgim_knng& g, int rev_cap, RefineBuffers& b, cudaStream_t s);
cudaError_t refine_join(const ShardTable& t, const float* X, const float* inv_norm, int metric, const fgim_knng& g,
                        RefineBuffers& b, const int32_t* vlist, long long nv, unsigned long long* pairs,
                        unsigned long long* cands, int* status, cudaStream_t s);
cudaError_t refine_merge(const fgim_knng& g, RefineBuffers& b, long long nprop, cudaStream_t s);
cudaError_t launch_prep_fp8(const float* X, long long N, int d, uint8_t* Xq, float4* tcm, cudaStream_t s);
// *out = some adjacency row of the input graphs repeats an id within a 32-entry chunk (uses
// status[2] as scratch; synchronizes the stream)
cudaError_t adjacency_has_repeats(const ShardTable& t, long long N, int* status, cudaStream_t s, bool* out);
cudaError_t launch_prep_bf16(const float* X, long long N, int d, __nv_bfloat16* Xb, float4* tcm, cudaStream_t s);
cudaError_t launch_indegree(const int32_t* ids, long long N, int k, int32_t* T, bool clear_replaced, uint8_t* flags,
                            cudaStream_t s);
// rounds rho0 .. rho0 + rounds - 1 of the Alg. 4 repair; ff[rho0 - 1] holds the first pending
// index, ff[rho] the first index after round rho
constexpr int kRepairWindow = 2048;
cudaError_t launch_repair_rounds(fgim_knng& g, int32_t* T, const int32_t* zeros, long long nz, long long rho0,
                                 int rounds, long long* ff, unsigned long long* owner, unsigned long long* repaired,
                                 int* status, cudaStream_t s);
cudaError_t launch_zero_flags(const int32_t* T, long long N, int32_t* flag, cudaStream_t s);
cudaError_t launch_nonzero_flags(const uint8_t* v, long long N, int32_t* flag, cudaStream_t s);

// ---- k_prune.cu
// Alg. 5 neighbour selection of the g.n lists of g (ids in 0 .. N - 1, rows of X) with `rule`
cudaError_t launch_prune(const float* X, const uint8_t* X8, const float* inv_norm, long long N, int d, int metric,
                         const fgim_knng& g, const int32_t* T, int R, PruneRule rule, int32_t* e_ids, float* e_dist,
                         int32_t* e_cnt, int* status, cudaStream_t s);
struct ReverseBuffers {
    int32_t* cnt;
    long long* off;
    int32_t* fill;
    uint64_t* rev;
    void* scan_tmp;
    size_t scan_bytes;
};
cudaError_t launch_reverse_insert(long long N, int R, const int32_t* e_ids, const float* e_dist, const int32_t* e_cnt,
                                  ReverseBuffers& b, int32_t* out_ids, float* out_dist, int32_t* out_deg,
                                  cudaStream_t s);
// reachability fix helpers
cudaError_t launch_bfs_init(int32_t* visited, long long N, int32_t* frontier, int32_t* st, int entry,
                            cudaStream_t s);
// the same from the ne sources entries[] (device)
cudaError_t launch_bfs_init_multi(int32_t* visited, long long N, int32_t* frontier, int32_t* st,
                                  const int32_t* entries, int ne, int* status, cudaStream_t s);
// batches run as one problem: start[r] = entries[m] of the merge m (id range off[m] .. off[m+1]-1)
// holding reps[r]; the rows of one merge copied out of the union graph, ids minus base
cudaError_t launch_rep_starts(const int32_t* reps, long long nr, const long long* off, const int32_t* entries, int nm,
                              int32_t* start, cudaStream_t s);
cudaError_t launch_split_rows(const int32_t* ids, const float* dist, const int32_t* deg, long long n, int R,
                              int32_t base, int32_t* out_ids, float* out_dist, int32_t* out_deg, cudaStream_t s);
// BFS levels level0 .. level0 + levels - 1 (state st: 8 ints, see k_prune.cu; level 1 reads fa)
cudaError_t launch_bfs_levels(const int32_t* graph, int R, long long N, int32_t* visited, int32_t* fa, int32_t* fb,
                              int32_t* st, int level0, int levels, cudaStream_t s);
cudaError_t launch_bfs_parents(const int32_t* graph, int R, long long N, const int32_t* level, int32_t* npar,
                               cudaStream_t s);
cudaError_t launch_cc_init(const int32_t* visited, long long N, int32_t* label, cudaStream_t s);
cudaError_t launch_cc_step(const int32_t* graph, int R, long long N, const int32_t* visited, int32_t* label,
                           int32_t* changed, cudaStream_t s);
cudaError_t launch_rep_flags(const int32_t* visited, const int32_t* label, long long N, int32_t* flag,
                             cudaStream_t s);
// `rounds` rounds of the representative attachment (rounds rho0 .. rho0 + rounds - 1) in one
// cooperative launch; ff[rho0 - 1] holds the first pending index, ff[rho] the first index
// after round rho; plan: scratch of kReachWindow entries
constexpr int kReachWindow = 2048;
cudaError_t launch_reach_rounds(int32_t* graph, float* gdist, int32_t* deg, const int32_t* level, int32_t* npar,
                                int R, const int32_t* reps, long long nr, long long rho0, int rounds, long long* ff,
                                const int32_t* cand, const float* cdist, int beam, unsigned long long* owner,
                                int4* plan, unsigned long long* attached, cudaStream_t s);

// ---- k_hnsw.cu (HNSW-adaptive merging, Sec. 4.3.3)
constexpr int kMaxHnswLevels = 16;
struct HnswThresholds {   // T_l = floor((2^64 - 1) / M^l), l = 1 .. count
    int count;
    unsigned long long t[kMaxHnswLevels];
};
cudaError_t launch_hnsw_levels(long long n, unsigned long long seed, const HnswThresholds& th, int32_t* levels,
                               cudaStream_t s);
// flag[v] = levels[v] >= level
cudaError_t launch_level_flags(const int32_t* levels, long long n, int level, int32_t* flag, cudaStream_t s);
// rows of width M into rows of width w (padding -1 / +inf)
cudaError_t launch_widen(const int32_t* ids, const float* dist, long long n, int M, int w, int32_t* oids, float* odist,
                         cudaStream_t s);
// the kk nearest rows of every row of Xl among the rows before it (n rows, FP32; X8l: the same
// as bytes or nullptr)
cudaError_t launch_layer_knn(const float* Xl, const uint8_t* X8l, const float* inv, long long n, int d, int metric,
                             int kk, int32_t* out_ids, float* out_dist, cudaStream_t s);
// hand-over between layer searches: best (positions in mem) -> qpos (positions in next) or,
// with next == nullptr, start (global ids); first: every query starts at entry's position
cudaError_t launch_hnsw_next(const int32_t* best, const int32_t* mem, long long nmem, const int32_t* next,
                             long long nnext, long long nq, int first, int entry, int32_t* qpos, int32_t* start,
                             int* status, cudaStream_t s);

// ---- k_pgbuild.cu: input PGs by batch-incremental insertion (see the file comment)
cudaError_t launch_pg_medoid(const float* X, long long n, int d, double* mean, unsigned long long* dist_bits,
                             unsigned long long* best, int* medoid, cudaStream_t s);
cudaError_t launch_pg_init(long long n, int M, const int* medoid, int32_t* order, int32_t* nbr, float* nd, int32_t* cnt,
                           int32_t* zeros, cudaStream_t s);
cudaError_t launch_pg_install(const int32_t* rows, long long b, int M, const int32_t* e_ids, const float* e_dist,
                              const int32_t* e_cnt, int32_t* nbr, float* nd, int32_t* cnt, int32_t* cin,
                              cudaStream_t s);
cudaError_t launch_pg_rev_fill(const int32_t* rows, long long b, int M, const int32_t* e_ids, const float* e_dist,
                               const int32_t* e_cnt, const long long* off, int32_t* fill, uint64_t* rev,
                               cudaStream_t s);
cudaError_t launch_pg_rev_merge(const int32_t* targets, long long nt, const long long* off, const uint64_t* rev, int M,
                                int W, int32_t* nbr, float* nd, int32_t* cnt, int32_t* ov_ids, float* ov_dist,
                                int32_t* ov_tgt, int* n_ov, cudaStream_t s);
cudaError_t launch_pg_write_back(const int32_t* ov_tgt, long long nov, int M, const int32_t* e_ids, const float* e_dist,
                                 const int32_t* e_cnt, int32_t* nbr, float* nd, int32_t* cnt, cudaStream_t s);
cudaError_t launch_pos_flags(const int32_t* c, long long n, int32_t* flag, cudaStream_t s);

// ---- fgim_abi.cu: launch shapes chosen by the autotuner (fgim_autotune)
// Beam-search kernels (cross query, searches): warps per block and visited-table bits, keyed by
// (metric, bytes per coordinate read, dim, pool L) on the current device; untuned keys keep the
// defaults passed in. Neither changes a result (the visited table may only forget ids).
unsigned long long beam_shape_key(int metric, int row_bytes, int dim, int L);
void tuned_beam_shape(unsigned long long key, int* wpb, int* htbits);

}  // namespace fgim
