// Input proximity graphs on the GPU: the batch-incremental insertion the synthetic workloads use
// for their input indexes (one flat HNSW-style graph per shard), built from the library's own
// Alg. 1 search and neighbour-selection kernels.
//
// The insertion order starts with the medoid (the row nearest, in FP64 squared L2, to the FP64
// mean of the rows; the lowest id on ties), then every other row in id order. Rows are inserted
// in batches of b = min(max(c / 2, 1), 1024) rows once c rows are in: every row of a batch
// searches the graph as it stood when the batch started (Alg. 1 from the medoid with pool ef,
// the same search HNSW's two-heap layer search performs), keeps up to M of the results with
// HNSW's heuristic (a candidate is dropped when a kept one is strictly nearer to it than the
// inserted row: the MRNG rule, no indegree clause), and gets that list; then every vertex that
// received reverse edges takes its list and the new edges, in ascending (distance, id), keeps
// all of them when they are at most M and otherwise the heuristic's M. The mean and the medoid
// distances are summed in the same sequential FP64 order as a plain loop, so the medoid is that
// of the plain loop bit for bit.
#include "fgim_launch.h"

namespace fgim {

static inline long long cdivp(long long a, long long b) { return (a + b - 1) / b; }

// mean[t] = (sum over rows i, in order, of X[i][t]) / n, in FP64 (one thread per dimension)
__global__ void k_col_mean(const float* __restrict__ X, long long n, int d, double* __restrict__ mean) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d) return;
    double s = 0.0;
    for (long long i = 0; i < n; ++i) s = __dadd_rn(s, (double)X[i * d + t]);
    mean[t] = __ddiv_rn(s, (double)n);
}

// squared FP64 distance of every row to the mean (sequential over the dimensions), the smallest
// one's bits (non-negative doubles order like their bits) folded into *best
__global__ void k_medoid_dist(const float* __restrict__ X, long long n, int d, const double* __restrict__ mean,
                              unsigned long long* __restrict__ dist_bits, unsigned long long* best) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a = 0.0;
    for (int t = 0; t < d; ++t) {
        const double z = __dsub_rn((double)X[i * d + t], mean[t]);
        a = __dadd_rn(a, __dmul_rn(z, z));
    }
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    dist_bits[i] = b;
    atomicMin(best, b);
}

// the lowest row at the smallest distance
__global__ void k_medoid_pick(const unsigned long long* __restrict__ dist_bits, long long n,
                              const unsigned long long* best, int* medoid) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && dist_bits[i] == *best) atomicMin(medoid, (int)i);
}

// insertion order: the medoid, then every other row in id order; and the empty graph
__global__ void k_pg_init(long long n, int M, const int* medoid, int32_t* __restrict__ order,
                          int32_t* __restrict__ nbr, float* __restrict__ nd, int32_t* __restrict__ cnt,
                          int32_t* __restrict__ zeros) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int m = *medoid;
    if (i < n) {
        order[i] = i == 0 ? m : (i - 1 < m ? (int32_t)(i - 1) : (int32_t)i);
        cnt[i] = 0;
        zeros[i] = 0;
    }
    if (i < n * M) {
        nbr[i] = -1;
        nd[i] = __int_as_float(0x7f800000);
    }
}

// the batch's lists go in; their entries become reverse-edge candidates of their targets
__global__ void k_pg_install(const int32_t* __restrict__ rows, long long b, int M, const int32_t* __restrict__ e_ids,
                             const float* __restrict__ e_dist, const int32_t* __restrict__ e_cnt,
                             int32_t* __restrict__ nbr, float* __restrict__ nd, int32_t* __restrict__ cnt,
                             int32_t* __restrict__ cin) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b * M) return;
    const long long bi = i / M;
    const int t = (int)(i - bi * M);
    const int32_t p = rows[bi];
    const int c = e_cnt[bi];
    if (t == 0) cnt[p] = c;
    nbr[(long long)p * M + t] = t < c ? e_ids[i] : -1;
    nd[(long long)p * M + t] = t < c ? e_dist[i] : __int_as_float(0x7f800000);
    if (t < c) atomicAdd(cin + e_ids[i], 1);
}

__global__ void k_pg_rev_fill(const int32_t* __restrict__ rows, long long b, int M, const int32_t* __restrict__ e_ids,
                              const float* __restrict__ e_dist, const int32_t* __restrict__ e_cnt,
                              const long long* __restrict__ off, int32_t* __restrict__ fill,
                              uint64_t* __restrict__ rev) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b * M) return;
    const long long bi = i / M;
    const int t = (int)(i - bi * M);
    if (t >= e_cnt[bi]) return;
    const int32_t v = e_ids[i];
    rev[off[v] + atomicAdd(fill + v, 1)] = mkkey(e_dist[i], rows[bi]);
}

// Per target v (warp per target): its list and its new reverse edges in ascending (distance, id);
// at most M of them stay as they are, more go to the overflow lists for the heuristic.
__global__ void __launch_bounds__(128) k_pg_rev_merge(const int32_t* __restrict__ targets, long long nt,
                                                      const long long* __restrict__ off,
                                                      const uint64_t* __restrict__ rev, int M, int W,
                                                      int32_t* __restrict__ nbr, float* __restrict__ nd,
                                                      int32_t* __restrict__ cnt, int32_t* __restrict__ ov_ids,
                                                      float* __restrict__ ov_dist, int32_t* __restrict__ ov_tgt,
                                                      int* __restrict__ n_ov) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const long long ti = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (ti >= nt) return;
    const int32_t v = targets[ti];
    uint64_t* list = reinterpret_cast<uint64_t*>(smem) + (size_t)warp * W;
    const int c0 = cnt[v];
    int n = 0;
    for (int s0 = 0; s0 < c0; s0 += 32) {
        const uint64_t key = s0 + lane < c0 ? mkkey(nd[(long long)v * M + s0 + lane], nbr[(long long)v * M + s0 + lane])
                                            : kEmptyKey;
        n = warp_merge<false>(list, nullptr, n, W, key, 0);
    }
    const long long b0 = off[v], m = off[v + 1] - off[v];
    for (long long s0 = 0; s0 < m; s0 += 32) {
        const uint64_t key = s0 + lane < m ? rev[b0 + s0 + lane] : kEmptyKey;
        n = warp_merge<false>(list, nullptr, n, W, key, 0);
    }
    if (n <= M) {
        for (int s = lane; s < M; s += 32) {
            nbr[(long long)v * M + s] = s < n ? key_id(list[s]) : -1;
            nd[(long long)v * M + s] = s < n ? key_dist(list[s]) : __int_as_float(0x7f800000);
        }
        if (lane == 0) cnt[v] = n;
        return;
    }
    int slot = 0;
    if (lane == 0) slot = atomicAdd(n_ov, 1);
    slot = __shfl_sync(kFull, slot, 0);
    for (int s = lane; s < W; s += 32) {
        ov_ids[(long long)slot * W + s] = s < n ? key_id(list[s]) : -1;
        ov_dist[(long long)slot * W + s] = s < n ? key_dist(list[s]) : __int_as_float(0x7f800000);
    }
    if (lane == 0) ov_tgt[slot] = v;
}

// the heuristic's lists of the overflowing targets back into the graph
__global__ void k_pg_write_back(const int32_t* __restrict__ ov_tgt, long long nov, int M,
                                const int32_t* __restrict__ e_ids, const float* __restrict__ e_dist,
                                const int32_t* __restrict__ e_cnt, int32_t* __restrict__ nbr, float* __restrict__ nd,
                                int32_t* __restrict__ cnt) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nov * M) return;
    const long long r = i / M;
    const int t = (int)(i - r * M);
    const int32_t v = ov_tgt[r];
    if (t == 0) cnt[v] = e_cnt[r];
    nbr[(long long)v * M + t] = e_ids[i];
    nd[(long long)v * M + t] = e_dist[i];
}

__global__ void k_pos_flags(const int32_t* __restrict__ c, long long n, int32_t* __restrict__ flag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = c[i] > 0 ? 1 : 0;
}

cudaError_t launch_pos_flags(const int32_t* c, long long n, int32_t* flag, cudaStream_t s) {
    LaunchScope ls("k_pos_flags", s);
    k_pos_flags<<<(unsigned)cdivp(n, 256), 256, 0, s>>>(c, n, flag);
    return cudaGetLastError();
}

cudaError_t launch_pg_medoid(const float* X, long long n, int d, double* mean, unsigned long long* dist_bits,
                             unsigned long long* best, int* medoid, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(best, 0xff, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(medoid, 0x7f, sizeof(int), s)) != cudaSuccess) return e;
    {
        LaunchScope ls("k_col_mean", s);
        k_col_mean<<<(unsigned)cdivp(d, 128), 128, 0, s>>>(X, n, d, mean);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        LaunchScope ls("k_medoid_dist", s);
        k_medoid_dist<<<(unsigned)cdivp(n, 256), 256, 0, s>>>(X, n, d, mean, dist_bits, best);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    LaunchScope ls("k_medoid_pick", s);
    k_medoid_pick<<<(unsigned)cdivp(n, 256), 256, 0, s>>>(dist_bits, n, best, medoid);
    return cudaGetLastError();
}

cudaError_t launch_pg_init(long long n, int M, const int* medoid, int32_t* order, int32_t* nbr, float* nd, int32_t* cnt,
                           int32_t* zeros, cudaStream_t s) {
    LaunchScope ls("k_pg_init", s);
    k_pg_init<<<(unsigned)cdivp(n * M, 256), 256, 0, s>>>(n, M, medoid, order, nbr, nd, cnt, zeros);
    return cudaGetLastError();
}

cudaError_t launch_pg_install(const int32_t* rows, long long b, int M, const int32_t* e_ids, const float* e_dist,
                              const int32_t* e_cnt, int32_t* nbr, float* nd, int32_t* cnt, int32_t* cin,
                              cudaStream_t s) {
    LaunchScope ls("k_pg_install", s);
    k_pg_install<<<(unsigned)cdivp(b * M, 256), 256, 0, s>>>(rows, b, M, e_ids, e_dist, e_cnt, nbr, nd, cnt, cin);
    return cudaGetLastError();
}

cudaError_t launch_pg_rev_fill(const int32_t* rows, long long b, int M, const int32_t* e_ids, const float* e_dist,
                               const int32_t* e_cnt, const long long* off, int32_t* fill, uint64_t* rev,
                               cudaStream_t s) {
    LaunchScope ls("k_pg_rev_fill", s);
    k_pg_rev_fill<<<(unsigned)cdivp(b * M, 256), 256, 0, s>>>(rows, b, M, e_ids, e_dist, e_cnt, off, fill, rev);
    return cudaGetLastError();
}

cudaError_t launch_pg_rev_merge(const int32_t* targets, long long nt, const long long* off, const uint64_t* rev, int M,
                                int W, int32_t* nbr, float* nd, int32_t* cnt, int32_t* ov_ids, float* ov_dist,
                                int32_t* ov_tgt, int* n_ov, cudaStream_t s) {
    if (nt <= 0) return cudaSuccess;
    const int wpb = 4;
    const size_t smem = (size_t)wpb * W * 8;
    cudaError_t e = cudaFuncSetAttribute(k_pg_rev_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    LaunchScope ls("k_pg_rev_merge", s);
    k_pg_rev_merge<<<(unsigned)cdivp(nt, wpb), wpb * 32, smem, s>>>(targets, nt, off, rev, M, W, nbr, nd, cnt, ov_ids,
                                                                   ov_dist, ov_tgt, n_ov);
    return cudaGetLastError();
}

cudaError_t launch_pg_write_back(const int32_t* ov_tgt, long long nov, int M, const int32_t* e_ids, const float* e_dist,
                                 const int32_t* e_cnt, int32_t* nbr, float* nd, int32_t* cnt, cudaStream_t s) {
    if (nov <= 0) return cudaSuccess;
    LaunchScope ls("k_pg_write_back", s);
    k_pg_write_back<<<(unsigned)cdivp(nov * M, 256), 256, 0, s>>>(ov_tgt, nov, M, e_ids, e_dist, e_cnt, nbr, nd, cnt);
    return cudaGetLastError();
}

}  // namespace fgim
