// Evaluation and reachability searches (Alg. 1 for batches of queries over one graph) and
// the byte-row check; the beam search itself is in k_beam.cuh.
#include "k_beam.cuh"

namespace fgim {

// Alg. 1 for a batch of queries over one graph with global ids. Queries are rows of Q
// (qids == nullptr) or rows qids[i] of X.
template <int METRIC, bool SMALLD, typename RT, int MAXS>
__global__ void __launch_bounds__(128, sizeof(RT) == 1 ? 8 : 5) k_search(const float* __restrict__ X, const RT* __restrict__ Xr,
                                                const float* __restrict__ inv_norm,
                                                long long n, int d, const int32_t* __restrict__ graph, int R,
                                                int entry, const int32_t* __restrict__ qentry, const float* __restrict__ Q,
                                                const float* __restrict__ q_inv, const int32_t* __restrict__ qids,
                                                long long nq, int topk, int L, int htbits,
                                                int32_t* __restrict__ out_ids, float* __restrict__ out_dist,
                                                unsigned long long* counters, int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const long long qi = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (qi >= nq) return;
    const WarpLayout lay = warp_layout(d, L, htbits, 0, sizeof(RT) != 1);
    unsigned char* base = smem + (size_t)warp * lay.bytes;
    float* q = reinterpret_cast<float*>(base + lay.q);
    uint64_t* pool = reinterpret_cast<uint64_t*>(base + lay.pool);
    uint8_t* pflag = base + lay.pflag;
    int32_t* ht = reinterpret_cast<int32_t*>(base + lay.ht);
    int32_t* scratch = reinterpret_cast<int32_t*>(base + lay.scratch);
    float* P = reinterpret_cast<float*>(base + lay.part);
    const float* qsrc = qids ? X + (long long)qids[qi] * d : Q + qi * d;
    const float4* src = reinterpret_cast<const float4*>(qsrc);
    float4* q4 = reinterpret_cast<float4*>(q);
    for (int c = lane; c < (d >> 2); c += 32) q4[c] = src[c];
    float qinv = 1.f;
    if (METRIC == FGIM_COSINE) qinv = qids ? inv_norm[qids[qi]] : q_inv[qi];
    __syncwarp();
    const float4 qreg = (SMALLD && lane < (d >> 2)) ? q4[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    QBytes qb;
    qb.w = make_uint4(0u, 0u, 0u, 0u);
    qb.q2 = 0u;
    if (sizeof(RT) == 1) qb = query_bytes(q, d, lane);
    WarpCounters ctr;
    const int ent = qentry ? qentry[qi] : entry;   // per-query entries (the HNSW descent's result)
    const int np = beam_search<METRIC, SMALLD, RT, MAXS>(Xr, inv_norm, graph, R, n, ent, 0, q, qreg, qb, qinv, d, L,
                                                         pool, pflag, ht, htbits, scratch, P, ctr, status);
    for (int s = lane; s < topk; s += 32) {
        if (s < np) {
            out_ids[qi * topk + s] = key_id(pool[s]);
            out_dist[qi * topk + s] = key_dist(pool[s]);
        } else {
            out_ids[qi * topk + s] = -1;
            out_dist[qi * topk + s] = __int_as_float(0x7f800000);
        }
    }
    warp_add_counters(ctr, counters);
}

cudaError_t launch_search(const float* X, const uint8_t* X8, const float* inv_norm, long long n, int d, int metric,
                          const int32_t* graph, int R, int entry, const float* Q, const float* q_inv,
                          const int32_t* qids, long long nq, int topk, int L, int32_t* out_ids, float* out_dist,
                          unsigned long long* counters, int* status, cudaStream_t s, const uint16_t* Xh,
                          const int32_t* qentry) {
    const bool bytes = X8 && qids && byte_rows_ok(d);
    const bool bf16 = !bytes && Xh && d > 128 && (reinterpret_cast<uintptr_t>(Xh) & 7u) == 0;
    int htbits = ht_bits_for(L), wpb = 4;   // the autotuner's choice for this workload, if any
    tuned_beam_shape(beam_shape_key(metric, bytes ? 1 : bf16 ? 2 : 4, d, L), &wpb, &htbits);
    const WarpLayout lay = warp_layout(d, L, htbits, 0, !bytes);
    const size_t smem = (size_t)lay.bytes * wpb;
    const long long blocks = (nq + wpb - 1) / wpb;
    if (blocks <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
#define FGIM_LAUNCH_S(MT, SD, RT, MS)                                                                                  \
    do {                                                                                                           \
        e = cudaFuncSetAttribute(k_search<MT, SD, RT, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);   \
        if (e != cudaSuccess) break;                                                                               \
        LaunchScope ls("k_search", s);                                                                             \
        k_search<MT, SD, RT, MS><<<(unsigned)blocks, wpb * 32, smem, s>>>(                                             \
            X, reinterpret_cast<const RT*>(rows), inv_norm, n, d, graph, R, entry, qentry, Q, q_inv, qids, nq, topk, L, \
            htbits, out_ids, out_dist, counters, status);                                                          \
        e = cudaGetLastError();                                                                                    \
    } while (0)
    if (bytes) {   // byte rows need integer queries: rows of X
        const void* rows = X8;
        FGIM_DISPATCH_ALL(metric, d, L, FGIM_LAUNCH_S, uint8_t);
    } else if (bf16) {   // BF16 storage: same values, half the bytes
        const void* rows = Xh;
        FGIM_DISPATCH_ALL_WIDE(metric, L, FGIM_LAUNCH_S, uint16_t);
    } else {
        const void* rows = X;
        FGIM_DISPATCH_ALL(metric, d, L, FGIM_LAUNCH_S, float);
    }
#undef FGIM_LAUNCH_S
    return e;
}

// ---------------------------------------------------------------------------- byte rows
// flag |= 1 unless every coordinate is an integer in [0, 255]; X8 = the coordinates as bytes
__global__ void k_narrow_u8(const float4* __restrict__ X, long long n4, uchar4* __restrict__ X8, int* flag) {
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 v = X[i];
        const float a[4] = {v.x, v.y, v.z, v.w};
        unsigned char b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool ok = a[q] >= 0.f && a[q] <= 255.f && a[q] == truncf(a[q]);
            bad |= !ok;
            b[q] = ok ? (unsigned char)a[q] : 0;
        }
        X8[i] = make_uchar4(b[0], b[1], b[2], b[3]);
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

cudaError_t launch_narrow_u8(const float* X, long long n_elems, uint8_t* X8, int* flag, cudaStream_t s) {
    if (n_elems <= 0) return cudaSuccess;
    LaunchScope ls("k_narrow_u8", s);
    const long long n4 = n_elems / 4;
    const long long blocks = std::min<long long>((n4 + 255) / 256, 152LL * 16);
    k_narrow_u8<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const float4*>(X), n4,
                                                 reinterpret_cast<uchar4*>(X8), flag);
    return cudaGetLastError();
}

}  // namespace fgim
