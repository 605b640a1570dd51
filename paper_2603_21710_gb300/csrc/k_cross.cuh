// Stage (a), Alg. 2 (PGs -> k-NNG): the cross-query kernel and its launcher, a template over
// the ID mapping with invalid vertices (PHI) whose two forms are compiled in k_cross.cu and
// k_cross_phi.cu; the beam search itself is in k_beam.cuh.
#pragma once
#include "k_beam.cuh"

namespace fgim {

// Stage (a), Alg. 2: for every global vertex g (warp per vertex) collect C_i^+(u) from its
// own PG and KNNSearch(x_u, G_j, L, L, ep_j) for every other shard j of its merge (L: the
// merge's pool, at most the launch's L, which sizes shared memory), keep the top-k by
// (delta, id), write ids / distances / new flags. With the ID mapping phi (Sec. 4.1.3) of
// invalid vertices, warp r serves input row rows_of[r]; local candidates and search results are
// renamed by phi and the invalid ones (phi = -1) dropped before the top-k (phi keeps the
// order of ids, so the pool order needs no change).
template <int METRIC, bool SMALLD, typename RT, int MAXS, bool PHI>
__global__ void __launch_bounds__(128, sizeof(RT) == 1 ? 8 : 5) k_cross_query(ShardTable t, const float* __restrict__ X,
                                                     const RT* __restrict__ Xr, const float* __restrict__ inv_norm, long long N, int k, int L,
                                                     int htbits, int32_t* __restrict__ out_ids,
                                                     float* __restrict__ out_dist, uint8_t* __restrict__ out_flags,
                                                     unsigned long long* counters, int* status,
                                                     const int32_t* __restrict__ phi, const int32_t* __restrict__ rows_of,
                                                     long long nq, bool dedupe) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const long long orow = (long long)blockIdx.x * (blockDim.x >> 5) + warp;   // output row
    if (orow >= nq) return;
    const long long g = PHI ? (long long)rows_of[orow] : orow;   // input row
    if (PHI && (g < 0 || g >= N)) {
        if (lane == 0) atomicOr(status, kErrBounds);
        return;
    }
    const int d = t.dim;
    const WarpLayout lay = warp_layout(d, L, htbits, k, sizeof(RT) != 1);
    unsigned char* base = smem + (size_t)warp * lay.bytes;
    float* q = reinterpret_cast<float*>(base + lay.q);
    uint64_t* pool = reinterpret_cast<uint64_t*>(base + lay.pool);
    uint8_t* pflag = base + lay.pflag;
    int32_t* ht = reinterpret_cast<int32_t*>(base + lay.ht);
    uint64_t* res = reinterpret_cast<uint64_t*>(base + lay.res);
    int32_t* scratch = reinterpret_cast<int32_t*>(base + lay.scratch);
    float* P = reinterpret_cast<float*>(base + lay.part);

    const float4* src = reinterpret_cast<const float4*>(X + g * d);
    float4* q4 = reinterpret_cast<float4*>(q);
    for (int c = lane; c < (d >> 2); c += 32) q4[c] = src[c];
    const float qinv = (METRIC == FGIM_COSINE) ? inv_norm[g] : 1.f;
    __syncwarp();
    const float4 qreg = (SMALLD && lane < (d >> 2)) ? q4[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    QBytes qb;
    qb.w = make_uint4(0u, 0u, 0u, 0u);
    qb.q2 = 0u;
    if (sizeof(RT) == 1) qb = query_bytes(q, d, lane);

    WarpCounters ctr;
    const int i = shard_of(t, g);
    const long long u = g - t.off[i];
    const long long ni = t.off[i + 1] - t.off[i];
    int nres = 0;
    // Alg. 2, local candidate neighbours C_i^+(u), mapped to global ids by phi
    const int Mi = t.M[i];
    const int32_t* arow = t.adj[i] + u * Mi;
    for (int c0 = 0; c0 < Mi; c0 += 32) {
        int v = (c0 + lane < Mi) ? arow[c0 + lane] : -1;
        if (v >= ni) {
            atomicOr(status, kErrBounds);
            v = -1;
        }
        if (v == u) v = -1;
        if (PHI && v >= 0 && phi[t.off[i] + v] < 0) v = -1;   // invalid: not a candidate
        const unsigned m = __ballot_sync(kFull, v >= 0);
        const int U = __popc(m);
        if (U == 0) continue;
        if (v >= 0) scratch[__popc(m & lt)] = (int32_t)(t.off[i] + v);
        __syncwarp();
        const float dd = rows_delta<METRIC, SMALLD, RT>(Xr, scratch, U, q, qreg, qb, d, lane, P);
        uint64_t cand = kEmptyKey;
        if (lane < U) {
            const int32_t gv = scratch[lane];
            const float inv = (METRIC == FGIM_COSINE) ? __fmul_rn(qinv, inv_norm[gv]) : 1.f;
            cand = mkkey(delta_finish<METRIC>(dd, inv), PHI ? phi[gv] : gv);
            ctr.ndc++;
        }
        __syncwarp();
        nres = warp_merge<true>(res, nullptr, nres, k, cand, 0);
    }
    // Alg. 2, cross querying of every other index of this vertex's merge, with its pool size
    const int Lq = t.gL[i];
    for (int j = t.grp[i]; j < t.gend[i]; ++j) {
        if (j == i) continue;
        const long long nj = t.off[j + 1] - t.off[j];
        const int np = beam_search<METRIC, SMALLD, RT, MAXS>(Xr + t.off[j] * d,
                                                             inv_norm ? inv_norm + t.off[j] : nullptr, t.adj[j], t.M[j],
                                                             nj, t.entry[j], t.off[j], q, qreg, qb, qinv, d, Lq, pool,
                                                             pflag, ht, htbits, scratch, P, ctr, status, dedupe);
        for (int c0 = 0; c0 < np; c0 += 32) {
            uint64_t cand = (c0 + lane < np) ? pool[c0 + lane] : kEmptyKey;
            if (PHI && cand != kEmptyKey) {
                const int32_t m = phi[key_id(cand)];
                cand = m < 0 ? kEmptyKey : mkkey(key_dist(cand), m);
            }
            nres = warp_merge<false>(res, nullptr, nres, k, cand, 0);
        }
    }
    // Alg. 2, sorted by distance and resized to k
    for (int s = lane; s < k; s += 32) {
        const long long o = (PHI ? orow : g) * k + s;
        if (s < nres) {
            out_ids[o] = key_id(res[s]);
            out_dist[o] = key_dist(res[s]);
            out_flags[o] = FGIM_FLAG_NEW;
        } else {
            out_ids[o] = -1;
            out_dist[o] = __int_as_float(0x7f800000);
            out_flags[o] = 0;
        }
    }
    warp_add_counters(ctr, counters);
}

template <bool PHI>
cudaError_t launch_cross_query_t(const ShardTable& t, const float* X, const uint8_t* X8, const float* inv_norm,
                                 long long N, int metric, int k, int L, fgim_knng* out,
                                 unsigned long long* counters, int* status, cudaStream_t s, const int32_t* phi,
                                 const int32_t* src, long long nq, const uint16_t* Xh) {
    const bool bytes = X8 && byte_rows_ok(t.dim);
    const bool bf16 = !bytes && Xh && t.dim > 128 && (reinterpret_cast<uintptr_t>(Xh) & 7u) == 0;
    int htbits = ht_bits_for(L), wpb = 4;   // the autotuner's choice for this workload, if any
    tuned_beam_shape(beam_shape_key(metric, bytes ? 1 : bf16 ? 2 : 4, t.dim, L), &wpb, &htbits);
    const WarpLayout lay = warp_layout(t.dim, L, htbits, k, !bytes);
    const size_t smem = (size_t)lay.bytes * wpb;
    if (nq < 0) nq = N;
    if ((phi == nullptr) != (src == nullptr)) return cudaErrorInvalidValue;
    const long long blocks = (nq + wpb - 1) / wpb;
    if (blocks <= 0) return cudaSuccess;
    // the searches skip their per-expansion duplicate check when no adjacency row repeats an id
    // within a 32-entry chunk (one pass over the input graphs; the usual case)
    bool dedupe = true;
    cudaError_t e = adjacency_has_repeats(t, N, status, s, &dedupe);
    if (e != cudaSuccess) return e;
#define FGIM_LAUNCH_CQ2(MT, SD, RT, MS, PH)                                                                          \
    do {                                                                                                           \
        e = cudaFuncSetAttribute(k_cross_query<MT, SD, RT, MS, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                 (int)smem);                                                                       \
        if (e != cudaSuccess) break;                                                                               \
        LaunchScope ls("k_cross_query", s);                                                                        \
        k_cross_query<MT, SD, RT, MS, PH><<<(unsigned)blocks, wpb * 32, smem, s>>>(                                    \
            t, X, reinterpret_cast<const RT*>(rows), inv_norm, N, k, L, htbits, out->ids, out->dist, out->flags,   \
            counters, status, phi, src, nq, dedupe);                                                               \
        e = cudaGetLastError();                                                                                    \
    } while (0)
#define FGIM_LAUNCH_CQ(MT, SD, RT, MS) FGIM_LAUNCH_CQ2(MT, SD, RT, MS, PHI)
    if (bytes) {
        const void* rows = X8;
        FGIM_DISPATCH_ALL(metric, t.dim, L, FGIM_LAUNCH_CQ, uint8_t);
    } else if (bf16) {   // BF16 storage: same values, half the bytes
        const void* rows = Xh;
        FGIM_DISPATCH_ALL_WIDE(metric, L, FGIM_LAUNCH_CQ, uint16_t);
    } else {
        const void* rows = X;
        FGIM_DISPATCH_ALL(metric, t.dim, L, FGIM_LAUNCH_CQ, float);
    }
#undef FGIM_LAUNCH_CQ
#undef FGIM_LAUNCH_CQ2
    return e;
}

extern template cudaError_t launch_cross_query_t<true>(const ShardTable&, const float*, const uint8_t*, const float*,
                                                       long long, int, int, int, fgim_knng*, unsigned long long*,
                                                       int*, cudaStream_t, const int32_t*, const int32_t*, long long,
                                                       const uint16_t*);

}  // namespace fgim
