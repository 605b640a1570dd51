// Stage (c): k-NNG -> PG (Alg. 5) and the reachability fix.
//
// Neighbour selection runs one warp per vertex u. The candidate rows of u are staged in
// shared memory (padded stride) when they fit; candidates are visited in ascending
// (delta, id); for each one every kept w is tested in parallel (one lane per w) with the
// selection rule (PruneRule: alpha-RNG delta(u, v) < alpha^2 * delta(w, v) keeps v, with alpha^2
// rounded once to FP32 and the product in FP32; or MRNG; or tau-MNG). A lane's own sequential FP32 distance decides whenever the decision is further
// from the boundary than the rounding margin between it and the canonical distance; the few
// decisions inside the margin are re-taken with the canonical distance (whole warp), so the
// outcome is exactly that of the canonical distance.
// A vertex whose only in-edge is u (T(v) = 1) is kept unconditionally (Alg. 5).
//
// Connectivity enhancement builds the reverse lists of the pruned snapshot E' by a
// counting sort and merges them into E'(u), keeping the R smallest (delta, id).
#include <algorithm>

#include <cooperative_groups.h>

#include <map>
#include <mutex>

#include "fgim_launch.h"

namespace fgim {

namespace cg = cooperative_groups;

static inline long long cdivl(long long a, long long b) { return (a + b - 1) / b; }

template <int METRIC, bool STAGE>
__global__ void __launch_bounds__(64) k_prune(const float* __restrict__ X, const float* __restrict__ inv_norm,
                                              long long N, long long nrows, int d, int k, const int32_t* __restrict__ ids,
                                              const float* __restrict__ dist, const int32_t* __restrict__ T, int R,
                                              PruneRule rule, int32_t* __restrict__ e_ids, float* __restrict__ e_dist,
                                              int32_t* __restrict__ e_cnt, int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const long long u = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (u >= nrows) return;
    const int stride = d + 4;
    const int nc4 = d >> 2;
    const size_t per_warp = ((size_t)(STAGE ? k * stride * 4 : 0) + (size_t)k * 12 + 16 + 15) & ~(size_t)15;
    unsigned char* base = smem + per_warp * warp;
    float* rows = reinterpret_cast<float*>(base);
    int32_t* cidv = reinterpret_cast<int32_t*>(base + (STAGE ? (size_t)k * stride * 4 : 0));
    int32_t* kept = cidv + k;
    float* nrm = reinterpret_cast<float*>(kept + k);
    const float eps = fp32_pair_margin(d);

    // valid prefix of list(u)
    int nv = 0;
    for (int s0 = 0; s0 < k; s0 += 32) {
        const int s = s0 + lane;
        int32_t id = s < k ? ids[u * k + s] : -1;
        if (id >= N) {
            atomicOr(status, kErrBounds);
            id = -1;
        }
        if (s < k) cidv[s] = id;
        nv += __popc(__ballot_sync(kFull, id >= 0));
    }
    __syncwarp();
    if (STAGE) {
        // coalesced: each warp pass copies one row
        for (int r = 0; r < nv; ++r) {
            const float4* src = reinterpret_cast<const float4*>(X + (long long)cidv[r] * d);
            float4* dst = reinterpret_cast<float4*>(rows + r * stride);
            for (int c = lane; c < nc4; c += 32) dst[c] = src[c];
        }
        __syncwarp();
    }
    auto rowp = [&](int idx) -> const float4* {
        return STAGE ? reinterpret_cast<const float4*>(rows + idx * stride)
                     : reinterpret_cast<const float4*>(X + (long long)cidv[idx] * d);
    };
    if (METRIC == FGIM_IP) {
        // norms bound the rounding margin of the inner products
        for (int r = lane; r < nv; r += 32) nrm[r] = sqrtf(seq_sum<FGIM_IP>(rowp(r), rowp(r), nc4)) * 1.0001f;
        __syncwarp();
    }
    int nk = 0;
    for (int t = 0; t < nv && nk < R; ++t) {
        const int32_t v = cidv[t];
        bool keep = T[v] == 1;
        if (!keep) {
            const float duv = dist[u * k + t];
            const float4* rv = rowp(t);
            bool occluded = false;
            for (int s0 = 0; s0 < nk && !occluded; s0 += 32) {
                const int s = s0 + lane;
                bool occ = false, near = false;
                float inv = 1.f;
                if (s < nk) {
                    const int wi = kept[s];
                    const float sum = seq_sum<METRIC>(rowp(wi), rv, nc4);
                    if (METRIC == FGIM_COSINE) inv = __fmul_rn(inv_norm[cidv[wi]], inv_norm[v]);
                    const float dt = delta_finish<METRIC>(sum, inv);
                    float md;   // bound on |filter distance - canonical distance|
                    if (METRIC == FGIM_L2SQ) md = eps * sum * 1.01f;
                    else if (METRIC == FGIM_IP) md = eps * nrm[wi] * nrm[t];
                    else md = 2.f * eps;
                    if (rule.kind == 0) {
                        const float bound = rule.alpha2 * dt;
                        // plus the rounding of the product
                        const float m = rule.alpha2 * md + 2.f * 5.9604645e-8f * fabsf(bound);
                        near = fabsf(duv - bound) <= m;
                        occ = !near && !(duv < bound);
                    } else {
                        const bool can = rule.kind == 1 || dist[u * k + wi] < duv;
                        const float thr = rule_thr(rule, duv);
                        near = can && fabsf(dt - thr) <= md;
                        occ = can && !near && dt < thr;
                    }
                }
                if (__any_sync(kFull, occ)) {
                    occluded = true;
                    break;
                }
                // undecided: re-take each near decision with the canonical distance
                unsigned nm = __ballot_sync(kFull, near);
                while (nm && !occluded) {
                    const int l = __ffs(nm) - 1;
                    nm &= nm - 1;
                    const int wi = kept[s0 + l];
                    const float invl = (METRIC == FGIM_COSINE) ? __fmul_rn(inv_norm[cidv[wi]], inv_norm[v]) : 1.f;
                    const float dc = delta_finish<METRIC>(
                        warp_butterfly(lane_part<METRIC>(rowp(wi), rv, nc4, lane)), invl);
                    if (rule_occludes(rule, duv, dist[u * k + wi], dc)) occluded = true;
                }
            }
            keep = !occluded;
        }
        if (keep) {
            if (lane == 0) kept[nk] = t;
            ++nk;
            __syncwarp();
        }
    }
    for (int s = lane; s < R; s += 32) {
        if (s < nk) {
            e_ids[u * R + s] = cidv[kept[s]];
            e_dist[u * R + s] = dist[u * k + kept[s]];
        } else {
            e_ids[u * R + s] = -1;
            e_dist[u * R + s] = __int_as_float(0x7f800000);
        }
    }
    if (lane == 0) e_cnt[u] = nk;
}

// Wide FP32 rows (d > 128): the warp forms every distance together in the canonical order
// (lane chunks, butterfly), reading both rows coalesced from global memory, and tests the
// kept neighbours of u one after another, stopping at the first that occludes v. Each
// decision is taken on the canonical distance, which is what the filter-and-recheck form
// decides as well, so the lists are the same; a rejected candidate usually costs a few
// distances instead of one per kept neighbour.
template <int METRIC>
__global__ void __launch_bounds__(128) k_prune_wide(const float* __restrict__ X, const float* __restrict__ inv_norm,
                                                    long long N, long long nrows, int d, int k, const int32_t* __restrict__ ids,
                                                    const float* __restrict__ dist, const int32_t* __restrict__ T,
                                                    int R, PruneRule rule, int32_t* __restrict__ e_ids,
                                                    float* __restrict__ e_dist, int32_t* __restrict__ e_cnt,
                                                    int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const long long u = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (u >= nrows) return;
    const int nc4 = d >> 2;
    int32_t* cidv = reinterpret_cast<int32_t*>(smem) + (size_t)warp * 2 * k;
    int32_t* kept = cidv + k;
    int nv = 0;
    for (int s0 = 0; s0 < k; s0 += 32) {
        const int s = s0 + lane;
        int32_t id = s < k ? ids[u * k + s] : -1;
        if (id >= N) {
            atomicOr(status, kErrBounds);
            id = -1;
        }
        if (s < k) cidv[s] = id;
        nv += __popc(__ballot_sync(kFull, id >= 0));
    }
    __syncwarp();
    int nk = 0;
    for (int t = 0; t < nv && nk < R; ++t) {
        const int32_t v = cidv[t];
        bool keep = T[v] == 1;
        if (!keep) {
            const float duv = dist[u * k + t];
            const float4* rv = reinterpret_cast<const float4*>(X + (long long)v * d);
            keep = true;
            for (int s = 0; s < nk; ++s) {
                const int32_t w = cidv[kept[s]];
                const float sum = warp_butterfly(
                    lane_part<METRIC>(reinterpret_cast<const float4*>(X + (long long)w * d), rv, nc4, lane));
                const float inv = (METRIC == FGIM_COSINE) ? __fmul_rn(inv_norm[w], inv_norm[v]) : 1.f;
                if (rule_occludes(rule, duv, dist[u * k + kept[s]], delta_finish<METRIC>(sum, inv))) {
                    keep = false;
                    break;
                }
            }
        }
        if (keep) {
            if (lane == 0) kept[nk] = t;
            ++nk;
            __syncwarp();
        }
    }
    for (int s = lane; s < R; s += 32) {
        if (s < nk) {
            e_ids[u * R + s] = cidv[kept[s]];
            e_dist[u * R + s] = dist[u * k + kept[s]];
        } else {
            e_ids[u * R + s] = -1;
            e_dist[u * R + s] = __int_as_float(0x7f800000);
        }
    }
    if (lane == 0) e_cnt[u] = nk;
}

__host__ __device__ inline size_t prune_bytes_per_warp(int k, int d) {
    return ((size_t)k * (d + 16) + (size_t)k * 16 + 15) & ~(size_t)15;
}

// Byte rows (every coordinate an integer in [0, 255], d <= 128, d % 16 == 0): the canonical
// FP32 distance of two rows is then an exact integer (every partial sum is an integer below
// 2^24), computed here directly: |a|^2 + |b|^2 - 2 a.b with four-way byte dot products. No
// filter or re-check is needed. The candidate rows of u are staged as bytes (stride d + 16,
// which spreads the lanes' rows over the banks), with their squared norms.
template <int METRIC>
__global__ void __launch_bounds__(128) k_prune_bytes(const uint8_t* __restrict__ X8, const float* __restrict__ inv_norm,
                                                     long long N, long long nrows, int d, int k, const int32_t* __restrict__ ids,
                                                     const float* __restrict__ dist, const int32_t* __restrict__ T,
                                                     int R, PruneRule rule, int32_t* __restrict__ e_ids,
                                                     float* __restrict__ e_dist, int32_t* __restrict__ e_cnt,
                                                     int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const long long u = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (u >= nrows) return;
    const int stride = d + 16;
    const size_t per_warp = prune_bytes_per_warp(k, d);
    unsigned char* base = smem + per_warp * warp;
    unsigned char* rows = base;
    uint32_t* n2 = reinterpret_cast<uint32_t*>(base + (size_t)k * stride);
    float* invs = reinterpret_cast<float*>(n2 + k);
    int32_t* cidv = reinterpret_cast<int32_t*>(invs + k);
    int32_t* kept = cidv + k;

    // valid prefix of list(u), and its T and delta(u, .) held two per lane
    int nv = 0;
    for (int s0 = 0; s0 < k; s0 += 32) {
        const int s = s0 + lane;
        int32_t id = s < k ? ids[u * k + s] : -1;
        if (id >= N) {
            atomicOr(status, kErrBounds);
            id = -1;
        }
        if (s < k) cidv[s] = id;
        nv += __popc(__ballot_sync(kFull, id >= 0));
    }
    __syncwarp();
    // stage the rows: 32 / lpr rows per warp load, lanes of a row take 16 bytes each
    const int lpr = byte_lanes(d);
    const int rpi = 32 >> byte_lanes_log2(d);
    const int lsh = byte_lanes_log2(d);
    const int sub = lane >> lsh, part = lane & (lpr - 1);
    const bool has = part < (d >> 4);
    for (int r0 = 0; r0 < nv; r0 += 4 * rpi) {
        uint4 w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = r0 + q * rpi + sub;
            w[q] = make_uint4(0u, 0u, 0u, 0u);
            if (r < nv && has) w[q] = *reinterpret_cast<const uint4*>(X8 + (long long)cidv[r] * d + 16 * part);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = r0 + q * rpi + sub;
            uint32_t sq = __dp4a(w[q].x, w[q].x, 0u);
            sq = __dp4a(w[q].y, w[q].y, sq);
            sq = __dp4a(w[q].z, w[q].z, sq);
            sq = __dp4a(w[q].w, w[q].w, sq);
            sq = row_group_sum(sq, lsh);
            if (r < nv) {
                if (has) *reinterpret_cast<uint4*>(rows + (size_t)r * stride + 16 * part) = w[q];
                if (part == 0) n2[r] = sq;
            }
        }
    }
    if (METRIC == FGIM_COSINE)
        for (int r = lane; r < nv; r += 32) invs[r] = inv_norm[cidv[r]];
    // T(v) and delta(u, v) of the candidates, two per lane
    int tA = 0, tB = 0;
    float dA = 0.f, dB = 0.f;
    if (lane < nv) {
        tA = T[cidv[lane]];
        dA = dist[u * k + lane];
    }
    if (lane + 32 < nv) {
        tB = T[cidv[lane + 32]];
        dB = dist[u * k + lane + 32];
    }
    __syncwarp();
    const int c16n = d >> 4;
    int nk = 0;
    for (int t = 0; t < nv && nk < R; ++t) {
        const int tv = __shfl_sync(kFull, t < 32 ? tA : tB, t & 31);
        bool keep = tv == 1;
        if (!keep) {
            const float duv = __shfl_sync(kFull, t < 32 ? dA : dB, t & 31);
            const unsigned char* rv = rows + (size_t)t * stride;
            bool occ = false;
            for (int s0 = 0; s0 < nk; s0 += 32) {
                const int s = s0 + lane;
                if (s < nk) {
                    const int wi = kept[s];
                    const unsigned char* rw = rows + (size_t)wi * stride;
                    // four independent chains (integer sums: any order gives the same total)
                    uint32_t d0 = 0u, d1 = 0u, d2 = 0u, d3 = 0u;
                    for (int c = 0; c < c16n; ++c) {
                        const uint4 a = *reinterpret_cast<const uint4*>(rw + 16 * c);
                        const uint4 b = *reinterpret_cast<const uint4*>(rv + 16 * c);
                        d0 = __dp4a(a.x, b.x, d0);
                        d1 = __dp4a(a.y, b.y, d1);
                        d2 = __dp4a(a.z, b.z, d2);
                        d3 = __dp4a(a.w, b.w, d3);
                    }
                    const uint32_t dot = (d0 + d1) + (d2 + d3);
                    float dc;
                    if (METRIC == FGIM_L2SQ) dc = (float)(n2[wi] + n2[t] - 2u * dot);
                    else if (METRIC == FGIM_IP) dc = delta_finish<FGIM_IP>((float)dot, 1.f);
                    else dc = delta_finish<FGIM_COSINE>((float)dot, __fmul_rn(invs[wi], invs[t]));
                    occ |= rule_occludes(rule, duv, dist[u * k + wi], dc);
                }
            }
            keep = !__any_sync(kFull, occ);
        }
        if (keep) {
            if (lane == 0) kept[nk] = t;
            ++nk;
            __syncwarp();
        }
    }
    for (int s = lane; s < R; s += 32) {
        if (s < nk) {
            e_ids[u * R + s] = cidv[kept[s]];
            e_dist[u * R + s] = dist[u * k + kept[s]];
        } else {
            e_ids[u * R + s] = -1;
            e_dist[u * R + s] = __int_as_float(0x7f800000);
        }
    }
    if (lane == 0) e_cnt[u] = nk;
}

cudaError_t launch_prune(const float* X, const uint8_t* X8, const float* inv_norm, long long N, int d, int metric,
                         const fgim_knng& g, const int32_t* T, int R, PruneRule rule, int32_t* e_ids, float* e_dist,
                         int32_t* e_cnt, int* status, cudaStream_t s) {
    const long long nrows = g.n;   // lists to prune (ids range over 0 .. N - 1)
    if (nrows <= 0) return cudaSuccess;
    const int k = g.k;
    if (X8 && byte_rows_ok(d) && k <= 64) {
        const int wpb = 4;
        const size_t smem = prune_bytes_per_warp(k, d) * wpb;
        cudaError_t e = cudaSuccess;
#define FGIM_LAUNCH_PB(MT)                                                                                        \
    do {                                                                                                          \
        e = cudaFuncSetAttribute(k_prune_bytes<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
        if (e != cudaSuccess) break;                                                                              \
        LaunchScope ls("k_prune", s);                                                                             \
        k_prune_bytes<MT><<<(unsigned)cdivl(nrows, wpb), wpb * 32, smem, s>>>(X8, inv_norm, N, nrows, d, k, g.ids, g.dist, T, \
                                                                          R, rule, e_ids, e_dist, e_cnt, status);\
        e = cudaGetLastError();                                                                                   \
    } while (0)
        if (metric == FGIM_L2SQ) FGIM_LAUNCH_PB(FGIM_L2SQ);
        else if (metric == FGIM_IP) FGIM_LAUNCH_PB(FGIM_IP);
        else FGIM_LAUNCH_PB(FGIM_COSINE);
#undef FGIM_LAUNCH_PB
        return e;
    }
    if (d > 128) {
        const int wpb = 4;
        const size_t smem = (size_t)wpb * 2 * k * sizeof(int32_t);
        cudaError_t e = cudaSuccess;
#define FGIM_LAUNCH_PW(MT)                                                                                        \
    do {                                                                                                          \
        LaunchScope ls("k_prune", s);                                                                             \
        k_prune_wide<MT><<<(unsigned)cdivl(nrows, wpb), wpb * 32, smem, s>>>(X, inv_norm, N, nrows, d, k, g.ids, g.dist, T, R,  \
                                                                         rule, e_ids, e_dist, e_cnt, status);   \
        e = cudaGetLastError();                                                                                   \
    } while (0)
        if (metric == FGIM_L2SQ) FGIM_LAUNCH_PW(FGIM_L2SQ);
        else if (metric == FGIM_IP) FGIM_LAUNCH_PW(FGIM_IP);
        else FGIM_LAUNCH_PW(FGIM_COSINE);
#undef FGIM_LAUNCH_PW
        return e;
    }
    const int wpb = 2;
    const size_t staged = ((size_t)k * (d + 4) * 4 + (size_t)k * 12 + 16 + 15) & ~(size_t)15;
    const size_t unstaged = ((size_t)k * 12 + 16 + 15) & ~(size_t)15;
    const bool stage = staged * wpb <= 160 * 1024;
    const size_t smem = (stage ? staged : unstaged) * wpb;
    cudaError_t e = cudaSuccess;
#define FGIM_LAUNCH_P(MT, ST)                                                                                     \
    do {                                                                                                          \
        e = cudaFuncSetAttribute(k_prune<MT, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
        if (e != cudaSuccess) break;                                                                              \
        LaunchScope ls("k_prune", s);                                                                             \
        k_prune<MT, ST><<<(unsigned)cdivl(nrows, wpb), wpb * 32, smem, s>>>(X, inv_norm, N, nrows, d, k, g.ids, g.dist, T, R, \
                                                                        rule, e_ids, e_dist, e_cnt, status);    \
        e = cudaGetLastError();                                                                                   \
    } while (0)
    if (stage) {
        if (metric == FGIM_L2SQ) FGIM_LAUNCH_P(FGIM_L2SQ, true);
        else if (metric == FGIM_IP) FGIM_LAUNCH_P(FGIM_IP, true);
        else FGIM_LAUNCH_P(FGIM_COSINE, true);
    } else {
        if (metric == FGIM_L2SQ) FGIM_LAUNCH_P(FGIM_L2SQ, false);
        else if (metric == FGIM_IP) FGIM_LAUNCH_P(FGIM_IP, false);
        else FGIM_LAUNCH_P(FGIM_COSINE, false);
    }
#undef FGIM_LAUNCH_P
    return e;
}

// ---------------------------------------------------------------------------- reverse insertion
__global__ void k_e_count(const int32_t* __restrict__ e_ids, long long total, int32_t* __restrict__ cnt) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int32_t v = e_ids[i];
    if (v >= 0) atomicAdd(cnt + v, 1);
}

__global__ void k_e_fill(const int32_t* __restrict__ e_ids, const float* __restrict__ e_dist, long long total, int R,
                         const long long* __restrict__ off, int32_t* __restrict__ fill, uint64_t* __restrict__ rev) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int32_t v = e_ids[i];
    if (v < 0) return;
    const int p = atomicAdd(fill + v, 1);
    rev[off[v] + p] = mkkey(e_dist[i], (int32_t)div_idx(i, R));
}

__global__ void __launch_bounds__(128) k_e_merge(const int32_t* __restrict__ e_ids, const float* __restrict__ e_dist,
                                                 const int32_t* __restrict__ e_cnt, long long N, int R,
                                                 const long long* __restrict__ off, const uint64_t* __restrict__ rev,
                                                 int32_t* __restrict__ out_ids, float* __restrict__ out_dist,
                                                 int32_t* __restrict__ out_deg) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const long long u = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (u >= N) return;
    uint64_t* list = reinterpret_cast<uint64_t*>(smem) + (size_t)warp * R;
    const int ne = e_cnt[u];
    for (int s = lane; s < ne; s += 32) list[s] = mkkey(e_dist[u * R + s], e_ids[u * R + s]);
    __syncwarp();
    int n = ne;
    const long long b = off[u], m = off[u + 1] - off[u];
    for (long long c0 = 0; c0 < m; c0 += 32) {
        const uint64_t key = (c0 + lane < m) ? rev[b + c0 + lane] : kEmptyKey;
        n = warp_merge<true>(list, nullptr, n, R, key, 0);
    }
    for (int s = lane; s < R; s += 32) {
        if (s < n) {
            out_ids[u * R + s] = key_id(list[s]);
            out_dist[u * R + s] = key_dist(list[s]);
        } else {
            out_ids[u * R + s] = -1;
            out_dist[u * R + s] = __int_as_float(0x7f800000);
        }
    }
    if (lane == 0) out_deg[u] = n;
}

cudaError_t launch_reverse_insert(long long N, int R, const int32_t* e_ids, const float* e_dist, const int32_t* e_cnt,
                                  ReverseBuffers& b, int32_t* out_ids, float* out_dist, int32_t* out_deg,
                                  cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const long long total = N * R;
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.cnt, 0, sizeof(int32_t) * N, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.fill, 0, sizeof(int32_t) * N, s)) != cudaSuccess) return e;
    const unsigned gb = (unsigned)cdivl(total, 256);
    {
        LaunchScope ls("k_e_count", s);
        k_e_count<<<gb, 256, 0, s>>>(e_ids, total, b.cnt);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = scan_counts(b.cnt, N, b.off, b.scan_tmp, b.scan_bytes, s)) != cudaSuccess) return e;
    {
        LaunchScope ls("k_e_fill", s);
        k_e_fill<<<gb, 256, 0, s>>>(e_ids, e_dist, total, R, b.off, b.fill, b.rev);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int wpb = 4;
    LaunchScope ls("k_e_merge", s);
    k_e_merge<<<(unsigned)cdivl(N, wpb), wpb * 32, (size_t)wpb * R * 8, s>>>(e_ids, e_dist, e_cnt, N, R, b.off, b.rev,
                                                                             out_ids, out_dist, out_deg);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- reachability fix
// BFS state: st[0..2] frontier sizes (level L reads st[L % 3], writes st[(L + 1) % 3] and
// clears st[(L + 2) % 3] for the level after), st[4..5] the number of reached vertices (int64)
__global__ void k_bfs_init(int32_t* visited, long long N, int32_t* frontier, int32_t* st, int entry) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) visited[i] = (i == entry) ? 1 : 0;
    if (i == 0) {
        frontier[0] = entry;
        st[1] = 1;   // level 1 reads st[1]
        st[2] = 0;
        st[0] = 0;
        *reinterpret_cast<long long*>(st + 4) = 1;
    }
}

cudaError_t launch_bfs_init(int32_t* visited, long long N, int32_t* frontier, int32_t* st, int entry,
                            cudaStream_t s) {
    LaunchScope ls("k_bfs_init", s);
    k_bfs_init<<<(unsigned)cdivl(N, 256), 256, 0, s>>>(visited, N, frontier, st, entry);
    return cudaGetLastError();
}

// BFS from several sources at once (the entries of the merges of a batch, each in its own
// component of the union graph): every entry is at level 1 and in the first frontier
__global__ void k_bfs_init_multi(int32_t* visited, long long N, int32_t* frontier, int32_t* st,
                                 const int32_t* __restrict__ entries, int ne) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) visited[i] = 0;
    if (i == 0) {
        st[1] = ne;
        st[2] = 0;
        st[0] = 0;
        *reinterpret_cast<long long*>(st + 4) = ne;
    }
}
__global__ void k_bfs_seed(int32_t* visited, long long N, int32_t* frontier, const int32_t* __restrict__ entries,
                           int ne, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const int32_t e = entries[i];
    if (e < 0 || e >= N) {
        atomicOr(status, kErrBounds);
        frontier[i] = 0;
        return;
    }
    visited[e] = 1;
    frontier[i] = e;
}

cudaError_t launch_bfs_init_multi(int32_t* visited, long long N, int32_t* frontier, int32_t* st,
                                  const int32_t* entries, int ne, int* status, cudaStream_t s) {
    {
        LaunchScope ls("k_bfs_init", s);
        k_bfs_init_multi<<<(unsigned)cdivl(N, 256), 256, 0, s>>>(visited, N, frontier, st, entries, ne);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    LaunchScope ls("k_bfs_init", s);
    k_bfs_seed<<<(unsigned)cdivl(ne, 256), 256, 0, s>>>(visited, N, frontier, entries, ne, status);
    return cudaGetLastError();
}

// one level L (grid-stride over (frontier vertex, neighbour slot)); visited[y] = BFS level
// (entry = 1); a level whose frontier is empty does nothing, so several levels can be
// queued without reading the frontier size on the host
__global__ void k_bfs_step(const int32_t* __restrict__ graph, int R, long long N, int32_t* __restrict__ visited,
                           const int32_t* __restrict__ fin, int32_t* __restrict__ fout, int32_t* __restrict__ st,
                           int level) {
    const long long nf = st[level % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) st[(level + 2) % 3] = 0;
    const int32_t next_level = level + 1;
    int added = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nf * R;
         i += (long long)gridDim.x * blockDim.x) {
        const long long fi = div_idx(i, R);
        const int32_t x = fin[fi];
        const int32_t y = graph[(long long)x * R + (i - fi * R)];
        if (y < 0 || y >= N) continue;
        if (visited[y] == 0 && atomicCAS(visited + y, 0, next_level) == 0) {
            fout[atomicAdd(st + (level + 1) % 3, 1)] = y;
            ++added;
        }
    }
    const unsigned m = __ballot_sync(kFull, added > 0);
    int sum = added;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(reinterpret_cast<unsigned long long*>(st + 4), (unsigned long long)sum);
}

cudaError_t launch_bfs_levels(const int32_t* graph, int R, long long N, int32_t* visited, int32_t* fa, int32_t* fb,
                              int32_t* st, int level0, int levels, cudaStream_t s) {
    const long long work = N * (long long)R;
    const unsigned blocks = (unsigned)std::min<long long>(cdivl(work, 256), 152LL * 16);
    for (int q = 0; q < levels; ++q) {
        const int level = level0 + q;
        // level L reads the frontier written by level L - 1: fa for odd L, fb for even L
        const int32_t* fin = (level & 1) ? fa : fb;
        int32_t* fout = (level & 1) ? fb : fa;
        LaunchScope ls("k_bfs_step", s);
        k_bfs_step<<<blocks, 256, 0, s>>>(graph, R, N, visited, fin, fout, st, level);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// number of BFS parents of every reached vertex: in-neighbours at a smaller level
__global__ void k_bfs_parents(const int32_t* __restrict__ graph, int R, long long N, const int32_t* __restrict__ level,
                              int32_t* __restrict__ npar) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * R) return;
    const int32_t lx = level[div_idx(i, R)];
    if (lx == 0) return;
    const int32_t y = graph[i];
    if (y >= 0 && y < N && level[y] > lx) atomicAdd(npar + y, 1);
}

cudaError_t launch_bfs_parents(const int32_t* graph, int R, long long N, const int32_t* level, int32_t* npar,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(npar, 0, sizeof(int32_t) * N, s);
    if (e != cudaSuccess) return e;
    LaunchScope ls("k_bfs_parents", s);
    k_bfs_parents<<<(unsigned)cdivl(N * R, 256), 256, 0, s>>>(graph, R, N, level, npar);
    return cudaGetLastError();
}

__global__ void k_cc_init(const int32_t* __restrict__ visited, long long N, int32_t* __restrict__ label) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) label[i] = visited[i] ? -1 : (int32_t)i;
}

cudaError_t launch_cc_init(const int32_t* visited, long long N, int32_t* label, cudaStream_t s) {
    LaunchScope ls("k_cc_init", s);
    k_cc_init<<<(unsigned)cdivl(N, 256), 256, 0, s>>>(visited, N, label);
    return cudaGetLastError();
}

// min-label propagation over the undirected edges between unreached vertices
__global__ void k_cc_step(const int32_t* __restrict__ graph, int R, long long N, const int32_t* __restrict__ visited,
                          int32_t* __restrict__ label, int32_t* __restrict__ changed) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * R) return;
    const long long x = div_idx(i, R);
    if (visited[x]) return;
    const int32_t y = graph[i];
    if (y < 0 || y >= N || visited[y]) return;
    const int32_t lx = label[x], ly = label[y];
    if (lx < ly) {
        if (atomicMin(label + y, lx) > lx) *changed = 1;
    } else if (ly < lx) {
        if (atomicMin(label + x, ly) > ly) *changed = 1;
    }
}

cudaError_t launch_cc_step(const int32_t* graph, int R, long long N, const int32_t* visited, int32_t* label,
                           int32_t* changed, cudaStream_t s) {
    LaunchScope ls("k_cc_step", s);
    k_cc_step<<<(unsigned)cdivl(N * R, 256), 256, 0, s>>>(graph, R, N, visited, label, changed);
    return cudaGetLastError();
}

__global__ void k_rep_flags(const int32_t* __restrict__ visited, const int32_t* __restrict__ label, long long N,
                            int32_t* __restrict__ flag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) flag[i] = (!visited[i] && label[i] == (int32_t)i) ? 1 : 0;
}

cudaError_t launch_rep_flags(const int32_t* visited, const int32_t* label, long long N, int32_t* flag,
                             cudaStream_t s) {
    LaunchScope ls("k_rep_flags", s);
    k_rep_flags<<<(unsigned)cdivl(N, 256), 256, 0, s>>>(visited, label, N, flag);
    return cudaGetLastError();
}

// Attachment of the representatives with the result of the sequential loop over them in
// ascending id, computed in parallel rounds (warp per representative). The action of x:
// the first search result p with room gets x appended; otherwise the first search result
// with a replaceable neighbour y (reached, keeps a BFS parent other than p) has its
// farthest such y replaced by x. Reads that other actions cannot change are not reserved:
// a full list stays full (degrees only grow) and a neighbour that is not replaceable stays
// so (parent counts only shrink). Only p (its list and degree) and y (its parent count)
// are reserved with atomicMin of a tag ordered by (round, representative index); the
// longest ascending prefix of the round's window holding its reservations is committed,
// the rest recomputed in the next round.
//
// Round rho works on the window [ff[rho - 1], min(ff[rho - 1] + W, nr)) and leaves in ff[rho]
// the first index it did not commit (the next round's start). Tags of later rounds are
// smaller than those of earlier ones, so owner needs no reset between rounds.
__device__ __forceinline__ unsigned long long reach_tag(long long rho, long long r) {
    return ((unsigned long long)(0xFFFFFFFFu - (uint32_t)rho) << 32) | (unsigned long long)(uint32_t)r;
}

// The action of representative r on the current graph (whole warp; the result is the same in
// every lane): (p, position in p's list, index of p among r's search results, victim or -1);
// p = -1: no action.
__device__ __forceinline__ int4 reach_plan(const int32_t* __restrict__ graph, const int32_t* __restrict__ deg,
                                           const int32_t* __restrict__ level, const int32_t* __restrict__ npar,
                                           int R, const int32_t* cr, int beam, int lane) {
    int p = -1, pos = -1, t_sel = -1;
    for (int t0 = 0; t0 < beam && p < 0; t0 += 32) {
        const int t = t0 + lane;
        const int32_t q = t < beam ? cr[t] : -1;
        const bool room = q >= 0 && deg[q] < R;
        const unsigned m = __ballot_sync(kFull, room);
        if (m) {
            t_sel = t0 + __ffs(m) - 1;
            p = cr[t_sel];
            pos = deg[p];
        }
    }
    for (int t = 0; t < beam && p < 0; ++t) {
        const int32_t q = cr[t];
        if (q < 0) break;
        const int dq = deg[q];
        const int32_t lq = level[q];
        int best = -1;
        for (int s0 = ((R - 1) >> 5) << 5; s0 >= 0 && best < 0; s0 -= 32) {
            const int s = s0 + lane;
            bool ok = false;
            if (s < dq) {
                const int32_t y = graph[(long long)q * R + s];
                const int32_t ly = level[y];
                ok = ly > 0 && npar[y] - (lq < ly ? 1 : 0) >= 1;
            }
            const unsigned m = __ballot_sync(kFull, ok);
            if (m) best = s0 + 31 - __clz(m);
        }
        if (best >= 0) {
            p = q;
            pos = best;
            t_sel = t;
        }
    }
    const int32_t victim = (p >= 0 && pos < deg[p]) ? graph[(long long)p * R + pos] : -1;
    return make_int4(p, pos, t_sel, victim);
}

// The rounds of one batch in one cooperative launch (warps stride over the window): plan
// (the action of every item and its reservations), check (the first item that lost one
// bounds the prefix), commit (the prefix); phases are separated by grid-wide barriers and an
// item's plan is computed once per round.
__global__ void __launch_bounds__(128) k_reach_rounds(int32_t* __restrict__ graph, float* __restrict__ gdist,
                                                      int32_t* __restrict__ deg, const int32_t* __restrict__ level,
                                                      int32_t* __restrict__ npar, int R,
                                                      const int32_t* __restrict__ reps, long long nr, long long rho0,
                                                      int rounds, long long window, long long* __restrict__ ff,
                                                      const int32_t* __restrict__ cand,
                                                      const float* __restrict__ cdist, int beam,
                                                      unsigned long long* __restrict__ owner, int4* __restrict__ plan,
                                                      unsigned long long* attached) {
    cg::grid_group grid = cg::this_grid();
    const int lane = lane_id();
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (int q = 0; q < rounds; ++q) {
        const long long rho = rho0 + q;
        const long long start = ff[rho - 1];   // written before the last barrier
        if (start >= nr) {                     // the same for every thread: all leave together
            if (blockIdx.x == 0 && threadIdx.x == 0)
                for (int t = q; t < rounds; ++t) ff[rho0 + t] = nr;
            return;
        }
        const long long wend = start + window < nr ? start + window : nr;
        if (blockIdx.x == 0 && threadIdx.x == 0) ff[rho] = wend;
        for (long long r = start + gw; r < wend; r += nw) {
            const int4 pl = reach_plan(graph, deg, level, npar, R, cand + r * beam, beam, lane);
            if (lane == 0) {
                plan[r - start] = pl;
                if (pl.x >= 0) {
                    const unsigned long long tag = reach_tag(rho, r);
                    atomicMin(owner + pl.x, tag);
                    if (pl.w >= 0) atomicMin(owner + pl.w, tag);
                }
            }
        }
        grid.sync();
        for (long long r = start + gw * 32 + lane; r < wend; r += nw * 32) {
            const int4 pl = plan[r - start];
            const unsigned long long tag = reach_tag(rho, r);
            if (pl.x >= 0 && (owner[pl.x] != tag || (pl.w >= 0 && owner[pl.w] != tag)))
                atomicMin((unsigned long long*)(ff + rho), (unsigned long long)r);
        }
        grid.sync();
        const long long cend = ff[rho];
        for (long long r = start + gw * 32 + lane; r < cend; r += nw * 32) {
            const int4 pl = plan[r - start];
            if (pl.x < 0) continue;
            const int32_t p = pl.x, victim = pl.w, x = reps[r];
            int pos = pl.y;
            int32_t* li = graph + (long long)p * R;
            float* ld = gdist + (long long)p * R;
            const float d = cdist[r * beam + pl.z];
            const uint64_t key = mkkey(d, x);
            if (pos == deg[p]) deg[p] += 1;
            else if (level[p] < level[victim]) npar[victim] -= 1;
            while (pos > 0 && mkkey(ld[pos - 1], li[pos - 1]) > key) {
                li[pos] = li[pos - 1];
                ld[pos] = ld[pos - 1];
                --pos;
            }
            while (pos + 1 < deg[p] && mkkey(ld[pos + 1], li[pos + 1]) < key) {
                li[pos] = li[pos + 1];
                ld[pos] = ld[pos + 1];
                ++pos;
            }
            li[pos] = x;
            ld[pos] = d;
            atomicAdd(attached, 1ull);
        }
        grid.sync();
    }
}

cudaError_t launch_reach_rounds(int32_t* graph, float* gdist, int32_t* deg, const int32_t* level, int32_t* npar,
                                int R, const int32_t* reps, long long nr, long long rho0, int rounds, long long* ff,
                                const int32_t* cand, const float* cdist, int beam, unsigned long long* owner,
                                int4* plan, unsigned long long* attached, cudaStream_t s) {
    // a cooperative grid: every block resident at once (the barriers wait for all of them);
    // the largest such grid is worked out once per device (devices may differ in SM count)
    static std::mutex mu;
    static std::map<int, int> max_blocks_of;
    cudaError_t e = cudaSuccess;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    int max_blocks = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = max_blocks_of.find(dev);
        if (it != max_blocks_of.end()) {
            max_blocks = it->second;
        } else {
            int per_sm = 0, sms = 0;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_reach_rounds, 128, 0)) != cudaSuccess)
                return e;
            max_blocks = per_sm * sms;
            if (max_blocks < 1) return cudaErrorCooperativeLaunchTooLarge;
            max_blocks_of[dev] = max_blocks;
        }
    }
    long long window = kReachWindow;
    const int blocks = (int)std::min<long long>(cdivl(window, 4), max_blocks);
    LaunchScope ls("k_reach_rounds", s);
    void* args[] = {&graph, &gdist, &deg, &level, &npar, &R, &reps, &nr, &rho0, &rounds, &window, &ff,
                    &cand, &cdist, &beam, &owner, &plan, &attached};
    return cudaLaunchCooperativeKernel((const void*)k_reach_rounds, dim3(blocks), dim3(128), args, 0, s);
}

}  // namespace fgim
