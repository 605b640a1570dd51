// HNSW-adaptive merging (Sec. 4.3.3): levels of the merged vertices, the exact neighbours of a
// layer's members among the earlier ones (the candidates the RNG heuristic then prunes, see
// fgim_abi.cu), and the hand-over between the per-layer searches of the layered search.
#include "k_beam.cuh"

namespace fgim {

// SplitMix64's v-th output from state `seed` (its published definition), and the level
// #{l >= 1 : r < T_l} with T_l = floor((2^64 - 1) / M^l)
__global__ void k_hnsw_levels(long long n, unsigned long long seed, HnswThresholds th, int32_t* __restrict__ levels) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)(v + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        int l = 0;
        for (int t = 0; t < th.count; ++t) l += z < th.t[t] ? 1 : 0;
        levels[v] = l;
    }
}

cudaError_t launch_hnsw_levels(long long n, unsigned long long seed, const HnswThresholds& th, int32_t* levels,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    LaunchScope ls("k_hnsw_levels", s);
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
    k_hnsw_levels<<<(unsigned)blocks, 256, 0, s>>>(n, seed, th, levels);
    return cudaGetLastError();
}

__global__ void k_level_flags(const int32_t* __restrict__ levels, long long n, int level, int32_t* __restrict__ flag) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        flag[v] = levels[v] >= level ? 1 : 0;
}

cudaError_t launch_level_flags(const int32_t* levels, long long n, int level, int32_t* flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    LaunchScope ls("k_level_flags", s);
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
    k_level_flags<<<(unsigned)blocks, 256, 0, s>>>(levels, n, level, flag);
    return cudaGetLastError();
}

// rows of width M copied into rows of width w >= M, the rest -1 / +inf
__global__ void k_widen(const int32_t* __restrict__ ids, const float* __restrict__ dist, long long n, int M, int w,
                        int32_t* __restrict__ oids, float* __restrict__ odist) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * w; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / w;
        const int s = (int)(i - r * w);
        oids[i] = s < M ? ids[r * M + s] : -1;
        odist[i] = s < M ? dist[r * M + s] : __int_as_float(0x7f800000);
    }
}

cudaError_t launch_widen(const int32_t* ids, const float* dist, long long n, int M, int w, int32_t* oids, float* odist,
                         cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    LaunchScope ls("k_widen", s);
    const long long blocks = std::min<long long>((n * w + 255) / 256, 152LL * 16);
    k_widen<<<(unsigned)blocks, 256, 0, s>>>(ids, dist, n, M, w, oids, odist);
    return cudaGetLastError();
}

// The kk nearest rows of every row u of Xl (n rows) among the rows before it (the members
// inserted before u in id order), by (delta, row): warp per row, 32 candidate rows per step
// through the canonical distances of the beam search, kept in a sorted list in shared memory.
template <int METRIC, bool SMALLD, typename RT>
__global__ void __launch_bounds__(128) k_layer_knn(const float* __restrict__ Xl, const RT* __restrict__ Xr,
                                                   const float* __restrict__ inv, long long n, int d, int kk,
                                                   int32_t* __restrict__ out_ids, float* __restrict__ out_dist) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const long long u = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (u >= n) return;
    const size_t per_warp = (size_t)align16(d * 4) + align16(kk * 8) + 32 * 4 + (sizeof(RT) == 1 ? 0 : 32 * 33 * 4);
    unsigned char* base = smem + per_warp * warp;
    float* q = reinterpret_cast<float*>(base);
    uint64_t* list = reinterpret_cast<uint64_t*>(base + align16(d * 4));
    int32_t* scratch = reinterpret_cast<int32_t*>(base + align16(d * 4) + align16(kk * 8));
    float* P = reinterpret_cast<float*>(base + align16(d * 4) + align16(kk * 8) + 32 * 4);
    const float4* src = reinterpret_cast<const float4*>(Xl + u * d);
    for (int c = lane; c < (d >> 2); c += 32) reinterpret_cast<float4*>(q)[c] = src[c];
    __syncwarp();
    const float4 qreg = (SMALLD && lane < (d >> 2)) ? reinterpret_cast<const float4*>(q)[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    QBytes qb;
    qb.w = make_uint4(0u, 0u, 0u, 0u);
    qb.q2 = 0u;
    if (sizeof(RT) == 1) qb = query_bytes(q, d, lane);
    const float qinv = METRIC == FGIM_COSINE ? inv[u] : 1.f;
    int nl = 0;
    for (long long c0 = 0; c0 < u; c0 += 32) {
        const long long v = c0 + lane;
        const bool ok = v < u;
        const unsigned m = __ballot_sync(kFull, ok);
        const int U = __popc(m);
        if (ok) scratch[__popc(m & lt)] = (int32_t)v;
        __syncwarp();
        const float dd = rows_delta<METRIC, SMALLD, RT>(Xr, scratch, U, q, qreg, qb, d, lane, P);
        uint64_t key = kEmptyKey;
        if (lane < U) {
            const int32_t w = scratch[lane];
            key = mkkey(delta_finish<METRIC>(dd, METRIC == FGIM_COSINE ? __fmul_rn(qinv, inv[w]) : 1.f), w);
        }
        __syncwarp();
        nl = warp_merge<false>(list, nullptr, nl, kk, key, 0);
    }
    for (int s = lane; s < kk; s += 32) {
        out_ids[u * kk + s] = s < nl ? key_id(list[s]) : -1;
        out_dist[u * kk + s] = s < nl ? key_dist(list[s]) : __int_as_float(0x7f800000);
    }
}

cudaError_t launch_layer_knn(const float* Xl, const uint8_t* X8l, const float* inv, long long n, int d, int metric,
                             int kk, int32_t* out_ids, float* out_dist, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const bool bytes = X8l && byte_rows_ok(d);
    const int wpb = 4;
    const size_t per_warp = (size_t)align16(d * 4) + align16(kk * 8) + 32 * 4 + (bytes ? 0 : 32 * 33 * 4);
    const size_t smem = per_warp * wpb;
    const unsigned blocks = (unsigned)((n + wpb - 1) / wpb);
    cudaError_t e = cudaSuccess;
#define FGIM_LAUNCH_LK(MT, SD, RT)                                                                               \
    do {                                                                                                         \
        e = cudaFuncSetAttribute(k_layer_knn<MT, SD, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) break;                                                                             \
        LaunchScope ls("k_layer_knn", s);                                                                        \
        k_layer_knn<MT, SD, RT><<<blocks, wpb * 32, smem, s>>>(Xl, reinterpret_cast<const RT*>(rows), inv, n, d, kk, \
                                                               out_ids, out_dist);                               \
        e = cudaGetLastError();                                                                                  \
    } while (0)
#define FGIM_LAUNCH_LK_D(MT, RT)                                                                                 \
    do {                                                                                                         \
        if (d <= 128) FGIM_LAUNCH_LK(MT, true, RT); else FGIM_LAUNCH_LK(MT, false, RT);                          \
    } while (0)
#define FGIM_LAUNCH_LK_M(RT)                                                                                     \
    do {                                                                                                         \
        if (metric == FGIM_L2SQ) FGIM_LAUNCH_LK_D(FGIM_L2SQ, RT);                                                \
        else if (metric == FGIM_IP) FGIM_LAUNCH_LK_D(FGIM_IP, RT);                                               \
        else FGIM_LAUNCH_LK_D(FGIM_COSINE, RT);                                                                  \
    } while (0)
    if (bytes) {
        const void* rows = X8l;
        FGIM_LAUNCH_LK_M(uint8_t);
    } else {
        const void* rows = Xl;
        FGIM_LAUNCH_LK_M(float);
    }
#undef FGIM_LAUNCH_LK_M
#undef FGIM_LAUNCH_LK_D
#undef FGIM_LAUNCH_LK
    return e;
}

// Between the layer searches of the layered search: query qi's nearest result in layer l
// (a position there) becomes its start in the layer below (a position in `next`, which holds
// every vertex of layer l since levels nest) or, after layer 1, its base-graph entry (a
// global id in `start`). first: every query starts at `entry`'s position in `mem`.
__global__ void k_hnsw_next(const int32_t* __restrict__ best, const int32_t* __restrict__ mem, long long nmem,
                            const int32_t* __restrict__ next, long long nnext, long long nq, int first, int entry,
                            int32_t* __restrict__ qpos, int32_t* __restrict__ start, int* status) {
    const long long qi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= nq) return;
    int32_t g = entry;
    if (!first) {
        const int32_t p = best[qi];
        if (p < 0 || p >= nmem) {
            atomicOr(status, kErrBounds);
            return;
        }
        g = mem[p];
    }
    if (next == nullptr) {
        start[qi] = g;
        return;
    }
    long long lo = 0, hi = nnext;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (next[mid] < g) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= nnext || next[lo] != g) {
        atomicOr(status, kErrBounds);
        lo = 0;
    }
    qpos[qi] = (int32_t)lo;
}

cudaError_t launch_hnsw_next(const int32_t* best, const int32_t* mem, long long nmem, const int32_t* next,
                             long long nnext, long long nq, int first, int entry, int32_t* qpos, int32_t* start,
                             int* status, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    LaunchScope ls("k_hnsw_next", s);
    k_hnsw_next<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(best, mem, nmem, next, nnext, nq, first, entry, qpos,
                                                             start, status);
    return cudaGetLastError();
}

}  // namespace fgim
