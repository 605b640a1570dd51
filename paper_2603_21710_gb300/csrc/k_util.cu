// Small building blocks: exclusive scans, compaction by flags, fills, inverse norms.
#include <algorithm>

#include "fgim_launch.h"

namespace fgim {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr long long kScanTile = (long long)kScanThreads * kScanItems;

template <typename TIN>
__global__ void __launch_bounds__(kScanThreads) k_scan_block(const TIN* __restrict__ in, long long n,
                                                             long long* __restrict__ out,
                                                             long long* __restrict__ bsum) {
    __shared__ long long sh[kScanThreads];
    const int tid = threadIdx.x;
    const long long base = (long long)blockIdx.x * kScanTile + (long long)tid * kScanItems;
    long long v[kScanItems];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long idx = base + i;
        v[i] = idx < n ? (long long)in[idx] : 0;
        s += v[i];
    }
    sh[tid] = s;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        long long add = tid >= off ? sh[tid - off] : 0;
        __syncthreads();
        sh[tid] += add;
        __syncthreads();
    }
    long long run = sh[tid] - s;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (tid == kScanThreads - 1) bsum[blockIdx.x] = sh[tid];
}

__global__ void k_scan_add(long long* __restrict__ out, long long n, const long long* __restrict__ boff) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += boff[i / kScanTile];
}

__global__ void k_copy1(long long* dst, const long long* src) { *dst = *src; }

static long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

size_t scan_scratch_bytes(long long n) {
    size_t words = 0;
    long long m = n;
    do {
        long long blocks = cdiv(m > 0 ? m : 1, kScanTile);
        words += 2 * blocks + 1;
        m = blocks;
    } while (m > 1);
    return (words + 8) * sizeof(long long);
}

template <typename TIN>
static cudaError_t scan_impl(const TIN* in, long long n, long long* out, long long* scratch, cudaStream_t s) {
    const long long blocks = cdiv(n > 0 ? n : 1, kScanTile);
    long long* bsum = scratch;
    long long* boff = scratch + blocks;
    {
        LaunchScope ls("k_scan_block", s);
        k_scan_block<TIN><<<(unsigned)blocks, kScanThreads, 0, s>>>(in, n, out, bsum);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (blocks == 1) {
        LaunchScope ls("k_copy1", s);
        k_copy1<<<1, 1, 0, s>>>(out + n, bsum);
        return cudaGetLastError();
    }
    e = scan_impl<long long>(bsum, blocks, boff, scratch + 2 * blocks + 1, s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        LaunchScope ls("k_scan_add", s);
        k_scan_add<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(out, n, boff);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    LaunchScope ls("k_copy1", s);
    k_copy1<<<1, 1, 0, s>>>(out + n, boff + blocks);
    return cudaGetLastError();
}

cudaError_t scan_counts(const int32_t* in, long long n, long long* out, void* scratch, size_t scratch_bytes,
                        cudaStream_t s) {
    if (scratch_bytes < scan_scratch_bytes(n)) return cudaErrorInvalidValue;
    return scan_impl<int32_t>(in, n, out, reinterpret_cast<long long*>(scratch), s);
}

__global__ void k_compact(const int32_t* __restrict__ flag, long long n, const long long* __restrict__ off,
                          int32_t* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[off[i]] = (int32_t)i;
}

cudaError_t compact_flags(const int32_t* flag, long long n, int32_t* out, long long* offsets, void* scan_scratch,
                          size_t scan_bytes, cudaStream_t s) {
    cudaError_t e = scan_counts(flag, n, offsets, scan_scratch, scan_bytes, s);
    if (e != cudaSuccess || n == 0) return e;
    LaunchScope ls("k_compact", s);
    k_compact<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(flag, n, offsets, out);
    return cudaGetLastError();
}

__global__ void k_fill_i32(int32_t* p, long long n, int32_t v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

cudaError_t launch_fill_i32(int32_t* p, long long n, int32_t v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    LaunchScope ls("k_fill_i32", s);
    k_fill_i32<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

// 1 / ||x|| of every row (warp per row), used by the cosine metric
__global__ void k_inv_norms(const float* __restrict__ X, long long n, int d, float* __restrict__ inv) {
    const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float4* x = reinterpret_cast<const float4*>(X + row * d);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int c = lane; c < (d >> 2); c += 32) {
        float4 v = x[c];
        s0 = fmaf(v.x, v.x, s0);
        s1 = fmaf(v.y, v.y, s1);
        s2 = fmaf(v.z, v.z, s2);
        s3 = fmaf(v.w, v.w, s3);
    }
    float s = (s0 + s1) + (s2 + s3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) inv[row] = s > 0.f ? __fdiv_rn(1.f, __fsqrt_rn(s)) : 0.f;
}

cudaError_t launch_inv_norms(const float* X, long long n, int d, float* inv, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    LaunchScope ls("k_inv_norms", s);
    k_inv_norms<<<(unsigned)cdiv(n * 32, 256), 256, 0, s>>>(X, n, d, inv);
    return cudaGetLastError();
}

__global__ void k_bf16_to_f32(const uint16_t* __restrict__ in, long long n, float* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __uint_as_float((uint32_t)in[i] << 16);
}

__global__ void k_valid_flags(const uint8_t* __restrict__ mask, long long n, int32_t* __restrict__ flag) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        flag[i] = (mask == nullptr || mask[i] != 0) ? 1 : 0;
}

cudaError_t launch_valid_flags(const uint8_t* mask, long long n, int32_t* flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    LaunchScope ls("k_valid_flags", s);
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 32);
    k_valid_flags<<<(unsigned)blocks, 256, 0, s>>>(mask, n, flag);
    return cudaGetLastError();
}

__global__ void k_phi(const int32_t* __restrict__ flag, const long long* __restrict__ off, long long n,
                      int32_t* __restrict__ phi) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        phi[i] = flag[i] ? (int32_t)off[i] : -1;
}

cudaError_t launch_phi(const int32_t* flag, const long long* off, long long n, int32_t* phi, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    LaunchScope ls("k_phi", s);
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 32);
    k_phi<<<(unsigned)blocks, 256, 0, s>>>(flag, off, n, phi);
    return cudaGetLastError();
}

// one warp per output row, float4 copies (d % 4 == 0, rows 16-byte aligned)
__global__ void k_gather_rows(const float4* __restrict__ X, const int32_t* __restrict__ src, long long nv, int d4,
                              float4* __restrict__ out) {
    const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= nv) return;
    const float4* a = X + (long long)src[r] * d4;
    float4* b = out + r * d4;
    for (int c = lane; c < d4; c += 32) b[c] = a[c];
}

cudaError_t launch_gather_rows(const float* X, const int32_t* src, long long nv, int d, float* out, cudaStream_t s) {
    if (nv <= 0) return cudaSuccess;
    if (d % 4 != 0) return cudaErrorInvalidValue;
    LaunchScope ls("k_gather_rows", s);
    k_gather_rows<<<(unsigned)((nv * 32 + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float4*>(X), src, nv,
                                                                     d / 4, reinterpret_cast<float4*>(out));
    return cudaGetLastError();
}

cudaError_t launch_bf16_to_f32(const uint16_t* in, long long n, float* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    LaunchScope ls("k_bf16_to_f32", s);
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 32);
    k_bf16_to_f32<<<(unsigned)blocks, 256, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- batches as one problem
// start[r] = entries[m] for the merge m whose id range off[m] .. off[m + 1] - 1 holds reps[r]
__global__ void k_rep_starts(const int32_t* __restrict__ reps, long long nr, const long long* __restrict__ off,
                             const int32_t* __restrict__ entries, int nm, int32_t* __restrict__ start) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    const long long x = reps[r];
    int lo = 0, hi = nm - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (x >= off[mid]) lo = mid;
        else hi = mid - 1;
    }
    start[r] = entries[lo];
}

cudaError_t launch_rep_starts(const int32_t* reps, long long nr, const long long* off, const int32_t* entries, int nm,
                              int32_t* start, cudaStream_t s) {
    if (nr <= 0) return cudaSuccess;
    LaunchScope ls("k_rep_starts", s);
    k_rep_starts<<<(unsigned)((nr + 255) / 256), 256, 0, s>>>(reps, nr, off, entries, nm, start);
    return cudaGetLastError();
}

// rows of one merge out of the union graph: ids renumbered to the merge (id - base), dist, deg
__global__ void k_split_rows(const int32_t* __restrict__ ids, const float* __restrict__ dist,
                             const int32_t* __restrict__ deg, long long n, int R, int32_t base,
                             int32_t* __restrict__ out_ids, float* __restrict__ out_dist, int32_t* __restrict__ out_deg) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n * R) {
        const int32_t v = ids[i];
        out_ids[i] = v >= 0 ? v - base : -1;
        out_dist[i] = dist[i];
    }
    if (i < n) out_deg[i] = deg[i];
}

cudaError_t launch_split_rows(const int32_t* ids, const float* dist, const int32_t* deg, long long n, int R,
                              int32_t base, int32_t* out_ids, float* out_dist, int32_t* out_deg, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    LaunchScope ls("k_split_rows", s);
    k_split_rows<<<(unsigned)((n * R + 255) / 256), 256, 0, s>>>(ids, dist, deg, n, R, base, out_ids, out_dist,
                                                                 out_deg);
    return cudaGetLastError();
}

// Does any adjacency row of the input graphs repeat an id within a 32-entry chunk? (warp per
// vertex; the beam searches check each chunk for repeats unless this says there are none)
__global__ void k_adj_repeats(ShardTable t, long long N, int* flag) {
    const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= N) return;
    const int i = shard_of(t, g);
    const int M = t.M[i];
    const int32_t* row = t.adj[i] + (g - t.off[i]) * M;
    const unsigned lt = (1u << lane) - 1u;
    for (int c0 = 0; c0 < M; c0 += 32) {
        const int v = c0 + lane < M ? row[c0 + lane] : -1;
        const unsigned same = __match_any_sync(kFull, v);   // every lane takes part
        const bool rep = v >= 0 && (same & lt) != 0u;
        if (__any_sync(kFull, rep)) {
            if (lane == 0) atomicOr(flag, 1);
            return;
        }
    }
}

cudaError_t adjacency_has_repeats(const ShardTable& t, long long N, int* status, cudaStream_t s, bool* out) {
    *out = true;
    if (N <= 0) return cudaSuccess;
    int* flag = status + 2;   // a free word of the call's status array
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    {
        LaunchScope ls("k_adj_repeats", s);
        k_adj_repeats<<<(unsigned)((N * 32 + 255) / 256), 256, 0, s>>>(t, N, flag);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    int h = 1;
    if ((e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *out = h != 0;
    return cudaSuccess;
}

}  // namespace fgim
