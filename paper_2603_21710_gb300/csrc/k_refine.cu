// Stage (b): k-NNG refinement, Alg. 3 (Visit + Update) and Alg. 4 (indegree repair).
//
// Synchronous form of one refinement pass:
//   Visit   reverse lists of new / old entries (counting sort by destination, then the
//           rev_cap smallest (delta, source) per vertex), C_n(v) = new forward U new
//           reverse, C_o(v) = (old forward U old reverse) \ C_n(v); forward new flags
//           are cleared once the sets are built.
//   Update  one CTA per vertex v evaluates every cross-graph pair of C_n(v)^2 U
//           C_n(v) x C_o(v) as a register-tiled distance tile (rows C_n, columns C_n ++
//           C_o, upper triangle in C_n), and emits a proposal "b for list(a)" only when
//           b is not already in list(a) (membership bitmask built in shared memory
//           from the candidates' lists) and (delta, b) beats list(a)'s worst key.
//   Merge   proposals are grouped by target (counting sort) and each list becomes the
//           top-k of its entries and its proposals, duplicates by id removed, inserted
//           entries flagged new. The result does not depend on the order of proposals.
// A proposal buffer that overflows marks the vertices whose proposals were dropped;
// the host merges what fits and re-runs those vertices (their pairs are re-evaluated
// against the updated lists), which yields the same final lists.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "fgim_launch.h"
#include "tc_sm100.cuh"

namespace fgim {

static inline long long cdivll(long long a, long long b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------- indegree
__global__ void k_indegree(const int32_t* __restrict__ ids, long long total, int32_t* __restrict__ T,
                           uint8_t* __restrict__ flags) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int32_t v = ids[i];
    if (v >= 0) atomicAdd(T + v, 1);
    if (flags) flags[i] &= (uint8_t)~FGIM_FLAG_REPLACED;
}

cudaError_t launch_indegree(const int32_t* ids, long long N, int k, int32_t* T, bool clear_replaced, uint8_t* flags,
                            cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(T, 0, sizeof(int32_t) * N, s);
    if (e != cudaSuccess) return e;
    const long long total = N * k;
    if (total == 0) return cudaSuccess;
    LaunchScope ls("k_indegree", s);
    k_indegree<<<(unsigned)cdivll(total, 256), 256, 0, s>>>(ids, total, T, clear_replaced ? flags : nullptr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- Visit
__global__ void k_rev_count(const int32_t* __restrict__ ids, const uint8_t* __restrict__ flags, long long total,
                            int32_t* __restrict__ cntN, int32_t* __restrict__ cntO) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int32_t v = ids[i];
    if (v < 0) return;
    atomicAdd((flags[i] & FGIM_FLAG_NEW) ? cntN + v : cntO + v, 1);
}

__global__ void k_rev_fill(const int32_t* __restrict__ ids, const float* __restrict__ dist,
                           const uint8_t* __restrict__ flags, long long total, int k,
                           const long long* __restrict__ offN, const long long* __restrict__ offO,
                           int32_t* __restrict__ fillN, int32_t* __restrict__ fillO, uint64_t* __restrict__ revN,
                           uint64_t* __restrict__ revO) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int32_t v = ids[i];
    if (v < 0) return;
    const int32_t u = (int32_t)div_idx(i, k);
    const uint64_t key = mkkey(dist[i], u);
    if (flags[i] & FGIM_FLAG_NEW) {
        const int p = atomicAdd(fillN + v, 1);
        revN[offN[v] + p] = key;
    } else {
        const int p = atomicAdd(fillO + v, 1);
        revO[offO[v] + p] = key;
    }
}

// the `cap` smallest (delta, source) keys of every reverse segment (warp per vertex), as a set:
// in segment order when the segment has at most `cap` entries, else ascending
__global__ void __launch_bounds__(128) k_rev_select(const long long* __restrict__ off, const uint64_t* __restrict__ rev,
                                                    long long N, int cap, int32_t* __restrict__ top,
                                                    int32_t* __restrict__ ntop) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const long long v = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (v >= N) return;
    uint64_t* list = reinterpret_cast<uint64_t*>(smem) + (size_t)warp * cap;
    const long long b = off[v], m = off[v + 1] - off[v];
    if (m <= cap) {   // the whole segment is the selection: the candidate sets are sets, so no order is needed
        for (long long s = lane; s < m; s += 32) top[v * cap + s] = key_id(rev[b + s]);
        if (lane == 0) ntop[v] = (int)m;
        return;
    }
    if (m <= 32) {   // one sort: the keys of a segment are distinct (one entry per source)
        const uint64_t sorted = warp_sort32(lane < m ? rev[b + lane] : kEmptyKey);
        const int nk = (int)(m < cap ? m : cap);
        if (lane < nk) top[v * cap + lane] = key_id(sorted);
        if (lane == 0) ntop[v] = nk;
        return;
    }
    int n = 0;
    for (long long c0 = 0; c0 < m; c0 += 32) {
        const uint64_t key = (c0 + lane < m) ? rev[b + c0 + lane] : kEmptyKey;
        n = warp_merge<false>(list, nullptr, n, cap, key, 0);
    }
    for (int s = lane; s < n; s += 32) top[v * cap + s] = key_id(list[s]);
    if (lane == 0) ntop[v] = n;
}

// C_n(v), C_o(v) of every vertex (warp per vertex); clears the forward new flags. An id
// enters the first set it is offered to (new forward, new reverse, old forward, old reverse,
// in this order): a per-warp hash set in shared memory (hs slots, at most half full) tells
// whether it is there already.
__global__ void __launch_bounds__(128) k_build_cands(const int32_t* __restrict__ ids, uint8_t* __restrict__ flags,
                                                     long long N, int k, const int32_t* __restrict__ topN,
                                                     const int32_t* __restrict__ ntopN,
                                                     const int32_t* __restrict__ topO,
                                                     const int32_t* __restrict__ ntopO, int rev_cap,
                                                     int32_t* __restrict__ cand, int32_t* __restrict__ nn_out,
                                                     int32_t* __restrict__ no_out, int cmax, int hs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const long long v = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (v >= N) return;
    int32_t* C = reinterpret_cast<int32_t*>(smem) + (size_t)warp * (cmax + hs);
    int32_t* H = C + cmax;
    for (int i = lane; i < hs; i += 32) H[i] = -1;
    __syncwarp();
    // true when id was not in the set (it is now)
    auto ins = [&](int32_t id) -> bool {
        int slot = (int)(((uint32_t)id * 2654435761u) >> 7) & (hs - 1);
        for (int p = 0; p < hs; ++p) {
            const int32_t prev = atomicCAS(H + slot, -1, id);
            if (prev == -1) return true;
            if (prev == id) return false;
            slot = (slot + 1) & (hs - 1);
        }
        return false;
    };
    const unsigned lt = (1u << lane) - 1u;
    int nn = 0, no = 0;
    auto offer = [&](int32_t id, bool ok, int& cnt, int base) {
        const bool take = ok && ins(id);
        const unsigned m = __ballot_sync(kFull, take);
        if (take) C[base + cnt + __popc(m & lt)] = id;
        cnt += __popc(m);
        __syncwarp();
    };
    for (int t0 = 0; t0 < k; t0 += 32) {   // new forward neighbours
        const int t = t0 + lane;
        const int32_t id = t < k ? ids[v * k + t] : -1;
        offer(id, id >= 0 && (flags[v * k + t] & FGIM_FLAG_NEW), nn, 0);
    }
    const int rn = ntopN[v];
    for (int t0 = 0; t0 < rn; t0 += 32) {   // new reverse neighbours
        const int t = t0 + lane;
        offer(t < rn ? topN[v * rev_cap + t] : -1, t < rn, nn, 0);
    }
    for (int t0 = 0; t0 < k; t0 += 32) {   // old forward neighbours
        const int t = t0 + lane;
        const int32_t id = t < k ? ids[v * k + t] : -1;
        offer(id, id >= 0 && !(flags[v * k + t] & FGIM_FLAG_NEW), no, nn);
    }
    const int ro = ntopO[v];
    for (int t0 = 0; t0 < ro; t0 += 32) {   // old reverse neighbours
        const int t = t0 + lane;
        offer(t < ro ? topO[v * rev_cap + t] : -1, t < ro, no, nn);
    }
    for (int s = lane; s < nn + no; s += 32) cand[v * cmax + s] = C[s];
    if (lane == 0) {
        nn_out[v] = nn;
        no_out[v] = no;
    }
    // Visit done: the forward new neighbours of v are old from now on
    for (int t = lane; t < k; t += 32) flags[v * k + t] &= (uint8_t)~FGIM_FLAG_NEW;
}

cudaError_t refine_visit(const fgim_knng& g, int rev_cap, RefineBuffers& b, cudaStream_t s) {
    const long long N = g.n;
    const int k = g.k;
    const long long total = N * k;
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.cntN, 0, sizeof(int32_t) * N, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.cntO, 0, sizeof(int32_t) * N, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.fillN, 0, sizeof(int32_t) * N, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.fillO, 0, sizeof(int32_t) * N, s)) != cudaSuccess) return e;
    const unsigned gb = (unsigned)cdivll(total, 256);
    {
        LaunchScope ls("k_rev_count", s);
        k_rev_count<<<gb, 256, 0, s>>>(g.ids, g.flags, total, b.cntN, b.cntO);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = scan_counts(b.cntN, N, b.offN, b.scan_tmp, b.scan_bytes, s)) != cudaSuccess) return e;
    if ((e = scan_counts(b.cntO, N, b.offO, b.scan_tmp, b.scan_bytes, s)) != cudaSuccess) return e;
    {
        LaunchScope ls("k_rev_fill", s);
        k_rev_fill<<<gb, 256, 0, s>>>(g.ids, g.dist, g.flags, total, k, b.offN, b.offO, b.fillN, b.fillO, b.revN,
                                      b.revO);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int wpb = 4;
    const unsigned wb = (unsigned)cdivll(N, wpb);
    {
        LaunchScope ls("k_rev_select", s);
        k_rev_select<<<wb, wpb * 32, (size_t)wpb * rev_cap * 8, s>>>(b.offN, b.revN, N, rev_cap, b.topN, b.ntopN);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        LaunchScope ls("k_rev_select", s);
        k_rev_select<<<wb, wpb * 32, (size_t)wpb * rev_cap * 8, s>>>(b.offO, b.revO, N, rev_cap, b.topO, b.ntopO);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        LaunchScope ls("k_build_cands", s);
        int hs = 64;   // hash set of the ids offered, at most half full
        while (hs < 2 * b.cmax) hs <<= 1;
        k_build_cands<<<wb, wpb * 32, (size_t)wpb * (b.cmax + hs) * 4, s>>>(g.ids, g.flags, N, k, b.topN, b.ntopN,
                                                                            b.topO, b.ntopO, rev_cap, b.cand, b.nn,
                                                                            b.no, b.cmax, hs);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The worst key of every list, (delta, id) of entry k - 1 or the empty key (8 bytes per vertex:
// the Update kernels read one per candidate, and the array stays in L2)
__global__ void k_worst_keys(const int32_t* __restrict__ ids, const float* __restrict__ dist, long long N, int k,
                             uint64_t* __restrict__ wk) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    const int32_t w = ids[v * k + k - 1];
    wk[v] = w < 0 ? kEmptyKey : mkkey(dist[v * k + k - 1], w);
}

// ---------------------------------------------------------------------------- Update
constexpr int kJThreads = 256;

__device__ __forceinline__ int jhash(int32_t id, int hs) { return (int)((((uint32_t)id * 2654435761u) >> 12) & (hs - 1)); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int sz = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// barrier of the 64 threads of one tile group (ids 1..4; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int grp) { asm volatile("bar.sync %0, 64;\n" ::"r"(grp + 1) : "memory"); }

// ---- Update kernel: every candidate row and list of v in shared memory, 32 x 32 tiles.
// The register tile forms FP32 distances in its own summation order; they only filter.
// A pair survives for direction a <- b when b is not in list(a) and its tile distance,
// lowered by the rounding margin between two FP32 orders (fp32_pair_margin), can still
// beat list(a)'s worst key. Survivors are re-ranked by the tile's thread group with the
// canonical distance (transpose reduction over 32 pairs) and proposed only when their
// exact key beats the worst key. Proposals gather in shared memory and leave the CTA
// with one global reservation.
constexpr int kST = 32;          // tile edge
constexpr int kSGroups = 4;      // tile groups of 64 threads
constexpr int kSQueue = kST * kST;
constexpr int kPropBuf = 512;    // proposals buffered per CTA

struct StagedLayout {
    int thr, cid, csh, cinv, nrm, hk, hv, mask, lists, rows, queue, pbuf_tgt, pbuf_key, misc, bytes, hs, words;
};

__host__ __device__ inline StagedLayout staged_layout(int cm, int k, int d) {
    StagedLayout l;
    int hs = 64;
    while (hs < 2 * cm) hs <<= 1;
    l.hs = hs;
    l.words = (cm + 31) >> 5;
    auto a16 = [](int x) { return (x + 15) & ~15; };
    int o = 0;
    l.thr = o;
    o += a16(cm * 8);
    l.pbuf_key = o;
    o += kPropBuf * 8;
    l.cid = o;
    o += a16(cm * 4);
    l.csh = o;
    o += a16(cm * 4);
    l.cinv = o;
    o += a16(cm * 4);
    l.nrm = o;
    o += a16(cm * 4);
    l.hk = o;
    o += hs * 4;
    l.hv = o;
    o += hs * 4;
    l.mask = o;
    o += a16(cm * l.words * 4);
    l.queue = o;
    o += kSGroups * kSQueue * 4;
    l.pbuf_tgt = o;
    o += kPropBuf * 4;
    l.misc = o;
    o += 64;
    l.lists = o;
    l.rows = o;
    o += cm * (d + 4) * 4;
    l.bytes = o;
    return l;
}

// out[0] = largest |C| and out[1] = largest |C_n| among the vertices that have pairs
// STAGE: the candidates' rows are copied to shared memory (stride d + 4); otherwise (sets of
// wide rows that do not fit) every read goes to the FP32 rows in global memory, mostly served
// by L2 (the same values, so the same distances).
template <int METRIC, bool STAGE>
__global__ void __launch_bounds__(kJThreads, 2) k_join_staged(
    ShardTable t, const float* __restrict__ X, const float* __restrict__ inv_norm, int k,
    const int32_t* __restrict__ ids, const float* __restrict__ dist, const int32_t* __restrict__ cand,
    const int32_t* __restrict__ nn_arr, const int32_t* __restrict__ no_arr, int cmax, int cm,
    const int32_t* __restrict__ vlist, int32_t* __restrict__ prop_tgt, uint64_t* __restrict__ prop_key,
    unsigned long long* prop_count, long long prop_cap, uint8_t* __restrict__ pending,
    unsigned long long* pairs_count, unsigned long long* cands_count, int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const long long v = vlist ? (long long)vlist[blockIdx.x] : (long long)blockIdx.x;
    const int nn = nn_arr[v];
    const int nc = nn + no_arr[v];
    if (nn == 0 || nc < 2) return;
    if (nc > cm) {   // the host sized shared memory for the largest set; never expected
        if (tid == 0) atomicOr(status, kErrBounds);
        return;
    }
    const int d = t.dim;
    const StagedLayout L = staged_layout(cm, k, STAGE ? d : 0);
    uint64_t* thr = reinterpret_cast<uint64_t*>(smem + L.thr);
    int32_t* cid = reinterpret_cast<int32_t*>(smem + L.cid);
    int32_t* csh = reinterpret_cast<int32_t*>(smem + L.csh);
    float* cinv = reinterpret_cast<float*>(smem + L.cinv);
    float* nrm = reinterpret_cast<float*>(smem + L.nrm);
    int32_t* hk = reinterpret_cast<int32_t*>(smem + L.hk);
    int32_t* hv = reinterpret_cast<int32_t*>(smem + L.hv);
    uint32_t* mask = reinterpret_cast<uint32_t*>(smem + L.mask);
    float* rows = reinterpret_cast<float*>(smem + L.rows);
    uint32_t* queue = reinterpret_cast<uint32_t*>(smem + L.queue);
    int32_t* pb_tgt = reinterpret_cast<int32_t*>(smem + L.pbuf_tgt);
    uint64_t* pb_key = reinterpret_cast<uint64_t*>(smem + L.pbuf_key);
    int* misc = reinterpret_cast<int*>(smem + L.misc);   // [0] proposals buffered, [1..4] queue sizes
    const int W = L.words, hs = L.hs, stride = d + 4;
    const int vq = d >> 2;
    const float eps = fp32_pair_margin(d);
    // row r of the candidate set: staged copy or the FP32 row itself
    auto rowp = [&](int r) -> const float* { return STAGE ? rows + r * stride : X + (long long)cid[r] * d; };

    for (int i = tid; i < nc; i += kJThreads) cid[i] = cand[v * cmax + i];
    for (int i = tid; i < hs; i += kJThreads) hk[i] = -1;
    for (int i = tid; i < nc * W; i += kJThreads) mask[i] = 0u;
    if (tid < 16) misc[tid] = 0;
    __syncthreads();
    if (STAGE)
        for (int item = tid; item < nc * vq; item += kJThreads) {
            const int r = item / vq, c = item - (item / vq) * vq;
            cp_async16(rows + r * stride + c * 4, X + (long long)cid[r] * d + c * 4, true);
        }
    cp_async_commit();
    for (int i = tid; i < nc; i += kJThreads) {
        const int32_t c = cid[i];
        csh[i] = shard_of(t, c);
        const int32_t wi = ids[(long long)c * k + k - 1];
        thr[i] = wi < 0 ? kEmptyKey : mkkey(dist[(long long)c * k + k - 1], wi);
        cinv[i] = (METRIC == FGIM_COSINE) ? inv_norm[c] : 1.f;
        int slot = jhash(c, hs);
        for (int probe = 0; probe < hs; ++probe) {
            if (atomicCAS(hk + slot, -1, c) == -1) {
                hv[slot] = i;
                break;
            }
            slot = (slot + 1) & (hs - 1);
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    // membership bits: bit (i, j) set when C[j] is already in list(C[i]); list entries are
    // read from global memory eight at a time per thread so the loads overlap
    {
        const int total = nc * k;
        for (int base = tid * 8; base < total; base += kJThreads * 8) {
            int32_t e8[8];
#pragma unroll
            for (int u8 = 0; u8 < 8; ++u8) {
                const int idx = base + u8;
                e8[u8] = idx < total ? ids[(long long)cid[idx / k] * k + (idx - (idx / k) * k)] : -1;
            }
#pragma unroll
            for (int u8 = 0; u8 < 8; ++u8) {
                const int32_t e = e8[u8];
                if (e < 0) continue;
                const int i = (base + u8) / k;
                int slot = jhash(e, hs);
                for (int probe = 0; probe < hs; ++probe) {
                    const int32_t h = hk[slot];
                    if (h == e) {
                        const int j = hv[slot];
                        atomicOr(mask + i * W + (j >> 5), 1u << (j & 31));
                        break;
                    }
                    if (h == -1) break;
                    slot = (slot + 1) & (hs - 1);
                }
            }
        }
    }
    if (METRIC == FGIM_IP)
        for (int i = tid; i < nc; i += kJThreads) {
            float ss = 0.f;
            for (int c = 0; c < d; ++c) ss = fmaf(rowp(i)[c], rowp(i)[c], ss);
            nrm[i] = sqrtf(ss) * 1.0001f;
        }
    __syncthreads();

    const int grp = tid >> 6;
    const int gt = tid & 63;
    const int tx = gt & 7, ty = gt >> 3;
    uint32_t* gq = queue + grp * kSQueue;
    int* gqn = misc + 1 + grp;
    const int RT = (nn + kST - 1) / kST, CT = (nc + kST - 1) / kST;
    unsigned long long my_pairs = 0;
    int tile_no = 0;
    for (int rt = 0; rt < RT; ++rt) {
        for (int ct = 0; ct < CT; ++ct) {
            const int r0 = rt * kST, c0 = ct * kST;
            if (min(c0 + kST, nc) - 1 <= r0) continue;     // no pair with j > i
            const bool mine = (tile_no++ % kSGroups) == grp;
            if (!mine) continue;
            float acc[4][4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[a][b][q] = 0.f;
            const float* ar[4];
            const float* br[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) ar[a] = rowp(min(r0 + ty + 8 * a, nc - 1));
#pragma unroll
            for (int b = 0; b < 4; ++b) br[b] = rowp(min(c0 + tx + 8 * b, nc - 1));
            for (int c = 0; c < vq; ++c) {
                float4 av[4], bv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) av[a] = *reinterpret_cast<const float4*>(ar[a] + c * 4);
#pragma unroll
                for (int b = 0; b < 4; ++b) bv[b] = *reinterpret_cast<const float4*>(br[b] + c * 4);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        if (METRIC == FGIM_L2SQ) {
                            const float e0 = av[a].x - bv[b].x, e1 = av[a].y - bv[b].y;
                            const float e2 = av[a].z - bv[b].z, e3 = av[a].w - bv[b].w;
                            acc[a][b][0] = fmaf(e0, e0, acc[a][b][0]);
                            acc[a][b][1] = fmaf(e1, e1, acc[a][b][1]);
                            acc[a][b][2] = fmaf(e2, e2, acc[a][b][2]);
                            acc[a][b][3] = fmaf(e3, e3, acc[a][b][3]);
                        } else {
                            acc[a][b][0] = fmaf(av[a].x, bv[b].x, acc[a][b][0]);
                            acc[a][b][1] = fmaf(av[a].y, bv[b].y, acc[a][b][1]);
                            acc[a][b][2] = fmaf(av[a].z, bv[b].z, acc[a][b][2]);
                            acc[a][b][3] = fmaf(av[a].w, bv[b].w, acc[a][b][3]);
                        }
                    }
            }
            // filter: queue (i, j, directions) of the pairs that may pass
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int i = r0 + ty + 8 * a;
                    const int j = c0 + tx + 8 * b;
                    if (!(i < nn && j < nc && j > i && csh[i] != csh[j])) continue;
                    ++my_pairs;
                    const float s = (acc[a][b][0] + acc[a][b][1]) + (acc[a][b][2] + acc[a][b][3]);
                    float lo;   // lower bound of the canonical distance
                    if (METRIC == FGIM_L2SQ) lo = s - eps * s;
                    else if (METRIC == FGIM_IP) lo = (1.f - s) - eps * nrm[i] * nrm[j];
                    else lo = (1.f - s * cinv[i] * cinv[j]) - 2.f * eps;
                    unsigned dm = 0;
                    if (!((mask[i * W + (j >> 5)] >> (j & 31)) & 1u) &&
                        (thr[i] == kEmptyKey || lo <= key_dist(thr[i])))
                        dm |= 1u;
                    if (!((mask[j * W + (i >> 5)] >> (i & 31)) & 1u) &&
                        (thr[j] == kEmptyKey || lo <= key_dist(thr[j])))
                        dm |= 2u;
                    if (dm) {
                        const int slot = atomicAdd(gqn, 1);
                        gq[slot] = (uint32_t)i | ((uint32_t)j << 10) | (dm << 20);
                    }
                }
            group_sync(grp);
            // re-rank the queued pairs with the canonical distance (one pair per warp step)
            const int nq = *gqn;
            const int gw = gt >> 5;   // warp within the group
            for (int qi = gw; qi < nq; qi += 2) {
                const uint32_t e = gq[qi];
                const int i = e & 1023, j = (e >> 10) & 1023;
                const unsigned dm = (e >> 20) & 3u;
                const float sc = warp_butterfly(lane_part<METRIC>(reinterpret_cast<const float4*>(rowp(i)),
                                                                  reinterpret_cast<const float4*>(rowp(j)), vq, lane));
                if (lane < 2 && ((dm >> lane) & 1u)) {
                    const float dd = delta_finish<METRIC>(sc, METRIC == FGIM_COSINE ? __fmul_rn(cinv[i], cinv[j]) : 1.f);
                    const int a = lane == 0 ? i : j, b = lane == 0 ? j : i;
                    const uint64_t key = mkkey(dd, cid[b]);
                    if (key < thr[a]) {
                        const int slot = atomicAdd(misc, 1);
                        if (slot < kPropBuf) {
                            pb_tgt[slot] = cid[a];
                            pb_key[slot] = key;
                        } else {
                            const unsigned long long pos = atomicAdd(prop_count, 1ull);
                            if (pos < (unsigned long long)prop_cap) {
                                prop_tgt[pos] = cid[a];
                                prop_key[pos] = key;
                            } else {
                                pending[v] = 1;
                                atomicOr(status, kErrOverflow);
                            }
                        }
                    }
                }
            }
            group_sync(grp);
            if (gt == 0) *gqn = 0;
            group_sync(grp);
        }
    }
    __syncthreads();
    // buffered proposals leave with one reservation
    const int nb = min(misc[0], kPropBuf);
    __shared__ unsigned long long base_s;
    if (tid == 0 && nb > 0) base_s = atomicAdd(prop_count, (unsigned long long)nb);
    __syncthreads();
    if (nb > 0) {
        const unsigned long long base = base_s;
        for (int i = tid; i < nb; i += kJThreads) {
            const unsigned long long pos = base + i;
            if (pos < (unsigned long long)prop_cap) {
                prop_tgt[pos] = pb_tgt[i];
                prop_key[pos] = pb_key[i];
            } else {
                pending[v] = 1;
                atomicOr(status, kErrOverflow);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_pairs += __shfl_xor_sync(kFull, my_pairs, o);
    if (lane == 0 && my_pairs) atomicAdd(pairs_count, my_pairs);
    if (threadIdx.x == 0) atomicAdd(cands_count, (unsigned long long)nc);
}

// ---- tensor-core filter (BF16 tcgen05 Gram tile), exact FP32 re-rank
//
// Per vertex v the candidate rows (BF16 copies) are staged in shared memory (K-major,
// 128-byte swizzle) and one 128 x N x d tcgen05.mma tile (FP32 accumulation in TMEM) gives
// D_ij ~ x_i . x_j for every pair of C_n x C. The filter value is
//   L2: n2_i + n2_j - 2 D_ij,  IP: 1 - D_ij,  cosine: 1 - D_ij * inv_i * inv_j,
// and a pair direction survives when the value minus a bound on its error can still beat
// the target's worst key. The bound (Cauchy-Schwarz on the BF16 conversion errors e = bf(x)
// - x, plus the FP32 accumulation and rounding terms of Higham's bound with g = (d + 16) u):
//   |D - x_i.x_j| <= |e_i||x_j| + |x_i||e_j| + |e_i||e_j| + g (|x_i| + |e_i|)(|x_j| + |e_j|).
// On integer-valued data the conversion is exact (e = 0) and the bound is tiny. Survivors are
// re-ranked with the canonical FP32 distance (from the staged rows when every one of them
// converted exactly, else from the FP32 rows); only exact keys are proposed.
constexpr int kTCThreads = 128;    // threads of the FP32-row variant (byte rows: 256)
constexpr int kTCQueue = 1024;     // filter survivors in flight per CTA (each warp re-ranks its share when full)
constexpr int kTCPropBuf = 256;    // proposals buffered per CTA
constexpr int kTCKChunk = 128;     // dimensions staged per K chunk of the Gram tile


__global__ void k_prep_bf16(const float* __restrict__ X, long long N, int d, __nv_bfloat16* __restrict__ Xb,
                            float4* __restrict__ tcm) {
    const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= N) return;
    const float* x = X + row * d;
    __nv_bfloat16* xb = Xb + row * d;
    float s = 0.f, se = 0.f;
    bool inexact = false;
    for (int c = lane; c < d; c += 32) {
        const float v = x[c];
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        xb[c] = b;
        const float e = __bfloat162float(b) - v;
        inexact |= e != 0.f;
        s = fmaf(v, v, s);
        se = fmaf(e, e, se);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(kFull, s, o);
        se += __shfl_xor_sync(kFull, se, o);
    }
    inexact = __any_sync(kFull, inexact);
    if (lane == 0) {
        // |e| == 0 exactly when the BF16 row equals the FP32 row; squares of conversion errors
        // below 2^-75 can underflow, so an inexact row never reports less than 1e-18
        const float en = inexact ? fmaxf(sqrtf(se) * 1.0001f, 1e-18f) : 0.f;
        tcm[row] = make_float4(s, sqrtf(s) * 1.0001f, en, 0.f);
    }
}

// FP8 E4M3 rows with one scale per vector: s = amax |x| / 448 (1 for an all-zero row),
// q = saturating round-to-nearest E4M3 of x / s; the MMA forms sum q_a q_b and the filter takes
// s_a s_b times it. tcm = (|x|^2, bound on |x|, bound on |x - s q|, s); the conversion error is
// what the filter's bound is built from (every row counts as inexact).
__global__ void k_prep_fp8(const float* __restrict__ X, long long N, int d, __nv_fp8_storage_t* __restrict__ Xq,
                           float4* __restrict__ tcm) {
    const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= N) return;
    const float* x = X + row * d;
    float amax = 0.f;
    for (int c = lane; c < d; c += 32) amax = fmaxf(amax, fabsf(x[c]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(kFull, amax, o));
    const float sc = amax > 0.f ? amax / 448.f : 1.f;
    __nv_fp8_storage_t* xq = Xq + row * d;
    float s = 0.f, se = 0.f;
    for (int c = lane; c < d; c += 32) {
        const float v = x[c];
        const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(v / sc, __NV_SATFINITE, __NV_E4M3);
        xq[c] = q;
        const float dq = __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3)));
        const float e = fmaf(-sc, dq, v);   // v - s q, one rounding
        s = fmaf(v, v, s);
        se = fmaf(e, e, se);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(kFull, s, o);
        se += __shfl_xor_sync(kFull, se, o);
    }
    if (lane == 0) tcm[row] = make_float4(s, sqrtf(s) * 1.0001f, fmaxf(sqrtf(se) * 1.001f, 1e-18f), sc);
}

cudaError_t launch_prep_fp8(const float* X, long long N, int d, uint8_t* Xq, float4* tcm, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    LaunchScope ls("k_prep_fp8", s);
    k_prep_fp8<<<(unsigned)cdivll(N * 32, 256), 256, 0, s>>>(X, N, d, reinterpret_cast<__nv_fp8_storage_t*>(Xq), tcm);
    return cudaGetLastError();
}

cudaError_t launch_prep_bf16(const float* X, long long N, int d, __nv_bfloat16* Xb, float4* tcm, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    LaunchScope ls("k_prep_bf16", s);
    k_prep_bf16<<<(unsigned)cdivll(N * 32, 256), 256, 0, s>>>(X, N, d, Xb, tcm);
    return cudaGetLastError();
}

// Tile row of candidate i for candidate sets of up to 128: candidates i = 4 m + q go to TMEM
// lane quarter q (row 32 q + m), so every lane quarter holds an even share of the new and old
// candidates and the warps of the four quarters get similar work. The columns of D follow
// the same order (both MMA operands are the one staged tile); the inverse is the same formula.
__host__ __device__ __forceinline__ int tc_row(int i) { return 32 * (i & 3) + (i >> 2); }
__host__ __device__ __forceinline__ int tc_cand(int row) { return 4 * (row & 31) + (row >> 5); }

// Shared memory of one k_join_tc CTA (offsets from the first 1024-byte boundary of the
// dynamic shared memory; `bytes` includes the slack for that alignment).
struct TCLayout {
    int op, rows_alloc, dpad, meta, colf, thr, pb_key, cid, hkv, mask, queue, pb_tgt, misc, bytes, hs, words;
};

__host__ __device__ inline TCLayout tc_layout(int cm, int d) {
    TCLayout l;
    int hs = 64;   // id -> index table, load factor <= 1/4: two probes find nearly every key
    while (hs < 4 * cm) hs <<= 1;
    l.hs = hs;
    const int npad = ((cm + 15) / 16) * 16;
    // membership bits per TMEM lane row in TMEM column order: 128 columns (interleaved order) or npad
    l.words = cm <= 128 ? 4 : (npad + 31) >> 5;
    // rows per panel (a multiple of 8: whole swizzle atoms); sets of up to 128 candidates are
    // staged in the quarter-interleaved row order (tc_row), which spans all 128 rows
    l.rows_alloc = cm <= 128 ? 128 : npad;
    // K is staged in chunks of at most kTCKChunk dimensions (whole 128-byte panels, zero beyond d);
    // the MMAs of successive chunks accumulate in TMEM, so d is not limited by shared memory
    l.dpad = ((d + 63) / 64) * 64;
    if (l.dpad > kTCKChunk) l.dpad = kTCKChunk;
    auto a16 = [](int x) { return (x + 15) & ~15; };
    int o = 0;
    l.op = o;
    o += l.rows_alloc * l.dpad * 2;   // a multiple of 1024
    l.meta = o;
    o += cm * 16;
    l.colf = o;
    o += cm * 16;
    l.thr = o;
    o += a16(cm * 8);
    l.pb_key = o;
    o += kTCPropBuf * 8;
    l.cid = o;
    o += a16(cm * 4);
    l.hkv = o;
    o += hs * 8;
    l.mask = o;   // two bit matrices (directions A and B), min(cm, 128) rows of `words` words
    o += 2 * (cm < 128 ? cm : 128) * l.words * 4;
    l.queue = o;
    o += kTCQueue * 4;
    l.pb_tgt = o;
    o += kTCPropBuf * 4;
    l.misc = o;
    o += 64;
    // The A operand spans 128 rows of every panel even when fewer are staged: rows past the
    // staged ones read whatever follows (the next panel, the arrays above) and only produce
    // rows of D that are never used. Keep all of it inside the allocation.
    const int a_end = (l.dpad / 64 - 1) * l.rows_alloc * 128 + 128 * 128;
    l.bytes = (o > a_end ? o : a_end) + 1024;
    return l;
}

// One CTA per vertex v (vlist[blockIdx.x]); C_n = the first nn candidates, C = all nc.
// FP8: the staged operand holds E4M3 rows with one scale per vector (k_prep_fp8) instead of BF16
// rows; each Gram entry is then scaled by the two vectors' scales, the filter's bound takes their
// conversion errors, and the re-rank always reads the FP32 rows.
template <int METRIC, bool BYTES, bool LARGE, bool FP8>
__global__ void __launch_bounds__(BYTES ? 256 : 128, 4) k_join_tc(
    ShardTable t, const float* __restrict__ X, const __nv_bfloat16* __restrict__ Xb, const uint8_t* __restrict__ X8,
    const float4* __restrict__ tcm, const float* __restrict__ inv_norm, int k, const int32_t* __restrict__ ids,
    const uint64_t* __restrict__ wk, const int32_t* __restrict__ cand, const int32_t* __restrict__ nn_arr, const int32_t* __restrict__ no_arr, int cmax,
    int cm, uint32_t tmem_cols, const int32_t* __restrict__ vlist, int32_t* __restrict__ prop_tgt,
    uint64_t* __restrict__ prop_key, unsigned long long* prop_count, long long prop_cap, uint8_t* __restrict__ pending,
    unsigned long long* pairs_count, unsigned long long* cands_count, int* status) {
    constexpr int NT = BYTES ? 256 : 128;   // threads (byte rows: eight warps, two per TMEM lane quarter)
    constexpr int NW = NT / 32;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const long long v = vlist ? (long long)vlist[blockIdx.x] : (long long)blockIdx.x;
    const int nn = nn_arr[v];
    const int nc = nn + no_arr[v];
    // candidate ids, read before nc is known (a row of cand holds cmax >= cm entries)
    const long long crow = v * (long long)cmax;
    const int32_t cA = tid < cm ? cand[crow + tid] : -1;
    const int32_t cB = tid + NT < cm ? cand[crow + tid + NT] : -1;
    if (nn == 0 || nc < 2) return;
    if (nc > cm || nn > 128 || cm > 2 * NT || (!LARGE && cm > 128)) {   // the host sized the launch
        if (tid == 0) atomicOr(status, kErrBounds);
        return;
    }
    const int d = t.dim;
    const int du = FP8 ? d / 2 : d;   // row length in 2-byte staging units (an E4M3 pair per unit)
    const TCLayout L = tc_layout(cm, du);
    unsigned char* op = smem + L.op;
    float4* meta = reinterpret_cast<float4*>(smem + L.meta);   // n2, |x| bound, |e| bound, cosine 1/|x|
    float4* colf = reinterpret_cast<float4*>(smem + L.colf);   // P, worst distance, shard (bits), -
    uint64_t* thr = reinterpret_cast<uint64_t*>(smem + L.thr);
    int32_t* cid = reinterpret_cast<int32_t*>(smem + L.cid);
    int2* hkv = reinterpret_cast<int2*>(smem + L.hkv);   // (candidate id or -1, its index)
    uint32_t* mask = reinterpret_cast<uint32_t*>(smem + L.mask);
    uint32_t* queue = reinterpret_cast<uint32_t*>(smem + L.queue);
    int32_t* pb_tgt = reinterpret_cast<int32_t*>(smem + L.pb_tgt);
    uint64_t* pb_key = reinterpret_cast<uint64_t*>(smem + L.pb_key);
    // misc: [0] proposals buffered, [2] rows whose BF16 copy is inexact,
    // [4..5] base of this CTA's proposals in the global buffer; mbarrier at byte 32, TMEM
    // address at byte 48, the byte rows' mbarrier at byte 56
    int* misc = reinterpret_cast<int*>(smem + L.misc);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.misc + 32);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc + 48);
    // byte rows of the re-rank: completes when every thread's copies of them have landed
    uint64_t* rows_bar = reinterpret_cast<uint64_t*>(smem + L.misc + 56);
    const int W = L.words, hs = L.hs, rows = L.rows_alloc;
    const int vq = d >> 2;           // float4 chunks per FP32 row
    const int kc = du >> 3;          // 16-byte chunks per staged (BF16 or E4M3) row
    const int kcp = L.dpad >> 3;     // 16-byte chunks per staged row
    const int npad = ((nc + 15) / 16) * 16;   // MMA N
    const int kcp_sh = (kcp & (kcp - 1)) == 0 ? __ffs(kcp) - 1 : -1;   // shift for / kcp when a power of two
    const int nch = (kc + kcp - 1) / kcp;   // K chunks
    const float g = (float)(d + 16) * 5.9604645e-8f;
    // squared L2 on exactly converted rows: lo = P_i + P_j - 2 D_ij with P = (1 - Cf) |x|^2
    // lies below (value - bound) of the general test (see the filter)
    const float Cf = 1.2f * (4.001f * g + 12.01f * 5.9604645e-8f);

    if (tid < nc) cid[tid] = cA;
    if (tid + NT < nc) cid[tid + NT] = cB;
    for (int i = tid; i < hs; i += NT) hkv[i] = make_int2(-1, -1);
    const int mrows = cm < 128 ? cm : 128;
    uint32_t* maskB = mask + mrows * W;
    for (int i = tid; i < 2 * mrows * W; i += NT) mask[i] = 0u;
    if (tid < 8) misc[tid] = 0;
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        tc::mbar_init(rows_bar, NT);
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, tmem_cols);
    __syncthreads();
    // One round trip for everything the candidate ids address: the BF16 rows (cp.async; rows
    // past nc are never used, their products land in ignored rows and columns of D; chunks
    // past d are zero), this thread's candidates' worst keys and row statistics, and the
    // first batch of list entries for the membership bits.
    auto stage = [&](int ch) {   // K chunk ch: 16-byte pieces ch * kcp .. ch * kcp + kcp - 1 of every row
        for (int item = tid; item < nc * kcp; item += NT) {
            const int r = kcp_sh >= 0 ? item >> kcp_sh : item / kcp;
            const int c = item - r * kcp;
            const int gc = ch * kcp + c;
            unsigned char* dst = op + tc::sw_offset(LARGE ? r : tc_row(r), c, rows);
            if (gc < kc) cp_async16(dst, Xb + (long long)cid[r] * du + gc * 8, true);
            else *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
        }
        cp_async_commit();
    };
    stage(0);
    uint64_t wkA = kEmptyKey, wkB = kEmptyKey;
    float invA = 1.f, invB = 1.f;
    float4 mA = make_float4(0.f, 0.f, 0.f, 0.f), mB = mA;
    if (tid < nc) {
        wkA = wk[cA];
        mA = tcm[cA];
        if (METRIC == FGIM_COSINE) invA = inv_norm[cA];
    }
    if (tid + NT < nc) {
        wkB = wk[cB];
        mB = tcm[cB];
        if (METRIC == FGIM_COSINE) invB = inv_norm[cB];
    }
    // membership items: 16 bytes (four entries) of a list when rows are 16-byte aligned, else one entry
    const bool vec = (k & 3) == 0 && (reinterpret_cast<uintptr_t>(ids) & 15u) == 0;
    const int per = vec ? (k >> 2) : k;
    const int mtotal = nc * per;
    const int per_sh = (per & (per - 1)) == 0 ? __ffs(per) - 1 : -1;
    // items are read kMB ahead through a rotating set of registers: the loop body (and its
    // hash probes) exists once in the code, and kMB loads per thread stay in flight
    constexpr int kMB = 4;
    auto load_item = [&](int idx) -> int4 {
        int4 r4 = make_int4(-1, -1, -1, -1);
        if (idx < mtotal) {
            const int i = per_sh >= 0 ? idx >> per_sh : idx / per;
            const int32_t* row = ids + (long long)cid[i] * k;
            if (vec) r4 = reinterpret_cast<const int4*>(row)[idx - i * per];
            else r4.x = row[idx - i * per];
        }
        return r4;
    };
    int4 e4[kMB];
#pragma unroll
    for (int u = 0; u < kMB; ++u) e4[u] = load_item(tid + u * NT);
    auto insert = [&](int32_t c, int i) {
        int slot = jhash(c, hs);
        for (int probe = 0; probe < hs; ++probe) {
            if (atomicCAS(&hkv[slot].x, -1, c) == -1) {
                hkv[slot].y = i;
                return;
            }
            slot = (slot + 1) & (hs - 1);
        }
    };
    if (tid < nc) insert(cA, tid);
    if (tid + NT < nc) insert(cB, tid + NT);
    __syncthreads();
    auto put_meta = [&](int i, int32_t c, uint64_t wkey, float4 m, float inv) {
        thr[i] = wkey;
        if (m.z != 0.f) atomicOr(misc + 2, 1);
        colf[i] = make_float4((1.f - Cf) * m.x, wkey == kEmptyKey ? __int_as_float(0x7f800000) : key_dist(wkey),
                              __int_as_float(shard_of(t, c)), FP8 ? m.w : 0.f);   // w: the E4M3 scale
        m.w = inv;
        meta[i] = m;
    };
    if (tid < nc) put_meta(tid, cA, wkA, mA, invA);
    if (tid + NT < nc) put_meta(tid + NT, cB, wkB, mB, invB);
    // membership bits, per TMEM lane row a and TMEM column c of candidate b (col(b)):
    //   A (mask):  bit (a, col(b)) = C[b] in N(C[a])  (a's list already holds b)
    //   B (maskB): bit (a, col(b)) = C[a] in N(C[b])  (b's list already holds a)
    // so the filter reads the bits of 16 consecutive columns with one shared-memory load.
    // List entry C[j] of N(C[i]) sets A (i, col(j)) and B (j, col(i)). The lookup is straight-line: the key's home
    // slot and the next one hold it (or an empty slot) for nearly every key at load <= 1/4, so
    // the lanes of a warp stay together; a warp takes the probing loop only if one of its lanes
    // met two other keys.
    auto member = [&](int i, int32_t e) {
        const int s0 = jhash(e, hs);
        const int2 p0 = hkv[s0], p1 = hkv[(s0 + 1) & (hs - 1)];
        int j = -1;
        bool slow = false;
        if (e >= 0) {
            if (p0.x == e) j = p0.y;
            else if (p1.x == e) j = p1.y;
            else slow = p0.x != -1 && p1.x != -1;
        }
        if (__any_sync(kFull, slow) && slow) {
            int slot = (s0 + 2) & (hs - 1);
            for (int probe = 2; probe < hs; ++probe) {
                const int2 pp = hkv[slot];
                if (pp.x == e) {
                    j = pp.y;
                    break;
                }
                if (pp.x == -1) break;
                slot = (slot + 1) & (hs - 1);
            }
        }
        if (j >= 0) {
            const int cj = LARGE ? j : tc_row(j), ci = LARGE ? i : tc_row(i);
            if (!LARGE || i < 128) atomicOr(mask + i * W + (cj >> 5), 1u << (cj & 31));
            if (!LARGE || j < 128) atomicOr(maskB + j * W + (ci >> 5), 1u << (ci & 31));
        }
    };
    // warp-uniform trip count (lanes past the end carry -1 entries), so the warp votes above
    // always see all 32 lanes
#pragma unroll 1
    for (int it = tid - lane; it < mtotal; it += NT) {
        const int idx = it + lane;
        const int4 cur = e4[0];
#pragma unroll
        for (int u = 0; u + 1 < kMB; ++u) e4[u] = e4[u + 1];
        e4[kMB - 1] = load_item(idx + kMB * NT);
        const int i = per_sh >= 0 ? idx >> per_sh : idx / per;
        member(i, cur.x);
        if (vec) {
            member(i, cur.y);
            member(i, cur.z);
            member(i, cur.w);
        }
    }
    cp_async_wait<0>();
    tc::fence_async_smem();
    tc::fence_mbar_init();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    // every row converted exactly to BF16 and the whole row fits one staged chunk: the re-rank
    // may read the staged tile instead of the FP32 rows
    const bool exact = !FP8 && misc[2] == 0 && nch == 1;
    const bool exact_rows = !FP8 && misc[2] == 0;
    bool ok_mma = true;
    for (int ch = 0; ch < nch && ok_mma; ++ch) {
        if (ch > 0) {
            // the previous chunk's MMAs have completed (every thread saw its barrier phase), so
            // the tile may be overwritten
            stage(ch);
            cp_async_wait<0>();
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
        }
        if (tid == 0) {
            const uint32_t idesc = FP8 ? tc::idesc_e4m3(128, LARGE ? npad : 128) : tc::idesc_bf16(128, LARGE ? npad : 128);
            const uint32_t base = tc::smem_u32(op);
            for (int s = 0; s < L.dpad / 16; ++s) {   // 32 bytes of every row per MMA
                const uint64_t desc = tc::smem_desc_sw128(base + (uint32_t)((s >> 2) * rows * 128 + (s & 3) * 32));
                if (FP8) tc::mma_e4m3(tmem, desc, desc, idesc, (ch > 0 || s > 0) ? 1u : 0u);
                else tc::mma_bf16(tmem, desc, desc, idesc, (ch > 0 || s > 0) ? 1u : 0u);
            }
            tc::commit_to(mbar);
        }
        ok_mma = __syncthreads_and(tc::mbar_wait(mbar, (uint32_t)(ch & 1), 1 << 24)) != 0;
        tc::fence_after_sync();
    }
    if (!ok_mma && tid == 0) atomicOr(status, kErrTimeout);
    // byte rows: the MMAs have read the BF16 tile, so its space takes the byte rows of the
    // candidates for the exact re-rank
    // (the copies run under the filter: each warp waits on rows_bar before its first re-rank)
    const int brs = d + 16;
    if (BYTES && ok_mma) {
        const int c16 = d >> 4;
        for (int item = tid; item < nc * c16; item += NT) {
            const int r = item / c16, c = item - r * c16;
            cp_async16(op + r * brs + c * 16, X8 + (long long)cid[r] * d + c * 16, true);
        }
        cp_async_commit();
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(tc::smem_u32(rows_bar)) : "memory");
    }
    bool rows_ready = !BYTES;

    // Filter. A pair survives when lo, a lower bound of its exact value, can still beat the
    // worst key of a list it is not already in. General test: lo = value - bound with the
    // bound of the file comment (cs term: e_i x_j + e_j (x_i + e_i) + g (x_i + e_i)(x_j + e_j)).
    // Squared L2 on exactly converted rows (e = 0): with s2 = n2_i + n2_j, 2 x_i x_j <= 1.0002 s2
    // and |D| <= (1 + g) x_i x_j, the general bound is at most 1.1 s2 (4.001 g + 12.01 u); Cf
    // adds margin for the rounding of P_i + P_j - 2 D, so lo = P_i + P_j - 2 D is lower still.
    //
    // Pairs are {i, j} with i < nn (new) and i < j < nc. Both MMA operands are the staged
    // tile, so D is symmetric and the lane of TMEM row r (candidate a) evaluates the pairs
    // {b, a} with b < min(a, nn) from its own row; with more than 128 candidates (natural row
    // order) the pairs with j >= 128 (no TMEM lane) are evaluated by lane i at columns
    // 128 .. nc - 1. Every pair is evaluated once.
    const int r = 32 * (warp & 3) + lane;   // TMEM lane quarter warp % 4
    const int a = LARGE ? r : tc_cand(r);    // this lane's candidate
    const bool r_ok = a < nc;
    const float4 fr = r_ok ? colf[a] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float Pr = fr.x, tdr = fr.y, sr = fr.w;
    const int shr = r_ok ? __float_as_int(fr.z) : -1;
    const float4 mr = r_ok ? meta[a] : make_float4(0.f, 0.f, 0.f, 1.f);
    const float n2r = mr.x, xr = mr.y, er = mr.z, cr = mr.w;
    const float xer = xr + er;
    const bool fast = METRIC == FGIM_L2SQ && (BYTES || exact_rows);
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long my_pairs = 0;
    // TMEM address of this warp's lane quarter
    auto trow_of = [&](int w) -> uint32_t { return tmem + ((uint32_t)(32 * (w & 3)) << 16); };
    // lo, a lower bound of the exact value of pair {a, b}, from its Gram entry
    auto lower = [&](int b, float dot, const float4& cc) -> float {
        if (FP8) dot = dot * (sr * cc.w);   // sum q_a q_b -> s_a s_b sum q_a q_b (two roundings, in the bound)
        if (fast) return fmaf(-2.f, dot, Pr + cc.x);
        const float4 mc = meta[b];
        const float cs = er * mc.y + mc.z * xer + g * xer * (mc.y + mc.z);
        float val, bound;
        if (METRIC == FGIM_L2SQ) {
            const float s2 = n2r + mc.x;
            val = s2 - 2.f * dot;
            bound = 1.1f * (2.f * cs + g * s2 + (2.f * 5.9604645e-8f + g) * fabsf(val) +
                            4.f * 5.9604645e-8f * (s2 + 2.f * fabsf(dot)));
        } else if (METRIC == FGIM_IP) {
            val = 1.f - dot;
            bound = 1.1f * (cs + g * fabsf(val)) + 2.4e-7f;
        } else {
            const float ccv = cr * mc.w;
            val = 1.f - dot * ccv;
            bound = 1.1f * (cs * ccv + g * fabsf(val)) + 4.8e-7f;
        }
        return val - bound;
    };
    // survivors go to this warp's own segment of the queue (a register count, no atomics)
    const int seg = kTCQueue / NW;
    uint32_t* wq = queue + warp * seg;
    int qn = 0;
    auto append = [&](int c, unsigned dm) {
        const unsigned vote = __ballot_sync(kFull, dm != 0u);
        if (dm) {
            const int slot = qn + __popc(vote & lt);
            if (slot < seg) wq[slot] = (uint32_t)a | ((uint32_t)c << 10) | (dm << 20);
        }
        qn += __popc(vote);
    };

    // Exact re-rank of this warp's survivors (no wait for the other warps) with the canonical
    // FP32 distance, kStep pairs per step; lane t < U proposes for pair t.
    //  - byte rows (integer coordinates in [0, 255], d <= 128, d % 16 == 0): every partial sum
    //    of the canonical FP32 value is an integer below 2^24, so it equals the exact integer
    //    |a|^2 + |b|^2 - 2 a.b; one pair per lane, from the byte rows that replace the BF16
    //    tile in shared memory once the MMAs are done (row stride d + 16 bytes: the rows of a
    //    warp's pairs fall in different banks).
    //  - otherwise the canonical FP32 additions, from the staged tile when every staged row is
    //    exact (the same values), else from the FP32 rows in global memory.
    constexpr int kStep = BYTES ? 32 : 8;
    auto rerank = [&](int nq) {
        if (BYTES && !rows_ready && nq > 0) {   // bounded wait for the byte rows (every lane)
            if (!tc::mbar_wait(rows_bar, 0u, 1 << 24)) atomicOr(status, kErrTimeout);
            rows_ready = true;
        }
        for (int q0 = 0; q0 < nq; q0 += kStep) {
            const int U = min(kStep, nq - q0);
            float sc = 0.f;
            if constexpr (BYTES) {
                // one pair per lane, both byte rows from the copy staged in shared memory
                if (lane < U) {
                    const uint32_t e = wq[q0 + lane];
                    const uint4* pa = reinterpret_cast<const uint4*>(op + (e & 1023u) * brs);
                    const uint4* pb = reinterpret_cast<const uint4*>(op + ((e >> 10) & 1023u) * brs);
                    // four independent chains (integer sums: any order gives the same total)
                    uint32_t d0 = 0u, d1 = 0u, d2 = 0u, d3 = 0u;
                    for (int c = 0; c < (d >> 4); ++c) {
                        const uint4 x = pa[c], y = pb[c];
                        d0 = __dp4a(x.x, y.x, d0);
                        d1 = __dp4a(x.y, y.y, d1);
                        d2 = __dp4a(x.z, y.z, d2);
                        d3 = __dp4a(x.w, y.w, d3);
                    }
                    const uint32_t dot = (d0 + d1) + (d2 + d3);
                    if (METRIC == FGIM_L2SQ) {
                        const uint32_t na = __float2uint_rn(meta[e & 1023u].x);
                        const uint32_t nb = __float2uint_rn(meta[(e >> 10) & 1023u].x);
                        sc = (float)(na + nb - 2u * dot);
                    } else {
                        sc = (float)dot;
                    }
                }
            } else {
                int ra[8], rb[8];
#pragma unroll
                for (int t8 = 0; t8 < 8; ++t8) {
                    const uint32_t e = wq[q0 + min(t8, U - 1)];
                    ra[t8] = (int)(e & 1023u);
                    rb[t8] = (int)((e >> 10) & 1023u);
                }
                float acc[8][4];
#pragma unroll
                for (int t8 = 0; t8 < 8; ++t8) acc[t8][0] = acc[t8][1] = acc[t8][2] = acc[t8][3] = 0.f;
                for (int c = lane; c < vq; c += 32) {
                    float4 xa[8], xb[8];
                    if (exact) {
#pragma unroll
                        for (int t8 = 0; t8 < 8; ++t8) {
                            const uint2 ua =
                                *reinterpret_cast<const uint2*>(op + tc::sw_offset(LARGE ? ra[t8] : tc_row(ra[t8]), c >> 1, rows) + (c & 1) * 8);
                            const uint2 ub =
                                *reinterpret_cast<const uint2*>(op + tc::sw_offset(LARGE ? rb[t8] : tc_row(rb[t8]), c >> 1, rows) + (c & 1) * 8);
                            xa[t8] = make_float4(__uint_as_float(ua.x << 16), __uint_as_float(ua.x & 0xffff0000u),
                                                 __uint_as_float(ua.y << 16), __uint_as_float(ua.y & 0xffff0000u));
                            xb[t8] = make_float4(__uint_as_float(ub.x << 16), __uint_as_float(ub.x & 0xffff0000u),
                                                 __uint_as_float(ub.y << 16), __uint_as_float(ub.y & 0xffff0000u));
                        }
                    } else {
#pragma unroll
                        for (int t8 = 0; t8 < 8; ++t8) {
                            xa[t8] = reinterpret_cast<const float4*>(X + (long long)cid[ra[t8]] * d)[c];
                            xb[t8] = reinterpret_cast<const float4*>(X + (long long)cid[rb[t8]] * d)[c];
                        }
                    }
#pragma unroll
                    for (int t8 = 0; t8 < 8; ++t8) {
                        const float4 x = xa[t8], y = xb[t8];
                        if (METRIC == FGIM_L2SQ) {
                            const float e0 = __fsub_rn(x.x, y.x), e1 = __fsub_rn(x.y, y.y);
                            const float e2 = __fsub_rn(x.z, y.z), e3 = __fsub_rn(x.w, y.w);
                            acc[t8][0] = fmaf(e0, e0, acc[t8][0]);
                            acc[t8][1] = fmaf(e1, e1, acc[t8][1]);
                            acc[t8][2] = fmaf(e2, e2, acc[t8][2]);
                            acc[t8][3] = fmaf(e3, e3, acc[t8][3]);
                        } else {
                            acc[t8][0] = fmaf(x.x, y.x, acc[t8][0]);
                            acc[t8][1] = fmaf(x.y, y.y, acc[t8][1]);
                            acc[t8][2] = fmaf(x.z, y.z, acc[t8][2]);
                            acc[t8][3] = fmaf(x.w, y.w, acc[t8][3]);
                        }
                    }
                }
#pragma unroll
                for (int t8 = 0; t8 < 8; ++t8) {
                    const float tot = warp_butterfly(__fadd_rn(__fadd_rn(acc[t8][0], acc[t8][1]),
                                                               __fadd_rn(acc[t8][2], acc[t8][3])));
                    if (lane == t8) sc = tot;
                }
            }
            // proposals: one shared-memory atomic per warp and direction
            uint64_t key[2] = {kEmptyKey, kEmptyKey};
            int32_t tgt[2] = {-1, -1};
            if (lane < U) {
                const uint32_t e = wq[q0 + lane];
                const int ia = (int)(e & 1023u), jb = (int)((e >> 10) & 1023u);
                const unsigned dm = (e >> 20) & 3u;
                const float dd =
                    delta_finish<METRIC>(sc, METRIC == FGIM_COSINE ? __fmul_rn(meta[ia].w, meta[jb].w) : 1.f);
#pragma unroll
                for (int dir = 0; dir < 2; ++dir) {
                    const int a2 = dir == 0 ? ia : jb, b2 = dir == 0 ? jb : ia;
                    const uint64_t kk = mkkey(dd, cid[b2]);
                    if (((dm >> dir) & 1u) && kk < thr[a2]) {
                        key[dir] = kk;
                        tgt[dir] = cid[a2];
                    }
                }
            }
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
                const bool has_p = tgt[dir] >= 0;
                const unsigned vote = __ballot_sync(kFull, has_p);
                if (vote == 0u) continue;
                const int leader = __ffs(vote) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(misc, __popc(vote));
                base = __shfl_sync(kFull, base, leader);
                if (has_p) {
                    const int slot = base + __popc(vote & lt);
                    if (slot < kTCPropBuf) {
                        pb_tgt[slot] = tgt[dir];
                        pb_key[slot] = key[dir];
                    } else {
                        const unsigned long long pos = atomicAdd(prop_count, 1ull);
                        if (pos < (unsigned long long)prop_cap) {
                            prop_tgt[pos] = tgt[dir];
                            prop_key[pos] = key[dir];
                        } else {
                            pending[v] = 1;
                            atomicOr(status, kErrOverflow);
                        }
                    }
                }
            }
        }
    };
    // Filter, one block of 16 TMEM columns at a time: every lane tests its pairs of the block
    // in registers (lo against the worst keys, cross-shard, valid pair) and keeps two bit masks
    // of directions (bit j: column j; A: a's list may take b, B: b's list may take a), minus the
    // membership bits of the block; only the survivors go to the warp's queue segment, which is
    // re-ranked and emptied whenever fewer than 32 slots are left, and once more at the end.
    // c0: first column, jn: columns in the block (warp-uniform), b0 + bstep j: candidate of
    // column c0 + j, vm: this lane's valid pairs.
    auto block = [&](int c0, int jn, int b0, int bstep, unsigned vm) {
        float dv[16];
        tc::tmem_ld16(trow_of(warp) + (uint32_t)c0, dv);
        unsigned dA = 0u, dB = 0u, xs = 0u;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j >= jn) break;
            const int b = b0 + bstep * j;
            const float4 cc = colf[b];
            const float lo = lower(b, dv[j], cc);
            const bool xsh = shr != __float_as_int(cc.z);
            if (xsh) xs |= 1u << j;
            if (xsh && lo <= tdr) dA |= 1u << j;
            if (xsh && lo <= cc.y) dB |= 1u << j;
        }
        my_pairs += __popc(xs & vm);
        if (r_ok) {   // drop the directions whose list already holds the other candidate
            const int wo = a * W + (c0 >> 5), sh = c0 & 16;
            dA &= ~(mask[wo] >> sh);
            dB &= ~(maskB[wo] >> sh);
        }
        dA &= vm;
        dB &= vm;
        unsigned sv = dA | dB;
        while (__any_sync(kFull, sv != 0u)) {
            if (qn > seg - 32) {
                rerank(qn);
                qn = 0;
            }
            unsigned dm = 0u;
            int b = 0;
            if (sv) {
                const int j = __ffs(sv) - 1;
                sv &= sv - 1;
                b = b0 + bstep * j;
                dm = ((dA >> j) & 1u) | (((dB >> j) & 1u) << 1);
            }
            append(b, dm);
        }
    };
    if (ok_mma) {
        // Column ranges. Interleaved order (up to 128 candidates): range rg = columns
        // 32 rg + m', m' < |{b < nn : b % 4 = rg}|, candidate b = 4 m' + rg; lane (a = 4 lane + q)
        // pairs with b < a, i.e. m' < lane + [rg < q]. Natural order: columns b < min(nn, 32 q + 31)
        // with b < a, then, for lanes of new candidates, columns 128 .. nc - 1. The NW / 4 warps
        // of a lane quarter take every (NW / 4)-th block of the quarter's ranges.
        // Within a range the blocks go round-robin over those warps, starting one warp further on
        // in each range, so the short last blocks of the ranges land on different warps.
        const int q = warp & 3;
        const int hw = warp >> 2;
        int rot = 0;
        auto run = [&](int cbase, int ccount, int bbase, int bstep, int lim) {
            int gb = rot++;
            for (int t0 = 0; t0 < ccount; t0 += 16, ++gb) {
                if (gb % (NW / 4) != hw) continue;
                const int nvp = min(max(lim - t0, 0), 16);
                block(cbase + t0, min(16, ccount - t0), bbase + bstep * t0, bstep,
                      nvp >= 16 ? 0xFFFFu : (1u << nvp) - 1u);
            }
        };
        if (LARGE) {
            const int cend0 = min(nn, 32 * q + 31);
            run(0, cend0, 0, 1, r_ok ? min(a, cend0) : 0);
            if (32 * q < nn) run(128, nc - 128, 128, 1, a < nn ? nc - 128 : 0);
        } else {
#pragma unroll 1
            for (int rg = 0; rg < 4; ++rg) {
                const int cnt = nn > rg ? (nn - rg + 3) >> 2 : 0;
                run(32 * rg, cnt, rg, 4, r_ok ? min(cnt, lane + (rg < q ? 1 : 0)) : 0);
            }
        }
        rerank(qn);
        qn = 0;
    }
    cp_async_wait<0>();   // no copy of this thread may still be writing shared memory at exit
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
    const int nb = min(misc[0], kTCPropBuf);
    unsigned long long* base_s = reinterpret_cast<unsigned long long*>(misc + 4);
    if (tid == 0 && nb > 0) *base_s = atomicAdd(prop_count, (unsigned long long)nb);
    __syncthreads();
    if (nb > 0) {
        const unsigned long long base = *base_s;
        for (int q = tid; q < nb; q += NT) {
            const unsigned long long pos = base + q;
            if (pos < (unsigned long long)prop_cap) {
                prop_tgt[pos] = pb_tgt[q];
                prop_key[pos] = pb_key[q];
            } else {
                pending[v] = 1;
                atomicOr(status, kErrOverflow);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_pairs += __shfl_xor_sync(kFull, my_pairs, o);
    if (lane == 0 && my_pairs) atomicAdd(pairs_count, my_pairs);
    if (tid == 0) atomicAdd(cands_count, (unsigned long long)nc);
}

// ---------------------------------------------------------------------------- Update, few new candidates
// A vertex whose C_n is small has few pairs to join (about |C_n| x |C|), while the tile form
// above pays for every candidate's list (the membership bits) and the staging regardless. Such
// vertices join one warp per vertex on byte rows, one lane per pair: lane j holds the row of
// C[j] in registers, the rows of C_n sit in shared memory (every lane reads the same one at a
// time), and every cross-graph pair {C[i], C[j]} (i < |C_n|, i < j < |C|) gets its exact
// distance straight away (no filter). A direction proposes when its key beats the list's
// worst key and the list does not hold the other vertex yet; both membership tests are bits
// per (i, j), found from the new candidates' own lists:
//   A (C[j] in list(C[i])): the entries of list(C[i]) looked up in a hash of C;
//   B (C[i] in list(C[j])): the reverse list of C[i] (the Visit step's, every u whose list
//      holds C[i]) looked up the same way. The lists have not changed since Visit in the first
//      run of a pass, so this form joins only there (a re-run after a proposal overflow reads
//      merged lists and goes to the tile form).
// The pairs, their distances (the exact integer values of the canonical FP32 sums, as in the
// tile form's re-rank) and the proposal rule are the tile form's, so the proposals are the same.
// A warp's global reads come in a few batches whose loads are all issued before any is used
// (candidates; their worst keys and rows; list entries and reverse-list bounds; reverse-list
// entries; the rows of each chunk of 32 candidates): one vertex is a chain of dependent reads.
constexpr int kSparseWarps = 4;
constexpr int kSparseBatch = 8;   // loads a lane keeps in flight in the list rounds

// Shared memory of one warp of k_join_sparse (byte offsets; cm = largest |C|, nnm = largest
// |C_n| of the launch, d = row bytes).
struct SparseLayout {
    int cthr, rbN, rbO, hkv, qrows, cid, csh, cinv, q2, rmN, rpre, memA, memB, bytes, hs, W;
};

__host__ __device__ inline SparseLayout sparse_layout(int cm, int nnm, int d) {
    SparseLayout l;
    int hs = 64;   // id -> index table, at most half full
    while (hs < 2 * cm) hs <<= 1;
    l.hs = hs;
    l.W = (cm + 31) >> 5;   // bit words per membership row
    auto a16 = [](int x) { return (x + 15) & ~15; };
    int o = 0;
    l.cthr = o;    // worst key of list(C[j])
    o += a16(cm * 8);
    l.rbN = o;     // start of the new / old reverse segment of C[i]
    o += a16(nnm * 8);
    l.rbO = o;
    o += a16(nnm * 8);
    l.hkv = o;     // (candidate id or -1, its index)
    o += hs * 8;
    l.qrows = o;   // byte rows of C_n (d is a multiple of 16)
    o += nnm * d;
    l.cid = o;
    o += a16(cm * 4);
    l.csh = o;     // graph of C[j]
    o += a16(cm * 4);
    l.cinv = o;    // 1 / |C[j]| (cosine)
    o += a16(cm * 4);
    l.q2 = o;      // |C[i]|^2 of the new candidates
    o += a16(nnm * 4);
    l.rmN = o;     // length of the new reverse segment of C[i]
    o += a16(nnm * 4);
    l.rpre = o;    // reverse entries of C[0 .. i) (new and old), nn + 1 of them
    o += a16((nnm + 1) * 4);
    l.memA = o;    // bit (i, j): C[j] in list(C[i])
    o += nnm * l.W * 4;
    l.memB = o;    // bit (i, j): C[i] in list(C[j])
    o += nnm * l.W * 4;
    l.bytes = a16(o);
    return l;
}

template <int METRIC>
__global__ void __launch_bounds__(kSparseWarps * 32, 8) k_join_sparse(
    ShardTable t, const uint8_t* __restrict__ X8, const float* __restrict__ inv_norm, int k,
    const int32_t* __restrict__ ids, const uint64_t* __restrict__ wk, const uint64_t* __restrict__ revN,
    const long long* __restrict__ offN, const uint64_t* __restrict__ revO, const long long* __restrict__ offO,
    const int32_t* __restrict__ cand, const int32_t* __restrict__ nn_arr, const int32_t* __restrict__ no_arr,
    int cmax, int cm, int nnm, const int32_t* __restrict__ vlist, long long nv, int32_t* __restrict__ prop_tgt,
    uint64_t* __restrict__ prop_key, unsigned long long* prop_count, long long prop_cap,
    uint8_t* __restrict__ pending, unsigned long long* pairs_count, unsigned long long* cands_count, int* status) {
    extern __shared__ __align__(16) unsigned char smem_sp[];
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const long long w = (long long)blockIdx.x * kSparseWarps + warp;
    if (w >= nv) return;
    const long long v = vlist[w];
    // read batch 1: the candidate row (read up to cm <= cmax entries before |C| is known) and the sizes
    const long long crow = v * (long long)cmax;
    int32_t cl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) cl[u] = 32 * u + lane < cm ? cand[crow + 32 * u + lane] : -1;
    const int nn = nn_arr[v];
    const int nc = nn + no_arr[v];
    if (nn == 0 || nc < 2) return;
    const int d = t.dim;
    if (nc > cm || nn > nnm || cm > 128 || (d & 15) != 0 || d > 128) {   // the host sized the launch
        if (lane == 0) atomicOr(status, kErrBounds);
        return;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (32 * u + lane >= nc) cl[u] = -1;
    const SparseLayout L = sparse_layout(cm, nnm, d);
    unsigned char* base = smem_sp + (size_t)warp * L.bytes;
    uint64_t* cthr = reinterpret_cast<uint64_t*>(base + L.cthr);
    long long* rbN = reinterpret_cast<long long*>(base + L.rbN);
    long long* rbO = reinterpret_cast<long long*>(base + L.rbO);
    int2* hkv = reinterpret_cast<int2*>(base + L.hkv);
    unsigned char* qrows = base + L.qrows;
    int32_t* cid = reinterpret_cast<int32_t*>(base + L.cid);
    int32_t* csh = reinterpret_cast<int32_t*>(base + L.csh);
    float* cinv = reinterpret_cast<float*>(base + L.cinv);
    uint32_t* q2s = reinterpret_cast<uint32_t*>(base + L.q2);
    int32_t* rmN = reinterpret_cast<int32_t*>(base + L.rmN);
    int32_t* rpre = reinterpret_cast<int32_t*>(base + L.rpre);
    uint32_t* memA = reinterpret_cast<uint32_t*>(base + L.memA);
    uint32_t* memB = reinterpret_cast<uint32_t*>(base + L.memB);
    const int hs = L.hs, W = L.W;
    const int c16 = d >> 4;   // 16-byte chunks per row
    // shifts for / c16 and / k when they are powers of two (the usual case), else -1
    const int c16_sh = (c16 & (c16 - 1)) == 0 ? __ffs(c16) - 1 : -1;
    const int k_sh = (k & (k - 1)) == 0 ? __ffs(k) - 1 : -1;
    const unsigned lt = (1u << lane) - 1u;
    for (int s = lane; s < hs; s += 32) hkv[s] = make_int2(-1, -1);
    for (int s = lane; s < 2 * nnm * W; s += 32) memA[s] = 0u;   // memB follows memA
    __syncwarp();
    // read batch 2: the candidates' worst keys
    uint64_t wl[4];
    float il[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        wl[u] = kEmptyKey;
        il[u] = 1.f;
        if (cl[u] >= 0) {
            wl[u] = wk[cl[u]];
            if (METRIC == FGIM_COSINE) il[u] = inv_norm[cl[u]];
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int j = 32 * u + lane;
        if (j >= nc) continue;
        const int32_t c = cl[u];
        cid[j] = c;
        csh[j] = shard_of(t, c);
        cthr[j] = wl[u];
        cinv[j] = il[u];
        int slot = jhash(c, hs);
        for (int p = 0; p < hs; ++p) {
            if (atomicCAS(&hkv[slot].x, -1, c) == -1) {
                hkv[slot].y = j;
                break;
            }
            slot = (slot + 1) & (hs - 1);
        }
    }
    __syncwarp();
    auto lookup = [&](int32_t x) -> int {   // index of x in C, or -1
        int slot = jhash(x, hs);
        for (int p = 0; p < hs; ++p) {
            const int2 kv = hkv[slot];
            if (kv.x == x) return kv.y;
            if (kv.x == -1) return -1;
            slot = (slot + 1) & (hs - 1);
        }
        return -1;
    };
    // read batch 3, all issued before any is used: the rows of C_n (copied to shared memory
    // asynchronously), the reverse-segment bounds of C_n, and the entries of the lists of C_n
    for (int it = lane; it < nn * c16; it += 32) {
        const int i = c16_sh >= 0 ? it >> c16_sh : it / c16, c = it - i * c16;
        cp_async16(qrows + i * d + 16 * c, X8 + (long long)cid[i] * d + 16 * c, true);
    }
    cp_async_commit();
    long long obn = 0, oen = 0, obo = 0, oeo = 0;   // bounds of C[lane] (the first 32 of C_n)
    if (lane < nn) {
        const int32_t ci = cid[lane];
        obn = offN[ci];
        oen = offN[ci + 1];
        obo = offO[ci];
        oeo = offO[ci + 1];
    }
    {
        const int total = nn * k;
        for (int b0 = 0; b0 < total; b0 += 32 * kSparseBatch) {
            int32_t x[kSparseBatch];
            int xi[kSparseBatch];
#pragma unroll
            for (int u = 0; u < kSparseBatch; ++u) {
                const int it = b0 + 32 * u + lane;
                x[u] = -1;
                xi[u] = 0;
                if (it < total) {
                    const int i = k_sh >= 0 ? it >> k_sh : it / k;
                    x[u] = ids[(long long)cid[i] * k + (it - i * k)];
                    xi[u] = i;
                }
            }
#pragma unroll
            for (int u = 0; u < kSparseBatch; ++u) {
                if (x[u] < 0) continue;
                const int j = lookup(x[u]);
                if (j >= 0) atomicOr(memA + xi[u] * W + (j >> 5), 1u << (j & 31));   // A bits
            }
        }
    }
    {
        int carry = 0;
        for (int i0 = 0; i0 < nn; i0 += 32) {
            const int i = i0 + lane;
            int cnt = 0;
            if (i < nn) {
                if (i0 > 0) {
                    const int32_t ci = cid[i];
                    obn = offN[ci];
                    oen = offN[ci + 1];
                    obo = offO[ci];
                    oeo = offO[ci + 1];
                }
                rbN[i] = obn;
                rbO[i] = obo;
                rmN[i] = (int)(oen - obn);
                cnt = (int)(oen - obn + oeo - obo);
            }
            int inc = cnt;   // inclusive prefix over the lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc += y;
            }
            if (i < nn) rpre[i] = carry + inc - cnt;
            carry += __shfl_sync(kFull, inc, 31);
        }
        if (lane == 0) rpre[nn] = carry;
    }
    __syncwarp();
    // read batch 4: the reverse-list entries of C_n, all at once (B bits)
    {
        const int total = rpre[nn];
        for (int b0 = 0; b0 < total; b0 += 32 * kSparseBatch) {
            int32_t x[kSparseBatch];
            int xi[kSparseBatch];
#pragma unroll
            for (int u = 0; u < kSparseBatch; ++u) {
                const int f = b0 + 32 * u + lane;
                x[u] = -1;
                xi[u] = 0;
                if (f < total) {
                    int lo = 0, hi = nn - 1;   // the i with rpre[i] <= f < rpre[i + 1]
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (rpre[mid] <= f) lo = mid;
                        else hi = mid - 1;
                    }
                    const int s = f - rpre[lo];
                    const uint64_t key = s < rmN[lo] ? revN[rbN[lo] + s] : revO[rbO[lo] + (s - rmN[lo])];
                    x[u] = key_id(key);
                    xi[u] = lo;
                }
            }
#pragma unroll
            for (int u = 0; u < kSparseBatch; ++u) {
                if (x[u] < 0) continue;
                const int j = lookup(x[u]);
                if (j >= 0) atomicOr(memB + xi[u] * W + (j >> 5), 1u << (j & 31));
            }
        }
    }
    cp_async_wait<0>();
    __syncwarp();
    if (METRIC == FGIM_L2SQ) {
        for (int i = lane; i < nn; i += 32) {
            const uint4* q = reinterpret_cast<const uint4*>(qrows + i * d);
            uint32_t s = 0u;
            for (int c = 0; c < c16; ++c) {
                const uint4 x = q[c];
                s = __dp4a(x.x, x.x, s);
                s = __dp4a(x.y, x.y, s);
                s = __dp4a(x.z, x.z, s);
                s = __dp4a(x.w, x.w, s);
            }
            q2s[i] = s;
        }
        __syncwarp();
    }
    uint32_t my_pairs = 0;
    for (int j0 = 0; j0 < nc; j0 += 32) {
        const int j = j0 + lane;
        const bool hj = j < nc;
        // this lane's row C[j] in registers, and |C[j]|^2
        uint4 xr[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
            xr[c] = (hj && c < c16) ? *reinterpret_cast<const uint4*>(X8 + (long long)cid[j] * d + 16 * c)
                                    : make_uint4(0u, 0u, 0u, 0u);
        uint32_t x2 = 0u;
        if (METRIC == FGIM_L2SQ) {
            uint32_t e0 = 0u, e1 = 0u, e2 = 0u, e3 = 0u;   // integer sums: any order, the same total
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                e0 = __dp4a(xr[c].x, xr[c].x, e0);
                e1 = __dp4a(xr[c].y, xr[c].y, e1);
                e2 = __dp4a(xr[c].z, xr[c].z, e2);
                e3 = __dp4a(xr[c].w, xr[c].w, e3);
            }
            x2 = (e0 + e1) + (e2 + e3);
        }
        const int32_t cj = hj ? cid[j] : -1;
        const int shj = hj ? csh[j] : -1;
        const uint64_t thrj = hj ? cthr[j] : 0ull;
        const float invj = (METRIC == FGIM_COSINE && hj) ? cinv[j] : 1.f;
        const int wj = j0 >> 5;
        const int ilim = min(nn, j0 + 31);   // a pair needs i < j <= j0 + 31
        for (int i = 0; i < ilim; ++i) {
            const bool valid = hj && i < j && csh[i] != shj;   // cross-graph pairs only
            if (!__any_sync(kFull, valid)) continue;
            my_pairs += valid ? 1u : 0u;
            const uint4* q = reinterpret_cast<const uint4*>(qrows + i * d);
            uint32_t e0 = 0u, e1 = 0u, e2 = 0u, e3 = 0u;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c < c16) {
                    const uint4 y = q[c];
                    e0 = __dp4a(y.x, xr[c].x, e0);
                    e1 = __dp4a(y.y, xr[c].y, e1);
                    e2 = __dp4a(y.z, xr[c].z, e2);
                    e3 = __dp4a(y.w, xr[c].w, e3);
                }
            }
            const uint32_t dot = (e0 + e1) + (e2 + e3);
            float dd;
            if (METRIC == FGIM_L2SQ) {
                dd = (float)(q2s[i] + x2 - 2u * dot);   // |a|^2 + |b|^2 - 2 a.b, an integer below 2^24
            } else {
                const float inv = METRIC == FGIM_COSINE ? __fmul_rn(cinv[i], invj) : 1.f;
                dd = delta_finish<METRIC>((float)dot, inv);
            }
            const int32_t ci = cid[i];
            const uint64_t kA = mkkey(dd, cj), kB = mkkey(dd, ci);
            const bool pA = valid && kA < cthr[i] && !((memA[i * W + wj] >> lane) & 1u);
            const bool pB = valid && kB < thrj && !((memB[i * W + wj] >> lane) & 1u);
            const unsigned va = __ballot_sync(kFull, pA), vb = __ballot_sync(kFull, pB);
            if ((va | vb) == 0u) continue;
            const int na = __popc(va);
            unsigned long long pos0 = 0;
            if (lane == 0) pos0 = atomicAdd(prop_count, (unsigned long long)(na + __popc(vb)));
            pos0 = __shfl_sync(kFull, pos0, 0);
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
                if (!(dir == 0 ? pA : pB)) continue;
                const unsigned long long pos = pos0 + (dir == 0 ? __popc(va & lt) : na + __popc(vb & lt));
                if (pos < (unsigned long long)prop_cap) {
                    prop_tgt[pos] = dir == 0 ? ci : cj;
                    prop_key[pos] = dir == 0 ? kA : kB;
                } else {
                    pending[v] = 1;
                    atomicOr(status, kErrOverflow);
                }
            }
        }
    }
    const uint32_t tot = __reduce_add_sync(kFull, my_pairs);
    if (lane == 0) {
        if (tot) atomicAdd(pairs_count, (unsigned long long)tot);
        atomicAdd(cands_count, (unsigned long long)nc);
    }
}

// Largest candidate set and C_n of the vertices in vlist (all when null), and the vertices
// split into kJoinLists lists (blist[q * cap ..]): the tensor-core launches by candidate-set
// size (|C| <= 64, <= 128, > 128), and the warp-per-vertex form (list 3) for the vertices with
// |C_n| <= sparse_nn and |C| <= kSparseMaxC. out: [0] max |C|, [1] max |C_n|, [2 + q] list sizes,
// [6 + q] max |C| per list.
constexpr int kTCLists = 3;
constexpr int kJoinLists = 4;
constexpr int kSparseMaxC = 128;
__device__ __forceinline__ int tc_list_of(int m) { return m <= 64 ? 0 : m <= 128 ? 1 : 2; }

__global__ void k_join_buckets(const int32_t* __restrict__ nn, const int32_t* __restrict__ no,
                               const int32_t* __restrict__ vlist, long long nv, int sparse_nn,
                               int32_t* __restrict__ out, int32_t* __restrict__ blist, long long cap) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int m = 0, mn = 0;
    long long v = 0;
    bool act = false;
    if (i < nv) {
        v = vlist ? vlist[i] : i;
        mn = nn[v];
        m = mn > 0 ? mn + no[v] : 0;
        act = mn > 0 && m >= 2;
    }
    const int q = (mn <= sparse_nn && m <= kSparseMaxC) ? 3 : tc_list_of(m);
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int b = 0; b < kJoinLists; ++b) {
        const bool mine = act && q == b;
        const unsigned vote = __ballot_sync(kFull, mine);
        int base = 0;
        if (lane == 0 && vote) base = atomicAdd(out + 2 + b, __popc(vote));
        base = __shfl_sync(kFull, base, 0);
        if (mine) blist[(long long)b * cap + base + __popc(vote & lt)] = (int32_t)v;
        int mb = mine ? m : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(kFull, mb, o));
        if (lane == 0 && mb > 0) atomicMax(out + 2 + kJoinLists + b, mb);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = max(m, __shfl_xor_sync(kFull, m, o));
        mn = max(mn, __shfl_xor_sync(kFull, mn, o));
    }
    if (lane == 0) {
        if (m > 0) atomicMax(out, m);
        if (mn > 0) atomicMax(out + 1, mn);
    }
}

// shared memory a k_join_tc launch asks for: its layout, raised so that no more CTAs fit on
// an SM than the 512 TMEM columns can serve at once (an allocation never has to wait)
static size_t tc_launch_smem(const TCLayout& TL, uint32_t cols) {
    const int per_sm = 233472;   // 228 KB of shared memory per SM, 1 KB of it reserved per CTA
    const int fit = (int)(512 / cols);
    const int floor_bytes = per_sm / (fit + 1) - 1024 + 16;
    return (size_t)(TL.bytes > floor_bytes ? TL.bytes : floor_bytes);
}

cudaError_t refine_join(const ShardTable& t, const float* X, const float* inv_norm, int metric, const fgim_knng& g,
                        RefineBuffers& b, const int32_t* vlist, long long nv, unsigned long long* pairs,
                        unsigned long long* cands, int* status, cudaStream_t s) {
    for (int q = 0; q < 5; ++q) b.class_count[q] = 0;
    if (nv <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    // the warp-per-vertex form works on byte rows, in the first run of a pass only (its
    // membership bits come from the reverse lists of Visit; a re-run reads merged lists)
    const bool bytes = b.X8 != nullptr && byte_rows_ok(t.dim) && !b.fp8;
    const int sparse_nn = bytes && vlist == nullptr ? std::min(b.sparse_nn, kSparseMaxC) : 0;
    constexpr int kOut = 2 + 2 * kJoinLists;
    if ((e = cudaMemsetAsync(b.max_nc, 0, kOut * sizeof(int32_t), s)) != cudaSuccess) return e;
    {
        LaunchScope ls("k_join_buckets", s);
        k_join_buckets<<<(unsigned)cdivll(nv, 256), 256, 0, s>>>(b.nn, b.no, vlist, nv, sparse_nn, b.max_nc,
                                                                  b.blist, b.blist_cap);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemcpyAsync(b.host_i32, b.max_nc, kOut * sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    int32_t hb[kOut];
    for (int q = 0; q < kOut; ++q) hb[q] = b.host_i32[q];
    const int32_t cm = hb[0], cmn = hb[1];
    if (cm < 2) return cudaSuccess;
    const int du = b.fp8 ? t.dim / 2 : t.dim;   // staged row length in 2-byte units
    bool use_tc = b.join_filter != 1 && b.Xb && du % 16 == 0 && cmn <= 128 && cm <= 256;
    if (use_tc)
        for (int q = 0; q < kTCLists; ++q)
            if (hb[2 + q] > 0 && tc_layout(hb[2 + kJoinLists + q], du).bytes > 227 * 1024) use_tc = false;
    if (use_tc) {
        {
            LaunchScope ls("k_worst_keys", s);
            k_worst_keys<<<(unsigned)cdivll(g.n, 256), 256, 0, s>>>(g.ids, g.dist, g.n, g.k, b.wk);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        for (int q = 0; q < kTCLists; ++q) {
            const int32_t count = hb[2 + q], cmq = hb[2 + kJoinLists + q];
            if (count <= 0) continue;
            b.class_count[q] += count;
            const TCLayout TL = tc_layout(cmq, du);
            const int ncols = cmq <= 128 ? 128 : ((cmq + 15) / 16) * 16;   // MMA N (interleaved order: 128)
            uint32_t cols = 32;
            while ((int)cols < ncols) cols <<= 1;
            const size_t smem = tc_launch_smem(TL, cols);
            const int32_t* list = b.blist + (long long)q * b.blist_cap;
#define FGIM_LAUNCH_TC4(MT, BY, LG, F8)                                                                           \
    do {                                                                                                          \
        e = cudaFuncSetAttribute(k_join_tc<MT, BY, LG, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                                 (int)smem);                                                                      \
        if (e != cudaSuccess) break;                                                                              \
        LaunchScope ls("k_join", s);                                                                              \
        k_join_tc<MT, BY, LG, F8><<<(unsigned)count, (BY) ? 256 : kTCThreads, smem, s>>>(                           \
            t, X, reinterpret_cast<const __nv_bfloat16*>(b.Xb), b.X8, b.tcm, inv_norm, g.k, g.ids, b.wk, b.cand,  \
            b.nn, b.no, b.cmax, cmq, cols, list, b.prop_tgt, b.prop_key, b.prop_count, b.prop_cap, b.pending,     \
            pairs, cands, status);                                                                                \
        e = cudaGetLastError();                                                                                   \
    } while (0)
#define FGIM_LAUNCH_TC3(MT, BY, LG) FGIM_LAUNCH_TC4(MT, BY, LG, false)
#define FGIM_LAUNCH_TC(MT, BY)                                                                                    \
    do {                                                                                                          \
        if (cmq > 128) FGIM_LAUNCH_TC3(MT, BY, true);                                                             \
        else FGIM_LAUNCH_TC3(MT, BY, false);                                                                      \
    } while (0)
#define FGIM_LAUNCH_TC8(MT)                                                                                       \
    do {                                                                                                          \
        if (cmq > 128) FGIM_LAUNCH_TC4(MT, false, true, true);                                                    \
        else FGIM_LAUNCH_TC4(MT, false, false, true);                                                             \
    } while (0)
            if (b.fp8) {
                if (metric == FGIM_L2SQ) FGIM_LAUNCH_TC8(FGIM_L2SQ);
                else if (metric == FGIM_IP) FGIM_LAUNCH_TC8(FGIM_IP);
                else FGIM_LAUNCH_TC8(FGIM_COSINE);
            } else if (metric == FGIM_L2SQ) {
                if (bytes) FGIM_LAUNCH_TC(FGIM_L2SQ, true); else FGIM_LAUNCH_TC(FGIM_L2SQ, false);
            } else if (metric == FGIM_IP) {
                if (bytes) FGIM_LAUNCH_TC(FGIM_IP, true); else FGIM_LAUNCH_TC(FGIM_IP, false);
            } else {
                if (bytes) FGIM_LAUNCH_TC(FGIM_COSINE, true); else FGIM_LAUNCH_TC(FGIM_COSINE, false);
            }
#undef FGIM_LAUNCH_TC8
#undef FGIM_LAUNCH_TC
#undef FGIM_LAUNCH_TC3
#undef FGIM_LAUNCH_TC4
            if (e != cudaSuccess) return e;
        }
        const int32_t count = hb[2 + 3], cms = hb[2 + kJoinLists + 3];
        if (count > 0) {   // the vertices with few new candidates, one warp each
            b.class_count[4] += count;
            const int nnm = std::min(sparse_nn, (int)cms);
            const size_t smem = (size_t)kSparseWarps * sparse_layout(cms, nnm, t.dim).bytes;
            const int32_t* list = b.blist + 3LL * b.blist_cap;
            const unsigned grid = (unsigned)cdivll(count, kSparseWarps);
#define FGIM_LAUNCH_SP(MT)                                                                                        \
    do {                                                                                                          \
        e = cudaFuncSetAttribute(k_join_sparse<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
        if (e != cudaSuccess) break;                                                                              \
        LaunchScope ls("k_join_sparse", s);                                                                       \
        k_join_sparse<MT><<<grid, kSparseWarps * 32, smem, s>>>(                                                  \
            t, b.X8, inv_norm, g.k, g.ids, b.wk, b.revN, b.offN, b.revO, b.offO, b.cand, b.nn, b.no, b.cmax,      \
            cms, nnm, list, count, b.prop_tgt, b.prop_key, b.prop_count, b.prop_cap, b.pending, pairs, cands,     \
            status);                                                                                              \
        e = cudaGetLastError();                                                                                   \
    } while (0)
            if (metric == FGIM_L2SQ) FGIM_LAUNCH_SP(FGIM_L2SQ);
            else if (metric == FGIM_IP) FGIM_LAUNCH_SP(FGIM_IP);
            else FGIM_LAUNCH_SP(FGIM_COSINE);
#undef FGIM_LAUNCH_SP
        }
        return e;
    }
    // the rows are staged when they fit the shared memory of a CTA, otherwise read from global memory
    const bool stage = staged_layout(cm, g.k, t.dim).bytes <= 227 * 1024;
    const StagedLayout SL = staged_layout(cm, g.k, stage ? t.dim : 0);
    if (SL.bytes > 227 * 1024) return cudaErrorNotSupported;
    b.class_count[3] += (long long)hb[2] + hb[3] + hb[4] + hb[5];   // the vertices with a pair to join
    const size_t smem = SL.bytes;
#define FGIM_LAUNCH_JS(MT, ST)                                                                                    \
    do {                                                                                                          \
        e = cudaFuncSetAttribute(k_join_staged<MT, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) break;                                                                              \
        LaunchScope ls("k_join", s);                                                                              \
        k_join_staged<MT, ST><<<(unsigned)nv, kJThreads, smem, s>>>(t, X, inv_norm, g.k, g.ids, g.dist, b.cand,    \
                                                                    b.nn, b.no, b.cmax, cm, vlist, b.prop_tgt,    \
                                                                    b.prop_key, b.prop_count, b.prop_cap,         \
                                                                    b.pending, pairs, cands, status);             \
        e = cudaGetLastError();                                                                                   \
    } while (0)
    if (stage) {
        if (metric == FGIM_L2SQ) FGIM_LAUNCH_JS(FGIM_L2SQ, true);
        else if (metric == FGIM_IP) FGIM_LAUNCH_JS(FGIM_IP, true);
        else FGIM_LAUNCH_JS(FGIM_COSINE, true);
    } else {
        if (metric == FGIM_L2SQ) FGIM_LAUNCH_JS(FGIM_L2SQ, false);
        else if (metric == FGIM_IP) FGIM_LAUNCH_JS(FGIM_IP, false);
        else FGIM_LAUNCH_JS(FGIM_COSINE, false);
    }
#undef FGIM_LAUNCH_JS
    return e;
}

// ---------------------------------------------------------------------------- Merge
__global__ void k_prop_count(const int32_t* __restrict__ tgt, long long P, int32_t* __restrict__ cnt) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) atomicAdd(cnt + tgt[i], 1);
}

__global__ void k_prop_scatter(const int32_t* __restrict__ tgt, const uint64_t* __restrict__ key, long long P,
                               const long long* __restrict__ off, int32_t* __restrict__ fill,
                               uint64_t* __restrict__ sorted) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const int32_t a = tgt[i];
    const int p = atomicAdd(fill + a, 1);
    sorted[off[a] + p] = key[i];
}

// list(a) <- top-k of list(a) U proposals(a), duplicates by id removed (warp per target)
__global__ void __launch_bounds__(128) k_prop_merge(const long long* __restrict__ off,
                                                    const uint64_t* __restrict__ sorted, long long N, int k,
                                                    int32_t* __restrict__ ids, float* __restrict__ dist,
                                                    uint8_t* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const long long a = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (a >= N) return;
    const long long b = off[a], m = off[a + 1] - off[a];
    if (m == 0) return;
    uint64_t* list = reinterpret_cast<uint64_t*>(smem) + (size_t)warp * k;
    uint8_t* aux = smem + (size_t)(blockDim.x >> 5) * k * 8 + (size_t)warp * k;
    int n = 0;
    for (int s0 = 0; s0 < k; s0 += 32) {
        const int s = s0 + lane;
        bool valid = false;
        if (s < k) {
            const int32_t id = ids[a * k + s];
            valid = id >= 0;
            list[s] = valid ? mkkey(dist[a * k + s], id) : kEmptyKey;
            aux[s] = flags[a * k + s];
        }
        n += __popc(__ballot_sync(kFull, valid));
    }
    __syncwarp();
    // A proposal of an id already in the list carries the list entry's key (the distance of a
    // pair is the same wherever it is formed), so duplicates are found by key: a binary search
    // of the sorted list instead of a scan over its ids.
    for (long long c0 = 0; c0 < m; c0 += 32) {
        const uint64_t key = (c0 + lane < m) ? sorted[b + c0 + lane] : kEmptyKey;
        n = warp_merge<false>(list, aux, n, k, key, FGIM_FLAG_NEW);
    }
    for (int s = lane; s < k; s += 32) {
        if (s < n) {
            ids[a * k + s] = key_id(list[s]);
            dist[a * k + s] = key_dist(list[s]);
            flags[a * k + s] = aux[s];
        } else {
            ids[a * k + s] = -1;
            dist[a * k + s] = __int_as_float(0x7f800000);
            flags[a * k + s] = 0;
        }
    }
}

cudaError_t refine_merge(const fgim_knng& g, RefineBuffers& b, long long P, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    const long long N = g.n;
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.pcnt, 0, sizeof(int32_t) * N, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.pfill, 0, sizeof(int32_t) * N, s)) != cudaSuccess) return e;
    const unsigned gp = (unsigned)cdivll(P, 256);
    {
        LaunchScope ls("k_prop_count", s);
        k_prop_count<<<gp, 256, 0, s>>>(b.prop_tgt, P, b.pcnt);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = scan_counts(b.pcnt, N, b.poff, b.scan_tmp, b.scan_bytes, s)) != cudaSuccess) return e;
    {
        LaunchScope ls("k_prop_scatter", s);
        k_prop_scatter<<<gp, 256, 0, s>>>(b.prop_tgt, b.prop_key, P, b.poff, b.pfill, b.prop_sorted);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int wpb = 4;
    LaunchScope ls("k_prop_merge", s);
    k_prop_merge<<<(unsigned)cdivll(N, wpb), wpb * 32, (size_t)wpb * g.k * 9, s>>>(b.poff, b.prop_sorted, N, g.k,
                                                                                   g.ids, g.dist, g.flags);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- Alg. 4
__global__ void k_zero_flags(const int32_t* __restrict__ T, long long N, int32_t* __restrict__ flag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) flag[i] = T[i] == 0;
}

cudaError_t launch_zero_flags(const int32_t* T, long long N, int32_t* flag, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    LaunchScope ls("k_zero_flags", s);
    k_zero_flags<<<(unsigned)cdivll(N, 256), 256, 0, s>>>(T, N, flag);
    return cudaGetLastError();
}

__global__ void k_nonzero_u8(const uint8_t* __restrict__ v, long long N, int32_t* __restrict__ flag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) flag[i] = v[i] != 0;
}

cudaError_t launch_nonzero_flags(const uint8_t* v, long long N, int32_t* flag, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    LaunchScope ls("k_nonzero_u8", s);
    k_nonzero_u8<<<(unsigned)cdivll(N, 256), 256, 0, s>>>(v, N, flag);
    return cudaGetLastError();
}

// Alg. 4 with the result of the sequential loop over v* in ascending id, computed in
// parallel rounds. In a round every pending v* (warp per v*) works out its action on
// the current lists: the neighbour v it would use and the entry of N(v) it would
// replace. The action reads N(v*), N(v) of every neighbour tried, and T of every entry
// scanned; it writes one entry of N(v), T(v') and T(v*). All those vertex ids are
// reserved with atomicMin of the pending index. The longest ascending prefix of
// pending vertices that hold all their reservations is committed: their actions touch
// disjoint vertices, so applying them at once equals applying them one after another,
// and each was computed on the state the sequential loop would have given it. The
// rest is recomputed in the next round. The lowest pending index always holds its
// reservations, so every round commits at least one action.
enum { kPlan = 0, kCheck = 1, kCommit = 2 };

// Round rho works on the window [ff[rho - 1], min(ff[rho - 1] + W, nz)) and leaves in ff[rho]
// the first index it did not commit (the next round's start). Reservations carry a tag
// ordered by (round, index) with later rounds smaller, so owner needs no reset.
__device__ __forceinline__ unsigned long long round_tag(long long rho, long long i) {
    return ((unsigned long long)(0xFFFFFFFFu - (uint32_t)rho) << 32) | (unsigned long long)(uint32_t)i;
}

template <int MODE>
__global__ void __launch_bounds__(128) k_repair_round(int32_t* __restrict__ ids, float* __restrict__ dist,
                                                      uint8_t* __restrict__ flags, long long N, int k,
                                                      int32_t* __restrict__ T, const int32_t* __restrict__ zeros,
                                                      long long nz, long long rho, long long window,
                                                      long long* __restrict__ ff,
                                                      unsigned long long* __restrict__ owner,
                                                      unsigned long long* repaired, int* status) {
    const int warp = threadIdx.x >> 5;
    const int lane = lane_id();
    const long long start = ff[rho - 1];
    const long long wend = start + window < nz ? start + window : nz;
    if (MODE == kPlan && blockIdx.x == 0 && threadIdx.x == 0) ff[rho] = wend;
    const long long i = start + (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= wend) return;
    if (MODE == kCommit && i >= ff[rho]) return;
    const unsigned long long tag = round_tag(rho, i);
    bool ok = true;
    auto touch = [&](int32_t x) {
        if (MODE == kPlan) atomicMin(owner + x, tag);
        else if (MODE == kCheck) ok = ok && owner[x] == tag;
    };
    const long long vs = zeros[i];
    if (vs < 0 || vs >= N) {
        if (lane == 0) atomicOr(status, kErrBounds);
        return;
    }
    if (lane == 0) touch((int32_t)vs);
    int a_sel = -1, best = -1;
    int32_t v_sel = -1;
    for (int a = 0; a < k; ++a) {
        const int32_t v = ids[vs * k + a];
        if (v < 0 || v >= N) break;
        if (lane == 0) touch(v);
        // farthest entry of N(v) that is not replaced and has T > 1 (entries scanned are touched)
        int bst = -1;
        for (int r = (k - 1) >> 5; r >= 0 && bst < 0; --r) {
            const int s = r * 32 + lane;
            int32_t e = -1;
            bool el = false;
            if (s < k) {
                e = ids[(long long)v * k + s];
                el = e >= 0 && e < N && !(flags[(long long)v * k + s] & FGIM_FLAG_REPLACED) && T[e] > 1;
            }
            const unsigned m = __ballot_sync(kFull, el);
            if (m) bst = r * 32 + 31 - __clz(m);
            if (e >= 0 && e < N && (bst < 0 || s >= bst)) touch(e);
        }
        if (bst >= 0) {
            a_sel = a;
            best = bst;
            v_sel = v;
            break;
        }
    }
    if (MODE == kCheck) {
        if (__any_sync(kFull, !ok) && lane == 0) atomicMin((unsigned long long*)(ff + rho), (unsigned long long)i);
        return;
    }
    if (MODE == kCommit && best >= 0 && lane == 0) {
        int32_t* li = ids + (long long)v_sel * k;
        float* ld = dist + (long long)v_sel * k;
        uint8_t* lf = flags + (long long)v_sel * k;
        const float dvs = dist[vs * k + a_sel];
        const int32_t old = li[best];
        T[old] -= 1;
        T[vs] += 1;
        const uint64_t key = mkkey(dvs, (int32_t)vs);
        int pos = best;
        while (pos > 0 && mkkey(ld[pos - 1], li[pos - 1]) > key) {
            li[pos] = li[pos - 1];
            ld[pos] = ld[pos - 1];
            lf[pos] = lf[pos - 1];
            --pos;
        }
        while (pos + 1 < k && li[pos + 1] >= 0 && mkkey(ld[pos + 1], li[pos + 1]) < key) {
            li[pos] = li[pos + 1];
            ld[pos] = ld[pos + 1];
            lf[pos] = lf[pos + 1];
            ++pos;
        }
        li[pos] = (int32_t)vs;
        ld[pos] = dvs;
        lf[pos] = FGIM_FLAG_NEW | FGIM_FLAG_REPLACED;
        atomicAdd(repaired, 1ull);
    }
}

cudaError_t launch_repair_rounds(fgim_knng& g, int32_t* T, const int32_t* zeros, long long nz, long long rho0,
                                 int rounds, long long* ff, unsigned long long* owner, unsigned long long* repaired,
                                 int* status, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    const int wpb = 4;
    const long long window = kRepairWindow;
    const unsigned blocks = (unsigned)cdivll(window, wpb);
    for (int q = 0; q < rounds; ++q) {
        const long long rho = rho0 + q;
        LaunchScope ls("k_repair_round", s);
        k_repair_round<kPlan><<<blocks, wpb * 32, 0, s>>>(g.ids, g.dist, g.flags, g.n, g.k, T, zeros, nz, rho, window,
                                                          ff, owner, repaired, status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_repair_round<kCheck><<<blocks, wpb * 32, 0, s>>>(g.ids, g.dist, g.flags, g.n, g.k, T, zeros, nz, rho,
                                                           window, ff, owner, repaired, status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_repair_round<kCommit><<<blocks, wpb * 32, 0, s>>>(g.ids, g.dist, g.flags, g.n, g.k, T, zeros, nz, rho,
                                                            window, ff, owner, repaired, status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return e;
}

}  // namespace fgim
