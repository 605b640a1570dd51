// Alg. 1 (KNNSearch) on the GPU, shared by the cross query of Alg. 2 (k_cross.cu) and the
// evaluation / reachability searches (k_search.cu).
//
// One warp runs one beam search. The pool C (<= L keys, sorted by (delta, id)) and its
// "expanded" marks live in shared memory; each expansion reads the expanded vertex's
// adjacency row (one id per lane), drops ids already evaluated, compacts the rest, loads
// their rows coalesced (each warp load covers one row, eight rows in flight), forms the
// canonical distances of up to 32 rows with one transpose reduction, and merges them
// into the pool with warp_merge.
//
// Evaluated ids are remembered in a small direct-mapped table that may forget an id
// when another id lands on its slot (never the reverse). A forgotten id is evaluated
// again: its key equals its earlier key, so it is dropped if it is still in the pool,
// and otherwise it cannot beat the pool's worst entry (once the pool is full its worst
// key only decreases, and an id leaves the pool or is refused only when L better keys
// are present). The pool therefore evolves exactly as with an exact visited set
// (Alg. 1's "not visited" test); only the number of distance evaluations grows.
//
// Rows are read as FP32 or, when every coordinate of the data set is an integer in
// [0, 255], as one byte per coordinate (the merge checks this once). Both decode to the
// same FP32 values, so every distance, and with it every result, is the same; the byte
// rows move a quarter of the bytes, and at d = 128 a million of them fit in L2.
#pragma once
#include <algorithm>

#include "fgim_internal.cuh"
#include "fgim_launch.h"

namespace fgim {

__device__ __forceinline__ int ht_slot(int v, int bits) { return (int)(((uint32_t)v * 2654435761u) >> (32 - bits)); }

struct WarpCounters {
    long long ndc = 0;
    long long hops = 0;
};

__device__ __forceinline__ float4 u8x4_to_float4(uint32_t w) {
    return make_float4((float)(w & 0xffu), (float)((w >> 8) & 0xffu), (float)((w >> 16) & 0xffu), (float)(w >> 24));
}

// float4 chunk c (coordinates 4c .. 4c + 3) of a row of FP32, BF16 or byte storage (BF16 and
// bytes decode exactly to the FP32 values the merge works on)
__device__ __forceinline__ float4 row_chunk(const float* row, int c) { return reinterpret_cast<const float4*>(row)[c]; }
__device__ __forceinline__ float4 row_chunk(const uint16_t* row, int c) {
    const uint2 w = reinterpret_cast<const uint2*>(row)[c];
    return make_float4(__uint_as_float(w.x << 16), __uint_as_float(w.x & 0xffff0000u), __uint_as_float(w.y << 16),
                       __uint_as_float(w.y & 0xffff0000u));
}
__device__ __forceinline__ float4 row_chunk(const uint8_t* row, int c) {
    return u8x4_to_float4(*reinterpret_cast<const uint32_t*>(row + 4 * c));
}

// lane_part over a row of either storage (the same additions as lane_part)
template <int METRIC, typename RT>
__device__ __forceinline__ float lane_part_rows(const float* q, const RT* row, int nc4, int lane) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int c = lane; c < nc4; c += 32) {
        const float4 x = reinterpret_cast<const float4*>(q)[c];
        const float4 y = row_chunk(row, c);
        if (METRIC == FGIM_L2SQ) {
            const float e0 = __fsub_rn(x.x, y.x), e1 = __fsub_rn(x.y, y.y);
            const float e2 = __fsub_rn(x.z, y.z), e3 = __fsub_rn(x.w, y.w);
            s0 = fmaf(e0, e0, s0);
            s1 = fmaf(e1, e1, s1);
            s2 = fmaf(e2, e2, s2);
            s3 = fmaf(e3, e3, s3);
        } else {
            s0 = fmaf(x.x, y.x, s0);
            s1 = fmaf(x.y, y.y, s1);
            s2 = fmaf(x.z, y.z, s2);
            s3 = fmaf(x.w, y.w, s3);
        }
    }
    return __fadd_rn(__fadd_rn(s0, s1), __fadd_rn(s2, s3));
}

// The query as bytes for byte rows: this lane's 16 bytes (chunk lane % lanes-per-row) and
// the sum of the squared coordinates.
struct QBytes {
    uint4 w;
    uint32_t q2;
};

__device__ __forceinline__ uint32_t pack4(const float* v) {
    return __float2uint_rn(v[0]) | (__float2uint_rn(v[1]) << 8) | (__float2uint_rn(v[2]) << 16) |
           (__float2uint_rn(v[3]) << 24);
}

__device__ __forceinline__ QBytes query_bytes(const float* q, int d, int lane) {
    QBytes b;
    const int lpr = byte_lanes(d);
    const int part = lane & (lpr - 1);
    b.w = make_uint4(0u, 0u, 0u, 0u);
    if (part < (d >> 4)) {
        const float* c = q + 16 * part;
        b.w = make_uint4(pack4(c), pack4(c + 4), pack4(c + 8), pack4(c + 12));
    }
    uint32_t s = 0;
    for (int c = lane; c < d; c += 32) s += __float2uint_rn(q[c]) * __float2uint_rn(q[c]);
    b.q2 = __reduce_add_sync(kFull, s);
    return b;
}

// Canonical distances between the query (q in shared memory; qreg = this lane's chunk when
// d <= 128) and the U <= 32 rows base[rid[r]]; lane r receives row r's distance.
// FP32 rows load coalesced (one warp load per row, eight rows in flight); every lane stores
// its partials in P (32 x 33 floats of this warp's shared memory) and lane r re-adds row r
// in tree order.
// Byte rows (d <= 128, d % 16 == 0): every partial sum of the canonical FP32 value is then an
// integer below 128 * 255^2 < 2^24, so it is exact and the canonical value is the exact
// integer result. Lanes take 16 bytes each (32 / lanes-per-row rows per warp load) and form
// |q|^2 + |x|^2 - 2 q.x with four-way byte dot products, summed over the row's lanes.
template <int METRIC, bool SMALLD, typename RT>
__device__ __forceinline__ float rows_delta(const RT* __restrict__ base, const int32_t* rid, int U, const float* q,
                                            float4 qreg, const QBytes& qb, int d, int lane, float* P) {
    const int nc4 = d >> 2;
    if constexpr (sizeof(RT) == 1) {
        const int lpr = byte_lanes(d);
        const int rpi = 32 >> byte_lanes_log2(d);   // rows per warp load
        const int lsh = byte_lanes_log2(d), rsh = 5 - lsh;   // lpr = 1 << lsh, rpi = 1 << rsh
        const int sub = lane >> lsh, part = lane & (lpr - 1);
        const bool has = part < (d >> 4);
        // rows in batches of four warp loads (all issued before the sums)
        uint32_t mine = 0u;
        for (int t0 = 0; t0 * rpi < U; t0 += 4) {
            uint4 w[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int r = (t0 + t) * rpi + sub;
                w[t] = make_uint4(0u, 0u, 0u, 0u);
                if (r < U && has) w[t] = *reinterpret_cast<const uint4*>(base + (long long)rid[r] * d + 16 * part);
            }
            uint32_t sv[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                uint32_t sq = __dp4a(qb.w.x, w[t].x, 0u);
                sq = __dp4a(qb.w.y, w[t].y, sq);
                sq = __dp4a(qb.w.z, w[t].z, sq);
                sq = __dp4a(qb.w.w, w[t].w, sq);
                if (METRIC == FGIM_L2SQ) {
                    uint32_t sx = __dp4a(w[t].x, w[t].x, 0u);
                    sx = __dp4a(w[t].y, w[t].y, sx);
                    sx = __dp4a(w[t].z, w[t].z, sx);
                    sx = __dp4a(w[t].w, w[t].w, sx);
                    sv[t] = sx - 2u * sq;   // modulo 2^32; the row total is exact
                } else {
                    sv[t] = sq;
                }
            }
            if (lsh == 3) {
                // eight lanes per row: the four loads' partials are summed over the eight lanes
                // together (each exchange step halves the values a lane keeps), so lane part p of
                // row group s ends with the total of load p / 2, row 4 (p / 2) + s of the batch;
                // unsigned additions in any order give the same (exact) totals
                const int p = lane & 7;
                const bool b2 = (p & 4) != 0, b1 = (p & 2) != 0;
                const uint32_t keep0 = b2 ? sv[2] : sv[0], keep1 = b2 ? sv[3] : sv[1];
                const uint32_t send0 = b2 ? sv[0] : sv[2], send1 = b2 ? sv[1] : sv[3];
                const uint32_t h0 = keep0 + __shfl_xor_sync(kFull, send0, 4);
                const uint32_t h1 = keep1 + __shfl_xor_sync(kFull, send1, 4);
                uint32_t x = (b1 ? h1 : h0) + __shfl_xor_sync(kFull, b1 ? h0 : h1, 2);
                x += __shfl_xor_sync(kFull, x, 1);
                // lane r of the batch (rows 4 t0 .. 4 t0 + 15) takes row r: load r / 4 - t0, group r % 4
                const int tn = (lane >> 2) - t0;
                const uint32_t got = __shfl_sync(kFull, x, 8 * (lane & 3) + 2 * (tn & 3));
                if (tn >= 0 && tn < 4) mine = got;
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if ((t0 + t) * rpi < U) {
                        const uint32_t tot = row_group_sum(sv[t], lsh);
                        const uint32_t got = __shfl_sync(kFull, tot, (lane & (rpi - 1)) << lsh);
                        if ((lane >> rsh) == t0 + t) mine = got;
                    }
                }
            }
        }
        if (METRIC == FGIM_L2SQ) mine += qb.q2;
        return lane < U ? (float)mine : 0.f;
    } else {
        if (SMALLD) {
            const bool has = lane < nc4;
            for (int b = 0; b < U; b += 8) {
                float4 y[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int r = b + t;
                    y[t] = (r < U && has) ? row_chunk(base + (long long)rid[r] * d, lane)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int r = b + t;
                    if (r < U) P[lane * 33 + r] = has ? chunk_part<METRIC>(qreg, y[t]) : 0.f;
                }
            }
        } else {
            // wide rows: eight rows at a time, chunk by chunk (eight loads in flight per lane);
            // each row keeps the four accumulators and the chunk order of lane_part_rows
            for (int b = 0; b < U; b += 8) {
                const RT* rowp[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) rowp[t] = base + (long long)rid[b + t < U ? b + t : b] * d;
                float acc[8][4];
#pragma unroll
                for (int t = 0; t < 8; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
                for (int c = lane; c < nc4; c += 32) {
                    const float4 x = reinterpret_cast<const float4*>(q)[c];
                    float4 y[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        y[t] = b + t < U ? row_chunk(rowp[t], c) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        if (METRIC == FGIM_L2SQ) {
                            const float e0 = __fsub_rn(x.x, y[t].x), e1 = __fsub_rn(x.y, y[t].y);
                            const float e2 = __fsub_rn(x.z, y[t].z), e3 = __fsub_rn(x.w, y[t].w);
                            acc[t][0] = fmaf(e0, e0, acc[t][0]);
                            acc[t][1] = fmaf(e1, e1, acc[t][1]);
                            acc[t][2] = fmaf(e2, e2, acc[t][2]);
                            acc[t][3] = fmaf(e3, e3, acc[t][3]);
                        } else {
                            acc[t][0] = fmaf(x.x, y[t].x, acc[t][0]);
                            acc[t][1] = fmaf(x.y, y[t].y, acc[t][1]);
                            acc[t][2] = fmaf(x.z, y[t].z, acc[t][2]);
                            acc[t][3] = fmaf(x.w, y[t].w, acc[t][3]);
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (b + t < U)
                        P[lane * 33 + b + t] = __fadd_rn(__fadd_rn(acc[t][0], acc[t][1]), __fadd_rn(acc[t][2], acc[t][3]));
            }
        }
        __syncwarp();
        const float s = lane < U ? smem_tree_sum(P, lane) : 0.f;
        __syncwarp();
        return s;
    }
}

// Alg. 1 over one graph whose rows are Xt[v] / adj[v * M] for local ids v < nt. Keys carry
// global ids (local + id_off). The pool C (<= L <= 32 * MAXS keys, sorted by (delta, id))
// lives in registers: entry e = 32 s + lane is pk[s] of that lane, its "expanded" mark bit s
// of expd. Candidates that cannot beat the worst entry of a full pool are never inserted.
// MAXS = 1 (L <= 32) inserts a batch at once: each candidate's rank among the pool (a
// binary search of the shared-memory copy, which holds the pool in slots 0 .. n - 1 and empty
// keys after) and among the other candidates, each pool entry's shift, one scatter through
// shared memory (pool, pflag). Larger pools insert one candidate at a time (one ballot for its
// rank, one shift).
// Returns the pool size and leaves the pool in pool[0 .. size).
// scratch: 32 ints of shared memory for the compacted neighbour ids.
constexpr int kPoolSlots = 4;

template <int MAXS>
__device__ __forceinline__ uint64_t pick_slot(const uint64_t (&pk)[MAXS], int s) {
    uint64_t v = pk[0];
#pragma unroll
    for (int t = 1; t < MAXS; ++t)
        if (s == t) v = pk[t];
    return v;
}

template <int METRIC, bool SMALLD, typename RT, int MAXS>
__device__ int beam_search(const RT* __restrict__ Xt, const float* __restrict__ invt, const int32_t* __restrict__ adj,
                           int M, long long nt, int ep, long long id_off, const float* q, float4 qreg,
                           const QBytes& qb, float qinv, int d, int L, uint64_t* pool, uint8_t* pflag, int32_t* ht,
                           int htbits, int32_t* scratch, float* P, WarpCounters& ctr, int* status,
                           bool dedupe = true) {
    const int lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const int H = 1 << htbits;
    const int S = MAXS == 1 ? 1 : (L + 31) >> 5;
    for (int s = lane; s < H; s += 32) ht[s] = -1;
    if (lane == 0) scratch[0] = ep;
    if (MAXS == 1) pool[lane] = kEmptyKey;   // slots past the pool size stay empty
    __syncwarp();
    if (ep < 0 || ep >= nt || L < 1 || S > MAXS || (MAXS == 1 && L > 32)) {
        if (lane == 0) atomicOr(status, kErrBounds);
        return 0;
    }
    uint64_t pk[MAXS];
#pragma unroll
    for (int s = 0; s < MAXS; ++s) pk[s] = kEmptyKey;
    unsigned expd = 0u;
    int n;
    uint64_t worst = kEmptyKey;   // pool entry L - 1 once the pool is full
    {
        const float dd = rows_delta<METRIC, SMALLD, RT>(Xt, scratch, 1, q, qreg, qb, d, lane, P);
        uint64_t key = kEmptyKey;
        if (lane == 0) {
            const float inv = (METRIC == FGIM_COSINE) ? __fmul_rn(qinv, invt[ep]) : 1.f;
            key = mkkey(delta_finish<METRIC>(dd, inv), (int32_t)(ep + id_off));
            ht[ht_slot(ep, htbits)] = ep;
            ctr.ndc++;
            pk[0] = key;
            pool[0] = key;
        }
        n = 1;
        if (L == 1) worst = shfl64(key, 0);
        __syncwarp();
    }
    // every vertex is expanded at most once, so nt + 1 iterations always suffice; status[1],
    // when positive, is a smaller expansion budget (a test hook for the timeout path)
    bool done = false;
    const int hop_budget = status[1];
    const long long budget = hop_budget > 0 ? (long long)hop_budget : nt + 1;
    for (long long it = 0; it <= nt; ++it) {
        int first = -1;
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
            if (s < S && first < 0) {
                const unsigned m = __ballot_sync(kFull, 32 * s + lane < n && !((expd >> s) & 1u));
                if (m) first = 32 * s + __ffs(m) - 1;
            }
        }
        if (first < 0) {
            done = true;
            break;
        }
        if (it >= budget) break;
        const uint64_t fk = shfl64(pick_slot<MAXS>(pk, first >> 5), first & 31);
        if (lane == (first & 31)) expd |= 1u << (first >> 5);
        if (lane == 0) ctr.hops++;
        const long long u = (long long)key_id(fk) - id_off;
        const int32_t* row = adj + u * M;
        for (int c0 = 0; c0 < M; c0 += 32) {
            int v = (c0 + lane < M) ? row[c0 + lane] : -1;
            if (v >= nt) {
                atomicOr(status, kErrBounds);
                v = -1;
            }
            // a neighbour listed twice is evaluated once (the lowest lane keeps it); skipped
            // (dedupe false) when the caller knows that no 32-entry chunk of a row repeats an id
            if (dedupe) {   // warp-uniform: every lane takes the match
                const unsigned same = __match_any_sync(kFull, v);
                if ((same & lt) != 0u) v = -1;
            }
            if (v >= 0) {
                const int s = ht_slot(v, htbits);
                if (ht[s] == v) v = -1;
                else ht[s] = v;
            }
            const unsigned m = __ballot_sync(kFull, v >= 0);
            const int U = __popc(m);
            if (U == 0) continue;
            if (v >= 0) scratch[__popc(m & lt)] = v;
            __syncwarp();
            const float dd = rows_delta<METRIC, SMALLD, RT>(Xt, scratch, U, q, qreg, qb, d, lane, P);
            uint64_t cand = kEmptyKey;
            if (lane < U) {
                const int32_t w = scratch[lane];
                const float inv = (METRIC == FGIM_COSINE) ? __fmul_rn(qinv, invt[w]) : 1.f;
                cand = mkkey(delta_finish<METRIC>(dd, inv), (int32_t)(w + id_off));
                ctr.ndc++;
            }
            __syncwarp();
            bool valid = cand < worst;
            if constexpr (MAXS == 1) {
                if (__ballot_sync(kFull, valid) == 0u) continue;
                // rank of the candidate among the pool entries (pool[e] is the empty key for
                // e >= n): five halving steps over the 32 slots. A valid candidate ranks below
                // slot 31 (it beats the worst entry of a full pool, or the pool has empty slots).
                // An equal entry means it is pooled already (the lossy visited table let it in).
                int pos = 0;
#pragma unroll
                for (int st = 16; st > 0; st >>= 1)
                    if (pool[pos + st - 1] < cand) pos += st;
                if (valid && pool[pos] == cand) valid = false;
                unsigned vm = __ballot_sync(kFull, valid);
                if (vm == 0u) continue;
                const int added = __popc(vm);
                // the candidates are distinct: rank among them, and each pool entry's shift
                int crank = 0, shift = 0;
                while (vm) {
                    const int j = __ffs(vm) - 1;
                    vm &= vm - 1;
                    const uint64_t cj = shfl64(cand, j);
                    crank += cj < cand ? 1 : 0;
                    shift += cj < pk[0] ? 1 : 0;
                }
                // merged order: pool entry e goes to e + shift, a candidate to pos + crank
                const bool in_pool = lane < n;
                const int pe = lane + shift, pc = pos + crank;
                __syncwarp();
                if (in_pool && pe < L) {
                    pool[pe] = pk[0];
                    pflag[pe] = (uint8_t)(expd & 1u);
                }
                if (valid && pc < L) {
                    pool[pc] = cand;
                    pflag[pc] = 0;
                }
                __syncwarp();
                n = n + added < L ? n + added : L;
                pk[0] = pool[lane];
                expd = lane < n ? (unsigned)pflag[lane] : 0u;
                __syncwarp();
                if (n == L) worst = shfl64(pk[0], L - 1);
            } else {
                unsigned vm;
                while ((vm = __ballot_sync(kFull, valid)) != 0u) {
                    const int src = __ffs(vm) - 1;
                    const uint64_t c = shfl64(cand, src);
                    if (lane == src) valid = false;
                    bool eq = false;
                    int pos = 0;
#pragma unroll
                    for (int s = 0; s < MAXS; ++s) {
                        if (s < S) {
                            eq |= pk[s] == c;
                            pos += __popc(__ballot_sync(kFull, pk[s] < c));
                        }
                    }
                    if (__any_sync(kFull, eq)) continue;   // already in the pool (same id, same key)
                    // entries pos .. n - 1 move up by one; the slots are updated from the last
                    // one down so every slot reads its predecessor's old entries
#pragma unroll
                    for (int s = MAXS - 1; s >= 0; --s) {
                        if (s < S) {
                            const uint64_t up = shfl64(pk[s], (lane + 31) & 31);
                            const unsigned eup = __shfl_sync(kFull, (expd >> s) & 1u, (lane + 31) & 31);
                            uint64_t prev = up;
                            unsigned eprev = eup;
                            if (s > 0) {
                                const uint64_t w31 = shfl64(pk[s > 0 ? s - 1 : 0], 31);
                                const unsigned e31 = __shfl_sync(kFull, (expd >> (s > 0 ? s - 1 : 0)) & 1u, 31);
                                if (lane == 0) {
                                    prev = w31;
                                    eprev = e31;
                                }
                            }
                            const int e = 32 * s + lane;
                            if (e > pos && !(s == 0 && lane == 0)) {
                                pk[s] = prev;
                                expd = (expd & ~(1u << s)) | (eprev << s);
                            } else if (e == pos) {
                                pk[s] = c;
                                expd &= ~(1u << s);
                            }
                            if (e >= L) {
                                pk[s] = kEmptyKey;
                                expd &= ~(1u << s);
                            }
                        }
                    }
                    n = n < L ? n + 1 : L;
                    if (n == L) worst = shfl64(pick_slot<MAXS>(pk, (L - 1) >> 5), (L - 1) & 31);
                    valid = valid && cand < worst;
                }
            }
        }
    }
    if (!done && lane == 0) atomicOr(status, kErrTimeout);
#pragma unroll
    for (int s = 0; s < MAXS; ++s)
        if (s < S && 32 * s + lane < n) pool[32 * s + lane] = pk[s];
    __syncwarp();
    return n;
}

__device__ __forceinline__ void warp_add_counters(WarpCounters& c, unsigned long long* out) {
    long long a = c.ndc, b = c.hops;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(kFull, a, o);
        b += __shfl_xor_sync(kFull, b, o);
    }
    if (lane_id() == 0 && out) {
        atomicAdd(out + 0, (unsigned long long)a);
        atomicAdd(out + 1, (unsigned long long)b);
    }
}

// shared-memory layout of one warp; all offsets multiples of 16 bytes
struct WarpLayout {
    int q, pool, pflag, ht, res, scratch, part, bytes;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

// part (the 32 x 33 partial matrix) is needed by FP32 rows only
__host__ __device__ inline WarpLayout warp_layout(int d, int L, int htbits, int kres, bool part = true) {
    WarpLayout w;
    int o = 0;
    w.q = o;
    o += align16(d * 4);
    // the pool holds at least 32 slots: a one-slot register pool searches all 32 for a rank
    const int ps = L < 32 ? 32 : L;
    w.pool = o;
    o += align16(ps * 8);
    w.pflag = o;
    o += align16(ps);
    w.ht = o;
    o += align16((1 << htbits) * 4);
    w.res = o;
    o += align16(kres * 8);
    w.scratch = o;
    o += 32 * 4;
    w.part = o;
    if (part) o += 32 * 33 * 4;
    w.bytes = o;
    return w;
}

// ---------------------------------------------------------------------------- host
static inline int ht_bits_for(int L) {
    int want = 32 * L;
    int b = 9;
    while ((1 << b) < want && b < 12) ++b;
    return b;
}

#define FGIM_DISPATCH_METRIC_D(M, D, MACRO, RT, MS)                                              \
    do {                                                                                         \
        const bool small_ = (D) <= 128;                                                          \
        if ((M) == FGIM_L2SQ) {                                                                  \
            if (small_) MACRO(FGIM_L2SQ, true, RT, MS); else MACRO(FGIM_L2SQ, false, RT, MS);    \
        } else if ((M) == FGIM_IP) {                                                             \
            if (small_) MACRO(FGIM_IP, true, RT, MS); else MACRO(FGIM_IP, false, RT, MS);        \
        } else {                                                                                 \
            if (small_) MACRO(FGIM_COSINE, true, RT, MS); else MACRO(FGIM_COSINE, false, RT, MS); \
        }                                                                                        \
    } while (0)
// BF16 rows (d > 128 only: small rows gain little)
#define FGIM_DISPATCH_ALL_WIDE(M, L, MACRO, RT)                                                     \
    do {                                                                                          \
        const int ms_ = (L) <= 32 ? 1 : kPoolSlots;                                               \
        if ((M) == FGIM_L2SQ) {                                                                   \
            if (ms_ == 1) MACRO(FGIM_L2SQ, false, RT, 1); else MACRO(FGIM_L2SQ, false, RT, kPoolSlots); \
        } else if ((M) == FGIM_IP) {                                                              \
            if (ms_ == 1) MACRO(FGIM_IP, false, RT, 1); else MACRO(FGIM_IP, false, RT, kPoolSlots); \
        } else {                                                                                  \
            if (ms_ == 1) MACRO(FGIM_COSINE, false, RT, 1); else MACRO(FGIM_COSINE, false, RT, kPoolSlots); \
        }                                                                                         \
    } while (0)
// register pool of one slot (L <= 32) or of kPoolSlots slots
#define FGIM_DISPATCH_ALL(M, D, L, MACRO, RT)                                                     \
    do {                                                                                         \
        if ((L) <= 32) FGIM_DISPATCH_METRIC_D(M, D, MACRO, RT, 1);                               \
        else FGIM_DISPATCH_METRIC_D(M, D, MACRO, RT, kPoolSlots);                                \
    } while (0)

}  // namespace fgim
