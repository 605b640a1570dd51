// C ABI of the FGIM library (see include/fgim.h): argument checks, scratch memory,
// stage orchestration, launch accounting. Every compute step runs in this library's
// kernels; the host only sequences launches and reads back small counters.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fgim_launch.h"
#include "k_beam.cuh"   // launch-shape helpers of the beam-search kernels (the autotuner)

namespace fgim {

// ---------------------------------------------------------------------------- accounting
static std::atomic<long long> g_launches{0};
static std::atomic<int> g_prof{0};
static std::mutex g_prof_mu;
struct ProfEntry {
    long long launches = 0;
    double ms = 0.0;
};
static std::map<std::string, ProfEntry> g_prof_table;
struct PendingEvent {
    const char* name;
    cudaEvent_t e0, e1;
};
static thread_local std::vector<PendingEvent> t_pending;
static thread_local fgim_stats t_stats;
static thread_local std::string t_last_error;

LaunchScope::LaunchScope(const char* n, cudaStream_t s) : name(n), stream(s), e0(nullptr), e1(nullptr), timed(false) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_prof.load(std::memory_order_relaxed)) {
        if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
            cudaEventRecord(e0, s) == cudaSuccess)
            timed = true;
    }
}

LaunchScope::~LaunchScope() {
    if (timed && cudaEventRecord(e1, stream) == cudaSuccess) {
        t_pending.push_back({name, e0, e1});
        return;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
}

// after the stream has drained: fold the recorded launches into the table
static void resolve_events() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& p : t_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
            ProfEntry& e = g_prof_table[p.name];
            e.launches += 1;
            e.ms += ms;
        }
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
    }
    t_pending.clear();
}

// ---------------------------------------------------------------------------- autotuned launch shapes
struct BeamShape {
    int wpb;
    int htbits;
};
static std::mutex g_tune_mu;
static std::map<unsigned long long, BeamShape> g_tuned;

unsigned long long beam_shape_key(int metric, int row_bytes, int dim, int L) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 0;
    }
    return ((unsigned long long)(sms & 0x3ff) << 40) | ((unsigned long long)(metric & 3) << 36) |
           ((unsigned long long)(row_bytes & 7) << 32) | ((unsigned long long)(dim & 0xffff) << 16) |
           (unsigned long long)(L & 0xffff);
}

void tuned_beam_shape(unsigned long long key, int* wpb, int* htbits) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it == g_tuned.end()) return;
    *wpb = it->second.wpb;
    *htbits = it->second.htbits;
}

// ---------------------------------------------------------------------------- scratch
// The library's scratch comes from its own stream-ordered pool per device, which keeps the
// memory it has mapped between calls (a merge needs several GB; mapping them again on every
// call costs tens of milliseconds). fgim_trim_memory hands the unused part back.
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

// test hooks (fgim_test_set): process-wide, off by default
static std::atomic<long long> g_test_prop_cap{0};
static std::atomic<int> g_test_hop_budget{0};
static std::atomic<long long> g_test_fail_after{-1};
static std::atomic<int> g_test_batch_union{1};
static std::atomic<int> g_test_sparse_nn{-1};   // >= 0: the cut-off of the warp-per-vertex Update form
static thread_local long long t_allocs = 0;   // scratch allocations of the current call

static cudaMemPool_t lib_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
    return pool;
}

class Scratch {
   public:
    explicit Scratch(cudaStream_t s) : s_(s), pool_(lib_pool()) {}
    ~Scratch() { release(); }
    template <typename T>
    T* alloc(long long count) {
        if (count <= 0) count = 1;
        const long long fail_after = g_test_fail_after.load(std::memory_order_relaxed);
        if (fail_after >= 0 && t_allocs >= fail_after) {
            ok_ = false;   // injected failure (test hook), reported like a real one
            return nullptr;
        }
        ++t_allocs;
        void* p = nullptr;
        const size_t bytes = ((size_t)count * sizeof(T) + 255) & ~(size_t)255;
        const cudaError_t e = pool_ ? cudaMallocFromPoolAsync(&p, bytes, pool_, s_) : cudaMallocAsync(&p, bytes, s_);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ok_ = false;
            return nullptr;
        }
        ptrs_.push_back(p);
        return static_cast<T*>(p);
    }
    bool ok() const { return ok_; }
    void release() {
        for (void* p : ptrs_) cudaFreeAsync(p, s_);
        ptrs_.clear();
    }

   private:
    cudaStream_t s_;
    cudaMemPool_t pool_;
    std::vector<void*> ptrs_;
    bool ok_ = true;
};

// ---------------------------------------------------------------------------- errors
struct Fail {
    fgim_status st;
};

static inline void ck(cudaError_t e) {
    if (e != cudaSuccess) {
        t_last_error = cudaGetErrorString(e);
        if (e == cudaErrorMemoryAllocation) throw Fail{FGIM_ENOMEM};
        if (e == cudaErrorNotSupported) {
            t_last_error = "candidate sets of this size do not fit the join's shared memory";
            throw Fail{FGIM_EUNSUPPORTED};
        }
        throw Fail{FGIM_ECUDA};
    }
}

static inline void need(bool ok, fgim_status st, const char* what) {
    if (!ok) {
        t_last_error = what;
        throw Fail{st};
    }
}

// counters on the device: [0] ndc, [1] hops, [2] pairs, [3] repaired, [4] attached
struct Ctx {
    cudaStream_t s;
    Scratch sc;
    int* status = nullptr;
    unsigned long long* ctr = nullptr;
    long long* host = nullptr;   // pinned readback slot
    explicit Ctx(cudaStream_t st) : s(st), sc(st) {
        status = sc.alloc<int>(4);
        ctr = sc.alloc<unsigned long long>(16);
        need(sc.ok(), FGIM_ENOMEM, "scratch allocation failed");
        ck(cudaMemsetAsync(status, 0, 4 * sizeof(int), s));
        ck(cudaMemsetAsync(ctr, 0, 16 * sizeof(unsigned long long), s));
        const int hop_budget = g_test_hop_budget.load(std::memory_order_relaxed);
        if (hop_budget > 0)   // status[1]: the beam searches' expansion budget (test hook)
            ck(cudaMemcpyAsync(status + 1, &hop_budget, sizeof(int), cudaMemcpyHostToDevice, s));
        host = pinned_slot();
    }
    // One pinned 128-byte readback slot per host thread, made once and kept for the thread's
    // life: pinning and releasing host memory on every call costs milliseconds now and then
    // (and the release synchronizes the device).
    static long long* pinned_slot() {
        struct Slot {
            long long* p = nullptr;
            ~Slot() {
                if (p) cudaFreeHost(p);
            }
        };
        thread_local Slot slot;
        if (!slot.p) ck(cudaMallocHost(&slot.p, 128));
        return slot.p;
    }
    template <typename T>
    T* alloc(long long n) {
        T* p = sc.alloc<T>(n);
        need(p != nullptr, FGIM_ENOMEM, "scratch allocation failed");
        return p;
    }
    long long read_ll(const long long* dev) {
        ck(cudaMemcpyAsync(host, dev, sizeof(long long), cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
        return host[0];
    }
    int read_i32(const int32_t* dev) {
        ck(cudaMemcpyAsync(host, dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
        return reinterpret_cast<int32_t*>(host)[0];
    }
    unsigned long long read_u64(const unsigned long long* dev) {
        ck(cudaMemcpyAsync(host, dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
        return reinterpret_cast<unsigned long long*>(host)[0];
    }
    // drain the stream, then report device-side errors and counters
    void finish(fgim_stats* st) {
        ck(cudaStreamSynchronize(s));
        int hs[4];
        unsigned long long hc[16];
        ck(cudaMemcpy(hs, status, sizeof(hs), cudaMemcpyDeviceToHost));
        ck(cudaMemcpy(hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost));
        if (st) {
            st->ndc += (int64_t)hc[0];
            st->hops += (int64_t)hc[1];
            st->join_pairs += (int64_t)hc[2];
            st->repaired += (int64_t)hc[3];
            st->attached += (int64_t)hc[4];
            st->join_cands += (int64_t)hc[5];
        }
        if (hs[0] & kErrTimeout) need(false, FGIM_ETIMEOUT, "a bounded device loop ran out");
        if (hs[0] & kErrBounds) need(false, FGIM_EINVAL, "an input index is out of range (graph ids or entry)");
    }
};

// NVTX range over one stage of a call on the host timeline (a profiler shows the stages; without
// one attached the calls do nothing)
struct StageRange {
    explicit StageRange(const char* name) { nvtxRangePushA(name); }
    ~StageRange() { nvtxRangePop(); }
    StageRange(const StageRange&) = delete;
    StageRange& operator=(const StageRange&) = delete;
};

// ---------------------------------------------------------------------------- validation
static long long total_n(const fgim_shard* sh, int h) {
    long long n = 0;
    for (int i = 0; i < h; ++i) n += sh[i].n;
    return n;
}

static void check_params(const fgim_params* p, bool need_merge) {
    need(p != nullptr, FGIM_EINVAL, "params is NULL");
    need(p->dim >= 4 && p->dim <= FGIM_MAX_DIM && p->dim % 4 == 0, FGIM_EINVAL, "dim must be a multiple of 4 in [4, 2048]");
    need(p->dtype == FGIM_F32 || p->dtype == FGIM_BF16, FGIM_EINVAL, "dtype must be FGIM_F32 or FGIM_BF16");
    need(p->metric == FGIM_L2SQ || p->metric == FGIM_IP || p->metric == FGIM_COSINE, FGIM_EINVAL, "unknown metric");
    if (!need_merge) return;
    need(p->k >= 1 && p->k <= FGIM_MAX_K, FGIM_EINVAL, "k must be in [1, 128]");
    need(p->R >= 1 && p->R <= FGIM_MAX_R, FGIM_EINVAL, "R must be in [1, 128]");
    need(std::isfinite(p->alpha) && p->alpha > 0.f, FGIM_EINVAL, "alpha must be a positive finite number");
    need(p->L >= 0 && p->L <= FGIM_MAX_L, FGIM_EINVAL, "L must be 0 or in [1, 128]");
    need(p->iters >= 0 && p->iters <= 1000, FGIM_EINVAL, "iters must be in [0, 1000]");
    need(p->rev_cap >= 0 && p->rev_cap <= FGIM_MAX_K, FGIM_EINVAL, "rev_cap must be 0 or in [1, 128]");
    need(p->reach_beam >= 0 && p->reach_beam <= FGIM_MAX_L, FGIM_EINVAL, "reach_beam must be 0 or in [1, 128]");
    need(p->join_filter >= FGIM_PREC_BF16 && p->join_filter <= FGIM_PREC_FP8E4M3, FGIM_EINVAL,
         "join_filter must be 0 (BF16 tensor core), 1 (FP32) or 2 (FP8 E4M3 tensor core)");
    need(p->byte_rows == 0 || p->byte_rows == 1, FGIM_EINVAL, "byte_rows must be 0 (auto) or 1 (off)");
    need(p->prune_rule >= FGIM_PRUNE_ALPHA_RNG && p->prune_rule <= FGIM_PRUNE_TAU_MNG, FGIM_EINVAL,
         "prune_rule must be 0 (alpha-RNG), 1 (MRNG) or 2 (tau-MNG)");
    need(std::isfinite(p->tau) && p->tau >= 0.f, FGIM_EINVAL, "tau must be a finite number >= 0");
}

static void check_shards(const fgim_shard* sh, int h, const fgim_params* p) {
    need(sh != nullptr, FGIM_EINVAL, "shards is NULL");
    need(h >= 2 && h <= FGIM_MAX_SHARDS, FGIM_EINVAL, "h must be in [2, 64]");
    long long n = 0;
    for (int i = 0; i < h; ++i) {
        need(sh[i].vectors != nullptr && sh[i].adj != nullptr, FGIM_EINVAL, "shard vectors/adj is NULL");
        need(((uintptr_t)sh[i].vectors & (p->dtype == FGIM_F32 ? 15u : 1u)) == 0, FGIM_EINVAL,
             "shard vectors must be 16-byte (FP32) or 2-byte (BF16) aligned");
        need(sh[i].n >= 1, FGIM_EINVAL, "shard n must be >= 1");
        need(sh[i].max_degree >= 1 && sh[i].max_degree <= FGIM_MAX_DEGREE, FGIM_EINVAL, "max_degree must be in [1, 128]");
        need(sh[i].entry >= 0 && sh[i].entry < sh[i].n, FGIM_EINVAL, "entry out of range");
        n += sh[i].n;
    }
    need(n < 0x7fffffffLL, FGIM_EINVAL, "total size must fit a 31-bit id");
}

// the shards of one merge, all in one group searched with pool L
static ShardTable make_table(const fgim_shard* sh, int h, int dim, int L) {
    ShardTable t;
    std::memset(&t, 0, sizeof(t));
    t.h = h;
    t.dim = dim;
    long long o = 0;
    for (int i = 0; i < h; ++i) {
        t.off[i] = o;
        t.adj[i] = sh[i].adj;
        t.M[i] = sh[i].max_degree;
        t.entry[i] = sh[i].entry;
        t.grp[i] = 0;
        t.gend[i] = h;
        t.gL[i] = L;
        o += sh[i].n;
    }
    t.off[h] = o;
    return t;
}

// vectors of all shards as one FP32 [N, dim] buffer (no copy when they are FP32 and already
// consecutive; BF16 vectors are decoded into a new buffer)
static const float* contiguous_vectors(Ctx& c, const fgim_shard* sh, int h, int dim, int dtype, long long N) {
    if (dtype == FGIM_BF16) {
        float* X = c.alloc<float>(N * dim);
        long long o = 0;
        for (int i = 0; i < h; ++i) {
            ck(launch_bf16_to_f32(static_cast<const uint16_t*>(sh[i].vectors), (long long)sh[i].n * dim, X + o * dim,
                                  c.s));
            o += sh[i].n;
        }
        return X;
    }
    const char* base = static_cast<const char*>(sh[0].vectors);
    bool contiguous = true;
    long long o = 0;
    for (int i = 0; i < h; ++i) {
        if (static_cast<const char*>(sh[i].vectors) != base + o * dim * 4) contiguous = false;
        o += sh[i].n;
    }
    if (contiguous) return reinterpret_cast<const float*>(base);
    float* X = c.alloc<float>(N * dim);
    o = 0;
    for (int i = 0; i < h; ++i) {
        ck(cudaMemcpyAsync(X + o * dim, sh[i].vectors, (size_t)sh[i].n * dim * 4, cudaMemcpyDeviceToDevice, c.s));
        o += sh[i].n;
    }
    return X;
}

static int resolve_L(const fgim_params* p, int h) { return p->L > 0 ? p->L : (p->k + (h - 1) - 1) / (h - 1); }
static int resolve_rev_cap(const fgim_params* p) { return p->rev_cap > 0 ? p->rev_cap : p->k; }

static int merged_entry(const fgim_shard* sh, int h) {
    int best = 0;
    for (int i = 1; i < h; ++i)
        if (sh[i].n > sh[best].n) best = i;
    long long o = 0;
    for (int i = 0; i < best; ++i) o += sh[i].n;
    return (int)(o + sh[best].entry);
}

// ---------------------------------------------------------------------------- stages
struct Problem {
    ShardTable t;
    const float* X;
    const uint8_t* X8;   // X as bytes when every coordinate is an integer in [0, 255], else nullptr
    const uint16_t* Xh;  // the BF16 rows X decodes from (BF16 storage), else nullptr
    const float* inv;
    long long N;
    int d;
    int metric;
};

// byte rows and cosine norms of P.X
static void finish_problem(Ctx& c, Problem& P, const fgim_params* p);

// BF16 vectors of all shards as one [N, dim] buffer (no copy when already consecutive)
static const uint16_t* contiguous_bf16(Ctx& c, const fgim_shard* sh, int h, int dim, long long N) {
    const char* base = static_cast<const char*>(sh[0].vectors);
    bool contiguous = true;
    long long o = 0;
    for (int i = 0; i < h; ++i) {
        if (static_cast<const char*>(sh[i].vectors) != base + o * dim * 2) contiguous = false;
        o += sh[i].n;
    }
    if (contiguous) return reinterpret_cast<const uint16_t*>(base);
    uint16_t* X = c.alloc<uint16_t>(N * dim);
    o = 0;
    for (int i = 0; i < h; ++i) {
        ck(cudaMemcpyAsync(X + o * dim, sh[i].vectors, (size_t)sh[i].n * dim * 2, cudaMemcpyDeviceToDevice, c.s));
        o += sh[i].n;
    }
    return X;
}

static Problem make_problem(Ctx& c, const fgim_shard* sh, int h, const fgim_params* p) {
    Problem P;
    P.N = total_n(sh, h);
    P.d = p->dim;
    P.metric = p->metric;
    P.t = make_table(sh, h, p->dim, resolve_L(p, h));
    P.X = contiguous_vectors(c, sh, h, p->dim, p->dtype, P.N);
    P.Xh = p->dtype == FGIM_BF16 ? contiguous_bf16(c, sh, h, p->dim, P.N) : nullptr;
    finish_problem(c, P, p);
    return P;
}

static void finish_problem(Ctx& c, Problem& P, const fgim_params* p) {
    P.inv = nullptr;
    P.X8 = nullptr;
    if (byte_rows_ok(P.d) && p->byte_rows == 0) {
        uint8_t* x8 = c.alloc<uint8_t>(P.N * P.d);
        int* flag = c.alloc<int>(1);
        ck(cudaMemsetAsync(flag, 0, sizeof(int), c.s));
        ck(launch_narrow_u8(P.X, P.N * P.d, x8, flag, c.s));
        if (c.read_i32(flag) == 0) P.X8 = x8;
    }
    if (p->metric == FGIM_COSINE) {
        float* inv = c.alloc<float>(P.N);
        ck(launch_inv_norms(P.X, P.N, P.d, inv, c.s));
        P.inv = inv;
    }
}

// ---------------------------------------------------------------------------- phi
// The ID mapping of Sec. 4.1.3 with invalid vertices: valid vertices are numbered
// consecutively in (shard, local id) order.
static bool has_valid(const fgim_shard* sh, int h) {
    for (int i = 0; i < h; ++i)
        if (sh[i].valid) return true;
    return false;
}

struct PhiMap {
    int32_t* phi = nullptr;   // [N] input row -> merged id, -1 = invalid
    int32_t* src = nullptr;   // [Nv] merged id -> input row
    long long Nv = 0;
    long long offv[FGIM_MAX_SHARDS + 1];   // first merged id of every shard
    int32_t entry = 0;        // merged entry (the rule of merged_entry, after phi)
};

static PhiMap build_phi(Ctx& c, const fgim_shard* sh, int h, long long N) {
    PhiMap F;
    int32_t* flag = c.alloc<int32_t>(N);
    long long o = 0;
    for (int i = 0; i < h; ++i) {
        ck(launch_valid_flags(sh[i].valid, sh[i].n, flag + o, c.s));
        o += sh[i].n;
    }
    long long* off = c.alloc<long long>(N + 1);
    const size_t sb = scan_scratch_bytes(N);
    void* tmp = c.alloc<unsigned char>((long long)sb);
    F.src = c.alloc<int32_t>(N);
    ck(compact_flags(flag, N, F.src, off, tmp, sb, c.s));
    F.phi = c.alloc<int32_t>(N);
    ck(launch_phi(flag, off, N, F.phi, c.s));
    o = 0;
    for (int i = 0; i < h; ++i) {
        F.offv[i] = c.read_ll(off + o);
        o += sh[i].n;
    }
    F.offv[h] = c.read_ll(off + N);
    F.Nv = F.offv[h];
    need(F.Nv >= 1, FGIM_EINVAL, "no shard has a valid vertex");
    // the shard with the most valid vertices (lowest index on ties): its entry if valid, else
    // its first valid vertex
    int best = 0;
    for (int i = 1; i < h; ++i)
        if (F.offv[i + 1] - F.offv[i] > F.offv[best + 1] - F.offv[best]) best = i;
    long long gb = sh[best].entry;
    for (int i = 0; i < best; ++i) gb += sh[i].n;
    const int e = c.read_i32(F.phi + gb);
    F.entry = e >= 0 ? e : (int32_t)F.offv[best];
    return F;
}

// the valid vertices alone, renumbered by phi: the problem of stages (b) and (c)
static Problem compact_problem(Ctx& c, const Problem& P, const PhiMap& F, const fgim_params* p) {
    Problem Q;
    Q.N = F.Nv;
    Q.d = P.d;
    Q.metric = P.metric;
    Q.t = P.t;
    for (int i = 0; i <= P.t.h; ++i) Q.t.off[i] = F.offv[i];
    float* X = c.alloc<float>(Q.N * Q.d);
    ck(launch_gather_rows(P.X, F.src, Q.N, Q.d, X, c.s));
    Q.X = X;
    Q.Xh = nullptr;
    finish_problem(c, Q, p);
    return Q;
}

static void stage_a(Ctx& c, const Problem& P, const fgim_params* p, int h, fgim_knng* g, const PhiMap* F = nullptr) {
    StageRange range("fgim stage a: cross query (Alg. 1, Alg. 2)");
    const int L = resolve_L(p, h);
    need(L >= 1 && L <= FGIM_MAX_L, FGIM_EINVAL, "resolved L out of range");
    ck(launch_cross_query(P.t, P.X, P.X8, P.inv, P.N, P.metric, g->k, L, g, c.ctr + 0, c.status, c.s,
                          F ? F->phi : nullptr, F ? F->src : nullptr, F ? F->Nv : P.N, P.Xh));
}

static void refine_pass(Ctx& c, const Problem& P, const fgim_params* p, fgim_knng* g, fgim_stats* st) {
    StageRange range("fgim stage b: Visit + Update (Alg. 3)");
    const long long N = P.N;
    const int k = g->k;
    const int rev_cap = resolve_rev_cap(p);
    RefineBuffers b;
    std::memset(&b, 0, sizeof(b));
    b.cntN = c.alloc<int32_t>(N);
    b.cntO = c.alloc<int32_t>(N);
    b.offN = c.alloc<long long>(N + 1);
    b.offO = c.alloc<long long>(N + 1);
    b.fillN = c.alloc<int32_t>(N);
    b.fillO = c.alloc<int32_t>(N);
    b.rev_capacity = N * k;
    b.revN = c.alloc<uint64_t>(N * k);
    b.revO = c.alloc<uint64_t>(N * k);
    b.topN = c.alloc<int32_t>(N * rev_cap);
    b.topO = c.alloc<int32_t>(N * rev_cap);
    b.ntopN = c.alloc<int32_t>(N);
    b.ntopO = c.alloc<int32_t>(N);
    b.cmax = 2 * (k + rev_cap);
    b.cand = c.alloc<int32_t>(N * b.cmax);
    b.nn = c.alloc<int32_t>(N);
    b.no = c.alloc<int32_t>(N);
    // proposal buffer (20 bytes per proposal): one Update pass of a fresh k-NNG proposes up to
    // a few k per vertex; vertices whose proposals do not fit are redone after the merge
    long long cap = 320LL * N;
    const long long per_vertex_max = 2LL * b.cmax * b.cmax;
    if (cap < 4 * per_vertex_max) cap = 4 * per_vertex_max;
    if (cap < (1LL << 22)) cap = 1LL << 22;
    const long long test_cap = g_test_prop_cap.load(std::memory_order_relaxed);
    if (test_cap > 0) cap = std::max(test_cap, per_vertex_max);   // test hook: force the re-run path
    b.prop_cap = cap;
    b.prop_tgt = c.alloc<int32_t>(cap);
    b.prop_key = c.alloc<uint64_t>(cap);
    b.prop_sorted = c.alloc<uint64_t>(cap);
    b.prop_count = c.alloc<unsigned long long>(1);
    b.pcnt = c.alloc<int32_t>(N);
    b.poff = c.alloc<long long>(N + 1);
    b.pfill = c.alloc<int32_t>(N);
    b.pending = c.alloc<uint8_t>(N);
    b.pend_flag = c.alloc<int32_t>(N);
    b.pend_list = c.alloc<int32_t>(N);
    b.pend_off = c.alloc<long long>(N + 1);
    b.scan_bytes = scan_scratch_bytes(N);
    b.scan_tmp = c.alloc<unsigned char>((long long)b.scan_bytes);
    b.max_nc = c.alloc<int32_t>(12);
    b.host_i32 = reinterpret_cast<int32_t*>(c.host + 4);   // 24 ints of the 128-byte pinned slot
    b.blist = c.alloc<int32_t>(4 * N);
    b.wk = c.alloc<uint64_t>(N);
    b.blist_cap = N;
    b.join_filter = p->join_filter;
    {
        // vertices with at most this many new candidates join one warp each on byte rows (their
        // pairs are few; the tile form's per-candidate costs dominate there)
        constexpr int kSparseNNDefault = 10;
        const int o = g_test_sparse_nn.load(std::memory_order_relaxed);
        b.sparse_nn = o >= 0 ? o : kSparseNNDefault;
    }
    b.X8 = P.X8;
    b.Xb = nullptr;
    b.fp8 = false;
    if (p->join_filter == FGIM_PREC_BF16 && P.d % 16 == 0) {
        b.Xb = c.alloc<__nv_bfloat16>(N * P.d);
        b.tcm = c.alloc<float4>(N);
        ck(launch_prep_bf16(P.X, N, P.d, reinterpret_cast<__nv_bfloat16*>(b.Xb), b.tcm, c.s));
    } else if (p->join_filter == FGIM_PREC_FP8E4M3 && P.d % 32 == 0) {
        // E4M3 rows (one byte per coordinate) with one scale per vector, addressed like BF16 pairs
        uint8_t* Xq = c.alloc<uint8_t>(N * P.d);
        b.tcm = c.alloc<float4>(N);
        ck(launch_prep_fp8(P.X, N, P.d, Xq, b.tcm, c.s));
        b.Xb = reinterpret_cast<__nv_bfloat16*>(Xq);
        b.fp8 = true;
    }

    ck(refine_visit(*g, rev_cap, b, c.s));
    ck(cudaMemsetAsync(b.pending, 0, N, c.s));
    ck(cudaMemsetAsync(b.prop_count, 0, sizeof(unsigned long long), c.s));
    ck(refine_join(P.t, P.X, P.inv, P.metric, *g, b, nullptr, N, c.ctr + 2, c.ctr + 5, c.status, c.s));
    for (int q = 0; q < 5; ++q) st->join_class[q] += b.class_count[q];
    unsigned long long cnt = c.read_u64(b.prop_count);
    long long total = (long long)cnt;
    ck(refine_merge(*g, b, cnt < (unsigned long long)cap ? (long long)cnt : cap, c.s));
    // vertices whose proposals did not all fit (proposal buffer full) are re-run against the
    // merged lists: a proposal that would have entered a list still beats its (only lower)
    // worst key and is still absent, so the merged result is the same
    long long prev_pending = -1;
    for (int rerun = 0;; ++rerun) {
        ck(launch_nonzero_flags(b.pending, N, b.pend_flag, c.s));
        ck(compact_flags(b.pend_flag, N, b.pend_list, b.pend_off, b.scan_tmp, b.scan_bytes, c.s));
        const long long np = c.read_ll(b.pend_off + N);
        if (np == 0) break;
        need(!(cnt <= (unsigned long long)cap && np == prev_pending), FGIM_EINTERNAL,
             "pending vertices without a proposal overflow");
        prev_pending = np;
        st->join_reruns += 1;
        need(st->join_reruns < 10000, FGIM_EINTERNAL, "proposal overflow does not shrink");
        ck(cudaMemsetAsync(b.pending, 0, N, c.s));
        ck(cudaMemsetAsync(b.prop_count, 0, sizeof(unsigned long long), c.s));
        ck(refine_join(P.t, P.X, P.inv, P.metric, *g, b, b.pend_list, np, c.ctr + 2, c.ctr + 5, c.status, c.s));
        for (int q = 0; q < 5; ++q) st->join_class[q] += b.class_count[q];
        cnt = c.read_u64(b.prop_count);
        total += (long long)cnt;
        ck(refine_merge(*g, b, cnt < (unsigned long long)cap ? (long long)cnt : cap, c.s));
    }
    st->proposals += total;
}

static void repair(Ctx& c, const Problem& P, fgim_knng* g, int32_t* T, fgim_stats* st) {
    StageRange range("fgim stage b: indegree repair (Alg. 4)");
    const long long N = P.N;
    ck(launch_indegree(g->ids, N, g->k, T, true, g->flags, c.s));
    int32_t* flag = c.alloc<int32_t>(N);
    int32_t* zeros = c.alloc<int32_t>(N);
    long long* off = c.alloc<long long>(N + 1);
    const size_t sb = scan_scratch_bytes(N);
    unsigned char* tmp = c.alloc<unsigned char>((long long)sb);
    ck(launch_zero_flags(T, N, flag, c.s));
    ck(compact_flags(flag, N, zeros, off, tmp, sb, c.s));
    const long long nz = c.read_ll(off + N);
    if (st) st->zero_indegree = nz;
    if (nz == 0) return;
    unsigned long long* owner = c.alloc<unsigned long long>(N);
    long long* ff = c.alloc<long long>(nz + 2);   // first uncommitted index after each round (one round commits >= 1)
    ck(cudaMemsetAsync(owner, 0xff, sizeof(unsigned long long) * N, c.s));
    ck(cudaMemsetAsync(ff, 0, sizeof(long long), c.s));
    long long start = 0, rho = 1;
    constexpr int kBatch = 16;   // rounds between host reads of the progress
    while (start < nz) {
        need(rho <= nz, FGIM_EINTERNAL, "indegree repair made no progress");
        const int rounds = (int)std::min<long long>(kBatch, nz + 1 - rho);
        ck(launch_repair_rounds(*g, T, zeros, nz, rho, rounds, ff, owner, c.ctr + 3, c.status, c.s));
        rho += rounds;
        const long long next = c.read_ll(ff + (rho - 1));
        need(next > start, FGIM_EINTERNAL, "indegree repair made no progress");
        start = next;
    }
}

static void prune(Ctx& c, const Problem& P, const fgim_params* p, const fgim_knng* g, const int32_t* T, int32_t* e_ids,
                  float* e_dist, int32_t* e_cnt) {
    StageRange range("fgim stage c: neighbour selection (Alg. 5)");
    PruneRule rule;
    rule.kind = p->prune_rule;
    rule.alpha2 = (float)((double)p->alpha * (double)p->alpha);   // alpha^2 and 3 tau rounded once to FP32
    rule.tau3 = (float)(3.0 * (double)p->tau);
    ck(launch_prune(P.X, P.X8, P.inv, P.N, P.d, P.metric, *g, T, p->R, rule, e_ids, e_dist, e_cnt, c.status, c.s));
}

static void reverse_insert(Ctx& c, long long N, int R, const int32_t* e_ids, const float* e_dist, const int32_t* e_cnt,
                           fgim_graph* out) {
    StageRange range("fgim stage c: reverse edges (Alg. 5)");
    ReverseBuffers b;
    b.cnt = c.alloc<int32_t>(N);
    b.off = c.alloc<long long>(N + 1);
    b.fill = c.alloc<int32_t>(N);
    b.rev = c.alloc<uint64_t>(N * R);
    b.scan_bytes = scan_scratch_bytes(N);
    b.scan_tmp = c.alloc<unsigned char>((long long)b.scan_bytes);
    ck(launch_reverse_insert(N, R, e_ids, e_dist, e_cnt, b, out->ids, out->dist, out->deg, c.s));
}

// The entry points the reachability fix works from: one merge (the graph's entry), or the merges
// of a batch run as one problem (entries[m] on the device, merge m owning ids off[m] .. off[m+1]-1).
struct Entries {
    const int32_t* ent = nullptr;    // device [nm], nullptr = the graph's entry
    const long long* off = nullptr;  // device [nm + 1]
    int nm = 1;
};

// BFS from the entry (or entries); returns the number of reached vertices
static long long bfs(Ctx& c, const fgim_graph* g, const Entries& E, int32_t* visited, int32_t* fa, int32_t* fb,
                     int32_t* counts) {
    const long long N = g->n;
    if (E.ent) ck(launch_bfs_init_multi(visited, N, fa, counts, E.ent, E.nm, c.status, c.s));
    else ck(launch_bfs_init(visited, N, fa, counts, g->entry, c.s));
    constexpr int kBatch = 8;   // levels between host reads of the frontier size
    for (int level = 1; level <= N; level += kBatch) {
        ck(launch_bfs_levels(g->ids, g->R, N, visited, fa, fb, counts, level, kBatch, c.s));
        const int last = level + kBatch - 1;   // its output frontier size is counts[(last + 1) % 3]
        if (c.read_i32(counts + (last + 1) % 3) == 0) break;
    }
    return c.read_ll(reinterpret_cast<const long long*>(counts + 4));
}

static void reach_fix(Ctx& c, const Problem& P, const fgim_params* p, fgim_graph* g, fgim_stats* st,
                      const Entries& E = Entries()) {
    StageRange range("fgim reachability fix");
    const long long N = g->n;
    const int R = g->R;
    const int beam = p->reach_beam > 0 ? p->reach_beam : 64;
    int32_t* visited = c.alloc<int32_t>(N);
    int32_t* fa = c.alloc<int32_t>(N);
    int32_t* fb = c.alloc<int32_t>(N);
    int32_t* counts = c.alloc<int32_t>(8);   // BFS state: three frontier sizes, reached (int64 at [4])
    int32_t* label = c.alloc<int32_t>(N);
    int32_t* flag = c.alloc<int32_t>(N);
    int32_t* reps = c.alloc<int32_t>(N);
    long long* off = c.alloc<long long>(N + 1);
    const size_t sb = scan_scratch_bytes(N);
    unsigned char* tmp = c.alloc<unsigned char>((long long)sb);
    int32_t* changed = c.alloc<int32_t>(1);
    int32_t* npar = c.alloc<int32_t>(N);
    unsigned long long* owner = c.alloc<unsigned long long>(N);
    long long* ff = c.alloc<long long>(N + 2);   // first uncommitted index after each round (one round commits >= 1)
    int4* plan = c.alloc<int4>(kReachWindow);    // the actions planned in a round
    int32_t* cand = nullptr;
    float* cdist = nullptr;
    int32_t* starts = nullptr;
    long long cand_cap = 0;
    long long reached = 0;
    for (int round = 0; round < 16; ++round) {
        reached = bfs(c, g, E, visited, fa, fb, counts);
        if (reached >= N) break;
        ck(launch_cc_init(visited, N, label, c.s));
        for (long long it = 0; it <= N; ++it) {
            ck(cudaMemsetAsync(changed, 0, sizeof(int32_t), c.s));
            ck(launch_cc_step(g->ids, R, N, visited, label, changed, c.s));
            if (c.read_i32(changed) == 0) break;
        }
        ck(launch_rep_flags(visited, label, N, flag, c.s));
        ck(compact_flags(flag, N, reps, off, tmp, sb, c.s));
        const long long nr = c.read_ll(off + N);
        if (nr == 0) break;
        if (nr > cand_cap) {
            cand = c.alloc<int32_t>(nr * beam);
            cdist = c.alloc<float>(nr * beam);
            if (E.ent) starts = c.alloc<int32_t>(nr);
            cand_cap = nr;
        }
        // each representative searches from its merge's entry
        if (E.ent) ck(launch_rep_starts(reps, nr, E.off, E.ent, E.nm, starts, c.s));
        ck(launch_search(P.X, P.X8, P.inv, N, P.d, P.metric, g->ids, R, g->entry, nullptr, nullptr, reps, nr, beam, beam,
                         cand, cdist, c.ctr + 0, c.status, c.s, P.Xh, E.ent ? starts : nullptr));
        ck(launch_bfs_parents(g->ids, R, N, visited, npar, c.s));
        // rounds run in batches between host reads of the progress; ff[0] = 0 starts round 1
        ck(cudaMemsetAsync(owner, 0xff, sizeof(unsigned long long) * N, c.s));
        ck(cudaMemsetAsync(ff, 0, sizeof(long long), c.s));
        long long start = 0, rho = 1;
        constexpr int kBatch = 64;   // rounds per cooperative launch (it stops early once all are done)
        while (start < nr) {
            need(rho <= nr, FGIM_EINTERNAL, "reachability fix made no progress");
            const int rounds = (int)std::min<long long>(kBatch, nr + 1 - rho);
            ck(launch_reach_rounds(g->ids, g->dist, g->deg, visited, npar, R, reps, nr, rho, rounds, ff, cand, cdist,
                                   beam, owner, plan, c.ctr + 4, c.s));
            rho += rounds;
            const long long next = c.read_ll(ff + (rho - 1));
            need(next > start, FGIM_EINTERNAL, "reachability fix made no progress");
            start = next;
        }
    }
    reached = bfs(c, g, E, visited, fa, fb, counts);
    if (st) st->unreached = N - reached;
}

}  // namespace fgim

// ============================================================================ C ABI
using namespace fgim;

template <typename F>
static fgim_status guarded(F&& f) {
    try {
        f();
        return FGIM_OK;
    } catch (const Fail& e) {
        return e.st;
    } catch (const std::bad_alloc&) {
        t_last_error = "host allocation failed";
        return FGIM_ENOMEM;
    } catch (...) {
        t_last_error = "internal error";
        return FGIM_EINTERNAL;
    }
}

static void begin_call() {
    std::memset(&t_stats, 0, sizeof(t_stats));
    t_last_error.clear();
    t_allocs = 0;
}

static void end_call() { resolve_events(); }

extern "C" {

fgim_status fgim_cross_query(const fgim_shard* shards, int32_t h, const fgim_params* params, fgim_knng* out,
                             void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        check_params(params, true);
        check_shards(shards, h, params);
        need(out && out->ids && out->dist && out->flags, FGIM_EINVAL, "knng buffers are NULL");
        const bool masked = has_valid(shards, h);
        need(out->k == params->k && (masked || out->n == total_n(shards, h)), FGIM_EINVAL, "knng shape mismatch");
        Ctx c((cudaStream_t)stream);
        Problem P = make_problem(c, shards, h, params);
        if (masked) {
            const PhiMap F = build_phi(c, shards, h, P.N);
            need(out->n == F.Nv, FGIM_EINVAL, "knng shape mismatch (n must be the number of valid vertices)");
            stage_a(c, P, params, h, out, &F);
        } else {
            stage_a(c, P, params, h, out);
        }
        c.finish(&t_stats);
    });
    end_call();
    return r;
}

fgim_status fgim_refine_pass(const fgim_shard* shards, int32_t h, const fgim_params* params, fgim_knng* knng,
                             void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        check_params(params, true);
        check_shards(shards, h, params);
        need(!has_valid(shards, h), FGIM_EUNSUPPORTED,
             "validity masks are honoured by fgim_merge, fgim_merge_batch and fgim_cross_query only");
        need(knng && knng->ids && knng->dist && knng->flags, FGIM_EINVAL, "knng buffers are NULL");
        need(knng->n == total_n(shards, h) && knng->k >= 1 && knng->k <= FGIM_MAX_K, FGIM_EINVAL, "knng shape mismatch");
        Ctx c((cudaStream_t)stream);
        Problem P = make_problem(c, shards, h, params);
        refine_pass(c, P, params, knng, &t_stats);
        c.finish(&t_stats);
    });
    end_call();
    return r;
}

fgim_status fgim_indegree_repair(const fgim_shard* shards, int32_t h, const fgim_params* params, fgim_knng* knng,
                                 int32_t* T_out, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        check_params(params, true);
        check_shards(shards, h, params);
        need(!has_valid(shards, h), FGIM_EUNSUPPORTED,
             "validity masks are honoured by fgim_merge, fgim_merge_batch and fgim_cross_query only");
        need(knng && knng->ids && knng->dist && knng->flags, FGIM_EINVAL, "knng buffers are NULL");
        need(knng->n == total_n(shards, h), FGIM_EINVAL, "knng shape mismatch");
        Ctx c((cudaStream_t)stream);
        Problem P;
        P.N = knng->n;
        int32_t* T = T_out ? T_out : c.alloc<int32_t>(P.N);
        repair(c, P, knng, T, &t_stats);
        c.finish(&t_stats);
    });
    end_call();
    return r;
}

fgim_status fgim_prune(const fgim_shard* shards, int32_t h, const fgim_params* params, const fgim_knng* knng,
                       const int32_t* T, int32_t* e_ids, float* e_dist, int32_t* e_cnt, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        check_params(params, true);
        check_shards(shards, h, params);
        need(!has_valid(shards, h), FGIM_EUNSUPPORTED,
             "validity masks are honoured by fgim_merge, fgim_merge_batch and fgim_cross_query only");
        need(knng && knng->ids && knng->dist && T && e_ids && e_dist && e_cnt, FGIM_EINVAL, "NULL buffer");
        need(knng->n == total_n(shards, h) && knng->k >= 1 && knng->k <= FGIM_MAX_K, FGIM_EINVAL, "knng shape mismatch");
        Ctx c((cudaStream_t)stream);
        Problem P = make_problem(c, shards, h, params);
        prune(c, P, params, knng, T, e_ids, e_dist, e_cnt);
        c.finish(&t_stats);
    });
    end_call();
    return r;
}

fgim_status fgim_reverse_insert(int64_t n, int32_t R, const int32_t* e_ids, const float* e_dist, const int32_t* e_cnt,
                                fgim_graph* out, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        need(n >= 1 && n < 0x7fffffffLL && R >= 1 && R <= FGIM_MAX_R, FGIM_EINVAL, "bad n or R");
        need(e_ids && e_dist && e_cnt && out && out->ids && out->dist && out->deg, FGIM_EINVAL, "NULL buffer");
        need(out->n == n && out->R == R, FGIM_EINVAL, "graph shape mismatch");
        Ctx c((cudaStream_t)stream);
        reverse_insert(c, n, R, e_ids, e_dist, e_cnt, out);
        c.finish(&t_stats);
    });
    end_call();
    return r;
}

fgim_status fgim_reach_fix(const fgim_shard* shards, int32_t h, const fgim_params* params, fgim_graph* graph,
                           void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        check_params(params, true);
        check_shards(shards, h, params);
        need(!has_valid(shards, h), FGIM_EUNSUPPORTED,
             "validity masks are honoured by fgim_merge, fgim_merge_batch and fgim_cross_query only");
        need(graph && graph->ids && graph->dist && graph->deg, FGIM_EINVAL, "NULL buffer");
        need(graph->n == total_n(shards, h) && graph->R == params->R, FGIM_EINVAL, "graph shape mismatch");
        need(graph->entry >= 0 && graph->entry < graph->n, FGIM_EINVAL, "graph entry out of range");
        Ctx c((cudaStream_t)stream);
        Problem P = make_problem(c, shards, h, params);
        reach_fix(c, P, params, graph, &t_stats);
        c.finish(&t_stats);
    });
    end_call();
    return r;
}

static void merge_impl(Ctx& c, const fgim_shard* shards, int32_t h, const fgim_params* params, fgim_knng* knng_out,
                       fgim_graph* out) {
    Problem P0 = make_problem(c, shards, h, params);
    const bool masked = has_valid(shards, h);
    PhiMap F;
    if (masked) F = build_phi(c, shards, h, P0.N);
    const long long N = masked ? F.Nv : P0.N;
    need(out->n == N, FGIM_EINVAL, "graph shape mismatch (n must be the number of valid vertices)");
    need(!knng_out || knng_out->n == N, FGIM_EINVAL, "knng shape mismatch (n must be the number of valid vertices)");
    const int k = params->k;
    fgim_knng g;
    if (knng_out) {
        g = *knng_out;
    } else {
        g.ids = c.alloc<int32_t>(N * k);
        g.dist = c.alloc<float>(N * k);
        g.flags = c.alloc<uint8_t>(N * k);
        g.n = N;
        g.k = k;
    }
    stage_a(c, P0, params, h, &g, masked ? &F : nullptr);
    const Problem P = masked ? compact_problem(c, P0, F, params) : P0;
    int32_t* T = c.alloc<int32_t>(N);
    for (int it = 0; it < params->iters; ++it) {
        refine_pass(c, P, params, &g, &t_stats);
        repair(c, P, &g, T, &t_stats);
    }
    if (params->iters == 0) ck(launch_indegree(g.ids, N, k, T, false, nullptr, c.s));
    int32_t* e_ids = c.alloc<int32_t>(N * params->R);
    float* e_dist = c.alloc<float>(N * params->R);
    int32_t* e_cnt = c.alloc<int32_t>(N);
    prune(c, P, params, &g, T, e_ids, e_dist, e_cnt);
    reverse_insert(c, N, params->R, e_ids, e_dist, e_cnt, out);
    out->entry = masked ? F.entry : merged_entry(shards, h);
    if (params->ensure_reachable) reach_fix(c, P, params, out, &t_stats);
    c.finish(&t_stats);
}

fgim_status fgim_merge(const fgim_shard* shards, int32_t h, const fgim_params* params, fgim_knng* knng_out,
                       fgim_graph* out, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        check_params(params, true);
        check_shards(shards, h, params);
        const long long N = total_n(shards, h);
        const bool masked = has_valid(shards, h);   // the row count is checked once phi is known
        need(out && out->ids && out->dist && out->deg, FGIM_EINVAL, "graph buffers are NULL");
        need((masked || out->n == N) && out->R == params->R, FGIM_EINVAL, "graph shape mismatch");
        if (knng_out) {
            need(knng_out->ids && knng_out->dist && knng_out->flags, FGIM_EINVAL, "knng buffers are NULL");
            need((masked || knng_out->n == N) && knng_out->k == params->k, FGIM_EINVAL, "knng shape mismatch");
        }
        Ctx c((cudaStream_t)stream);
        merge_impl(c, shards, h, params, knng_out, out);
    });
    end_call();
    return r;
}

// A batch of independent merges as ONE problem over the disjoint union of their vertices: the
// shards of every merge get consecutive global ids (merge after merge), the shard table groups
// each merge's shards (the cross query of a vertex searches only its own merge's other shards,
// with its merge's L), and each stage's kernels run once for the whole batch instead of once
// per merge. The outputs are those of the merges run one by one: no list ever holds an id of
// another merge (stage a draws candidates from the vertex's own merge, Update pairs candidates of
// one list, prune and reverse edges stay inside lists), and the sequential loops that are run in
// rounds (indegree repair, reachability fix) commit exactly the sequential result, whose steps
// for one merge never read another merge's vertices; the reachability fix starts its BFS from
// every merge's entry and each representative's search from its own merge's entry.
static bool union_batch_ok(const fgim_shard* const* shards, const int32_t* h, int n) {
    long long shard_count = 0, N = 0;
    for (int m = 0; m < n; ++m) {
        if (has_valid(shards[m], h[m])) return false;
        shard_count += h[m];
        N += total_n(shards[m], h[m]);
    }
    return n > 1 && shard_count <= kMaxTableShards && N < 0x7fffffffLL;
}

static void merge_union(Ctx& c, const fgim_shard* const* shards, const int32_t* h, int nm, const fgim_params* p,
                        fgim_graph* outs) {
    const int d = p->dim, k = p->k, R = p->R;
    std::vector<long long> moff(nm + 1, 0);
    Problem P;
    std::memset(&P.t, 0, sizeof(P.t));
    P.t.dim = d;
    int H = 0, Lmax = 1;
    long long o = 0;
    for (int m = 0; m < nm; ++m) {
        const int L = resolve_L(p, h[m]);
        need(L >= 1 && L <= FGIM_MAX_L, FGIM_EINVAL, "resolved L out of range");
        Lmax = std::max(Lmax, L);
        const int first = H;
        for (int i = 0; i < h[m]; ++i, ++H) {
            const fgim_shard& sh = shards[m][i];
            P.t.off[H] = o;
            P.t.adj[H] = sh.adj;
            P.t.M[H] = sh.max_degree;
            P.t.entry[H] = sh.entry;
            P.t.grp[H] = first;
            P.t.gend[H] = first + h[m];
            P.t.gL[H] = L;
            o += sh.n;
        }
        moff[m + 1] = o;
    }
    P.t.h = H;
    P.t.off[H] = o;
    const long long N = o;
    P.N = N;
    P.d = d;
    P.metric = p->metric;
    // the vectors of every shard in one buffer (FP32 working copy; BF16 rows kept beside it)
    float* X = c.alloc<float>(N * d);
    uint16_t* Xh = p->dtype == FGIM_BF16 ? c.alloc<uint16_t>(N * d) : nullptr;
    for (int m = 0, q = 0; m < nm; ++m)
        for (int i = 0; i < h[m]; ++i, ++q) {
            const fgim_shard& sh = shards[m][i];
            const long long at = P.t.off[q] * d, cnt = (long long)sh.n * d;
            if (Xh) {
                ck(launch_bf16_to_f32(static_cast<const uint16_t*>(sh.vectors), cnt, X + at, c.s));
                ck(cudaMemcpyAsync(Xh + at, sh.vectors, (size_t)cnt * 2, cudaMemcpyDeviceToDevice, c.s));
            } else {
                ck(cudaMemcpyAsync(X + at, sh.vectors, (size_t)cnt * 4, cudaMemcpyDeviceToDevice, c.s));
            }
        }
    P.X = X;
    P.Xh = Xh;
    finish_problem(c, P, p);
    fgim_knng g;
    g.ids = c.alloc<int32_t>(N * k);
    g.dist = c.alloc<float>(N * k);
    g.flags = c.alloc<uint8_t>(N * k);
    g.n = N;
    g.k = k;
    ck(launch_cross_query(P.t, P.X, P.X8, P.inv, N, P.metric, k, Lmax, &g, c.ctr + 0, c.status, c.s, nullptr, nullptr,
                          N, P.Xh));
    int32_t* T = c.alloc<int32_t>(N);
    for (int it = 0; it < p->iters; ++it) {
        refine_pass(c, P, p, &g, &t_stats);
        repair(c, P, &g, T, &t_stats);
    }
    if (p->iters == 0) ck(launch_indegree(g.ids, N, k, T, false, nullptr, c.s));
    int32_t* e_ids = c.alloc<int32_t>(N * R);
    float* e_dist = c.alloc<float>(N * R);
    int32_t* e_cnt = c.alloc<int32_t>(N);
    prune(c, P, p, &g, T, e_ids, e_dist, e_cnt);
    fgim_graph U;
    U.ids = c.alloc<int32_t>(N * R);
    U.dist = c.alloc<float>(N * R);
    U.deg = c.alloc<int32_t>(N);
    U.n = N;
    U.R = R;
    reverse_insert(c, N, R, e_ids, e_dist, e_cnt, &U);
    std::vector<int32_t> ent(nm);
    for (int m = 0; m < nm; ++m) ent[m] = (int32_t)(moff[m] + merged_entry(shards[m], h[m]));
    U.entry = ent[0];
    if (p->ensure_reachable) {
        Entries E;
        int32_t* ent_d = c.alloc<int32_t>(nm);
        long long* off_d = c.alloc<long long>(nm + 1);
        ck(cudaMemcpyAsync(ent_d, ent.data(), sizeof(int32_t) * nm, cudaMemcpyHostToDevice, c.s));
        ck(cudaMemcpyAsync(off_d, moff.data(), sizeof(long long) * (nm + 1), cudaMemcpyHostToDevice, c.s));
        E.ent = ent_d;
        E.off = off_d;
        E.nm = nm;
        reach_fix(c, P, p, &U, &t_stats, E);
    }
    for (int m = 0; m < nm; ++m) {
        ck(launch_split_rows(U.ids + moff[m] * R, U.dist + moff[m] * R, U.deg + moff[m], moff[m + 1] - moff[m], R,
                             (int32_t)moff[m], outs[m].ids, outs[m].dist, outs[m].deg, c.s));
        outs[m].entry = ent[m] - (int32_t)moff[m];
    }
    c.finish(&t_stats);
}

fgim_status fgim_merge_batch(const fgim_shard* const* shards, const int32_t* h, int32_t n_merges,
                             const fgim_params* params, fgim_graph* outs, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        check_params(params, true);
        need(n_merges >= 0, FGIM_EINVAL, "n_merges must be >= 0");
        need(n_merges == 0 || (shards && h && outs), FGIM_EINVAL, "shards, h or outs is NULL");
        for (int m = 0; m < n_merges; ++m) {
            check_shards(shards[m], h[m], params);
            need(outs[m].ids && outs[m].dist && outs[m].deg, FGIM_EINVAL, "graph buffers are NULL");
            need((has_valid(shards[m], h[m]) || outs[m].n == total_n(shards[m], h[m])) && outs[m].R == params->R,
                 FGIM_EINVAL, "graph shape mismatch");
        }
        if (g_test_batch_union.load(std::memory_order_relaxed) && union_batch_ok(shards, h, n_merges)) {
            Ctx c((cudaStream_t)stream);
            merge_union(c, shards, h, n_merges, params, outs);
            return;
        }
        for (int m = 0; m < n_merges; ++m) {
            Ctx c((cudaStream_t)stream);
            merge_impl(c, shards[m], h[m], params, nullptr, &outs[m]);
        }
    });
    end_call();
    return r;
}

fgim_status fgim_merge_host(const void* vectors_host, const int32_t* adj_host, const int32_t* sizes,
                            const int32_t* entries, int32_t h, int32_t max_degree, const fgim_params* params,
                            int32_t* out_ids_host, int32_t* out_deg_host, int32_t* out_entry_host, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        check_params(params, true);
        need(vectors_host && adj_host && sizes && entries && out_ids_host && out_deg_host && out_entry_host,
             FGIM_EINVAL, "NULL host buffer");
        need(h >= 2 && h <= FGIM_MAX_SHARDS, FGIM_EINVAL, "h must be in [2, 64]");
        need(max_degree >= 1 && max_degree <= FGIM_MAX_DEGREE, FGIM_EINVAL, "max_degree must be in [1, 128]");
        long long N = 0;
        for (int i = 0; i < h; ++i) {
            need(sizes[i] >= 1, FGIM_EINVAL, "shard size must be >= 1");
            N += sizes[i];
        }
        need(N < 0x7fffffffLL, FGIM_EINVAL, "total size must fit a 31-bit id");
        Ctx c((cudaStream_t)stream);
        const int d = params->dim;
        const size_t esz = params->dtype == FGIM_BF16 ? 2 : 4;
        unsigned char* X = c.alloc<unsigned char>(N * d * (long long)esz);
        int32_t* A = c.alloc<int32_t>(N * max_degree);
        ck(cudaMemcpyAsync(X, vectors_host, (size_t)N * d * esz, cudaMemcpyHostToDevice, c.s));
        ck(cudaMemcpyAsync(A, adj_host, (size_t)N * max_degree * 4, cudaMemcpyHostToDevice, c.s));
        std::vector<fgim_shard> sh(h);
        long long o = 0;
        for (int i = 0; i < h; ++i) {
            sh[i].vectors = X + o * d * (long long)esz;
            sh[i].adj = A + o * max_degree;
            sh[i].n = sizes[i];
            sh[i].max_degree = max_degree;
            sh[i].entry = entries[i];
            sh[i].reserved = 0;
            sh[i].valid = nullptr;
            o += sizes[i];
        }
        check_shards(sh.data(), h, params);
        fgim_graph g;
        g.ids = c.alloc<int32_t>(N * params->R);
        g.dist = c.alloc<float>(N * params->R);
        g.deg = c.alloc<int32_t>(N);
        g.n = N;
        g.R = params->R;
        merge_impl(c, sh.data(), h, params, nullptr, &g);
        ck(cudaMemcpyAsync(out_ids_host, g.ids, (size_t)N * params->R * 4, cudaMemcpyDeviceToHost, c.s));
        ck(cudaMemcpyAsync(out_deg_host, g.deg, (size_t)N * 4, cudaMemcpyDeviceToHost, c.s));
        ck(cudaStreamSynchronize(c.s));
        *out_entry_host = g.entry;
    });
    end_call();
    return r;
}

// ---------------------------------------------------------------------------- HNSW layers
static HnswThresholds hnsw_thresholds(int M) {
    HnswThresholds th;
    std::memset(&th, 0, sizeof(th));
    unsigned long long p = (unsigned long long)M;
    while (th.count < kMaxHnswLevels) {
        th.t[th.count++] = ~0ull / p;
        if (p > ~0ull / (unsigned long long)M) break;
        p *= (unsigned long long)M;
    }
    return th;
}

// the FP32 rows of `vectors` (decoded when BF16)
static const float* f32_rows(Ctx& c, const void* vectors, long long n, int dim, int dtype) {
    if (dtype == FGIM_F32) return static_cast<const float*>(vectors);
    float* X = c.alloc<float>(n * dim);
    ck(launch_bf16_to_f32(static_cast<const uint16_t*>(vectors), n * dim, X, c.s));
    return X;
}

fgim_status fgim_hnsw_levels(int64_t n, int32_t M, uint64_t seed, int32_t* levels, int64_t* counts, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        need(levels && counts, FGIM_EINVAL, "NULL buffer");
        need(n >= 1 && n < 0x7fffffffLL, FGIM_EINVAL, "bad n");
        need(M >= 2 && M <= FGIM_MAX_R, FGIM_EINVAL, "M must be in [2, 128]");
        Ctx c((cudaStream_t)stream);
        ck(launch_hnsw_levels(n, (unsigned long long)seed, hnsw_thresholds(M), levels, c.s));
        std::vector<int32_t> h(n);
        ck(cudaMemcpyAsync(h.data(), levels, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c.s));
        c.finish(&t_stats);
        for (int l = 0; l <= FGIM_MAX_LEVELS; ++l) counts[l] = 0;
        for (long long v = 0; v < n; ++v)
            for (int l = 0; l <= h[v] && l <= FGIM_MAX_LEVELS; ++l) ++counts[l];
    });
    end_call();
    return r;
}

// One PG over the rows `members` (nl ascending ids) of the FP32 rows X: each member's exact ef
// nearest among the members before it, the RNG heuristic to M, bidirectional edges, the
// heuristic again over the union of own and reverse edges. adj [nl, M] holds positions in
// members (-1 padded), deg [nl] the degrees.
static void build_layer_graph(Ctx& c, const float* X, int dim, int metric, const int32_t* members, long long nl,
                              int M, int ef, int32_t* adj, int32_t* deg) {
    Problem L;
    std::memset(&L.t, 0, sizeof(L.t));
    L.t.h = 1;
    L.t.dim = dim;
    L.t.off[1] = nl;
    L.N = nl;
    L.d = dim;
    L.metric = metric;
    float* Xl = c.alloc<float>(nl * dim);
    ck(launch_gather_rows(X, members, nl, dim, Xl, c.s));
    L.X = Xl;
    L.Xh = nullptr;
    fgim_params lp;
    std::memset(&lp, 0, sizeof(lp));
    lp.metric = metric;
    finish_problem(c, L, &lp);
    // the exact ef nearest earlier members, the RNG heuristic to M, bidirectional edges,
    // the heuristic again over the union of own and reverse edges
    const int kk = (int)std::min<long long>(ef, std::max<long long>(nl - 1, 1));
    int32_t* k_ids = c.alloc<int32_t>(nl * kk);
    float* k_dist = c.alloc<float>(nl * kk);
    ck(launch_layer_knn(L.X, L.X8, L.inv, nl, dim, metric, kk, k_ids, k_dist, c.s));
    int32_t* T = c.alloc<int32_t>(nl);   // never 1: no indegree clause
    ck(cudaMemsetAsync(T, 0, sizeof(int32_t) * nl, c.s));
    fgim_knng g1;
    std::memset(&g1, 0, sizeof(g1));
    g1.ids = k_ids;
    g1.dist = k_dist;
    g1.n = nl;
    g1.k = kk;
    int32_t* e_ids = c.alloc<int32_t>(nl * M);
    float* e_dist = c.alloc<float>(nl * M);
    int32_t* e_cnt = c.alloc<int32_t>(nl);
    const PruneRule rng = {FGIM_PRUNE_ALPHA_RNG, 1.f, 0.f};   // HNSW's heuristic: alpha = 1, no indegree clause
    ck(launch_prune(L.X, L.X8, L.inv, nl, dim, metric, g1, T, M, rng, e_ids, e_dist, e_cnt, c.status, c.s));
    const int wide = FGIM_MAX_K;   // own and reverse edges together (their 128 nearest if more)
    int32_t* w_ids = c.alloc<int32_t>(nl * wide);
    float* w_dist = c.alloc<float>(nl * wide);
    ck(launch_widen(e_ids, e_dist, nl, M, wide, w_ids, w_dist, c.s));
    fgim_graph u;
    std::memset(&u, 0, sizeof(u));
    u.ids = c.alloc<int32_t>(nl * wide);
    u.dist = c.alloc<float>(nl * wide);
    u.deg = c.alloc<int32_t>(nl);
    u.n = nl;
    u.R = wide;
    reverse_insert(c, nl, wide, w_ids, w_dist, e_cnt, &u);
    fgim_knng g2;
    std::memset(&g2, 0, sizeof(g2));
    g2.ids = u.ids;
    g2.dist = u.dist;
    g2.n = nl;
    g2.k = wide;
    float* f_dist = c.alloc<float>(nl * M);
    ck(launch_prune(L.X, L.X8, L.inv, nl, dim, metric, g2, T, M, rng, adj, f_dist, deg, c.status, c.s));
}

fgim_status fgim_hnsw_layer(const void* vectors, int64_t n, int32_t dim, int32_t dtype, int32_t metric,
                            const int32_t* levels, int32_t level, int32_t M, int32_t ef, int32_t* members,
                            int32_t* adj, int32_t* deg, int64_t n_layer, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        need(vectors && levels && members && adj && deg, FGIM_EINVAL, "NULL buffer");
        need(n >= 1 && n < 0x7fffffffLL, FGIM_EINVAL, "bad n");
        need(dim >= 4 && dim <= FGIM_MAX_DIM && dim % 4 == 0, FGIM_EINVAL, "dim must be a multiple of 4 in [4, 2048]");
        need(dtype == FGIM_F32 || dtype == FGIM_BF16, FGIM_EINVAL, "dtype must be FGIM_F32 or FGIM_BF16");
        need(metric == FGIM_L2SQ || metric == FGIM_IP || metric == FGIM_COSINE, FGIM_EINVAL, "unknown metric");
        need(level >= 1 && level <= FGIM_MAX_LEVELS, FGIM_EINVAL, "level must be in [1, 16]");
        need(M >= 1 && M <= 64, FGIM_EINVAL, "M must be in [1, 64]");
        need(ef >= 1 && ef <= FGIM_MAX_K, FGIM_EINVAL, "ef must be in [1, 128]");
        need(n_layer >= 0 && n_layer <= n, FGIM_EINVAL, "bad n_layer");
        need(((uintptr_t)vectors & (dtype == FGIM_F32 ? 15u : 1u)) == 0, FGIM_EINVAL, "vectors misaligned");
        Ctx c((cudaStream_t)stream);
        // members: the vertices of level >= `level`, ascending
        int32_t* flag = c.alloc<int32_t>(n);
        long long* off = c.alloc<long long>(n + 1);
        const size_t sb = scan_scratch_bytes(n);
        void* tmp = c.alloc<unsigned char>((long long)sb);
        int32_t* mem = c.alloc<int32_t>(n);
        ck(launch_level_flags(levels, n, level, flag, c.s));
        ck(compact_flags(flag, n, mem, off, tmp, sb, c.s));
        const long long nl = c.read_ll(off + n);
        need(nl == n_layer, FGIM_EINVAL, "n_layer is not the number of vertices of that level");
        if (nl == 0) return;
        ck(cudaMemcpyAsync(members, mem, sizeof(int32_t) * nl, cudaMemcpyDeviceToDevice, c.s));
        const float* X = f32_rows(c, vectors, n, dim, dtype);
        build_layer_graph(c, X, dim, metric, members, nl, M, ef, adj, deg);
        c.finish(&t_stats);
    });
    end_call();
    return r;
}
fgim_status fgim_build_pg(const void* vectors, int64_t n, int32_t dim, int32_t dtype, int32_t metric, int32_t M,
                          int32_t ef, int32_t* adj, int32_t* deg, int32_t* entry_out, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        need(vectors && adj && deg && entry_out, FGIM_EINVAL, "NULL buffer");
        need(n >= 1 && n < 0x7fffffffLL, FGIM_EINVAL, "bad n");
        need(dim >= 4 && dim <= FGIM_MAX_DIM && dim % 4 == 0, FGIM_EINVAL, "dim must be a multiple of 4 in [4, 2048]");
        need(dtype == FGIM_F32 || dtype == FGIM_BF16, FGIM_EINVAL, "dtype must be FGIM_F32 or FGIM_BF16");
        need(metric == FGIM_L2SQ || metric == FGIM_IP || metric == FGIM_COSINE, FGIM_EINVAL, "unknown metric");
        need(M >= 1 && M <= FGIM_MAX_DEGREE, FGIM_EINVAL, "M must be in [1, 128]");
        need(ef >= 1 && ef <= FGIM_MAX_L, FGIM_EINVAL, "ef must be in [1, 128]");
        need(((uintptr_t)vectors & (dtype == FGIM_F32 ? 15u : 1u)) == 0, FGIM_EINVAL, "vectors misaligned");
        Ctx c((cudaStream_t)stream);
        Problem P;
        std::memset(&P.t, 0, sizeof(P.t));
        P.N = n;
        P.d = dim;
        P.metric = metric;
        P.X = f32_rows(c, vectors, n, dim, dtype);
        P.Xh = dtype == FGIM_BF16 ? static_cast<const uint16_t*>(vectors) : nullptr;
        fgim_params lp;
        std::memset(&lp, 0, sizeof(lp));
        lp.metric = metric;
        finish_problem(c, P, &lp);   // byte rows when the data allow, cosine norms
        // the medoid and the insertion order
        double* mean = c.alloc<double>(dim);
        unsigned long long* dbits = c.alloc<unsigned long long>(n);
        unsigned long long* best = c.alloc<unsigned long long>(1);
        int* medoid_d = c.alloc<int>(1);
        ck(launch_pg_medoid(P.X, n, dim, mean, dbits, best, medoid_d, c.s));
        int32_t* order = c.alloc<int32_t>(n);
        float* nd = c.alloc<float>(n * M);
        int32_t* zeros = c.alloc<int32_t>(n);
        ck(launch_pg_init(n, M, medoid_d, order, adj, nd, deg, zeros, c.s));
        const int medoid = c.read_i32(medoid_d);
        need(medoid >= 0 && medoid < n, FGIM_EINTERNAL, "medoid out of range");
        // per-batch scratch
        const long long bmax = std::min<long long>(1024, n);
        const int W = M + (int)bmax;   // a target's list and the batch's reverse edges to it
        int32_t* res_ids = c.alloc<int32_t>(bmax * ef);
        float* res_d = c.alloc<float>(bmax * ef);
        int32_t* e_ids = c.alloc<int32_t>(bmax * M);
        float* e_dist = c.alloc<float>(bmax * M);
        int32_t* e_cnt = c.alloc<int32_t>(bmax);
        int32_t* cin = c.alloc<int32_t>(n);
        int32_t* fill = c.alloc<int32_t>(n);
        long long* off = c.alloc<long long>(n + 1);
        uint64_t* rev = c.alloc<uint64_t>(bmax * M);
        int32_t* flag = c.alloc<int32_t>(n);
        int32_t* targets = c.alloc<int32_t>(n);
        long long* toff = c.alloc<long long>(n + 1);
        const size_t sb = scan_scratch_bytes(n);
        unsigned char* tmp = c.alloc<unsigned char>((long long)sb);
        const long long tmax = std::min<long long>(n, bmax * M);
        int32_t* ov_ids = c.alloc<int32_t>(tmax * W);
        float* ov_dist = c.alloc<float>(tmax * W);
        int32_t* ov_tgt = c.alloc<int32_t>(tmax);
        int* n_ov = c.alloc<int>(1);
        int32_t* o_ids = c.alloc<int32_t>(tmax * M);
        float* o_dist = c.alloc<float>(tmax * M);
        int32_t* o_cnt = c.alloc<int32_t>(tmax);
        PruneRule heur;   // HNSW's heuristic: MRNG's rule, no indegree clause (T = 0 everywhere)
        heur.kind = FGIM_PRUNE_MRNG;
        heur.alpha2 = 1.f;
        heur.tau3 = 0.f;
        for (long long done = 1; done < n;) {
            const long long b = std::min(std::min(std::max(done / 2, 1LL), bmax), n - done);
            // 1. every row of the batch searches the graph as it stands (Alg. 1 from the medoid)
            ck(launch_search(P.X, P.X8, P.inv, n, dim, metric, adj, M, medoid, nullptr, nullptr, order + done, b, ef,
                             ef, res_ids, res_d, c.ctr + 0, c.status, c.s, P.Xh));
            fgim_knng g1;
            std::memset(&g1, 0, sizeof(g1));
            g1.ids = res_ids;
            g1.dist = res_d;
            g1.n = b;
            g1.k = ef;
            ck(launch_prune(P.X, P.X8, P.inv, n, dim, metric, g1, zeros, M, heur, e_ids, e_dist, e_cnt, c.status, c.s));
            // 2. the batch's lists go in, their entries are reverse edges of their targets
            ck(cudaMemsetAsync(cin, 0, sizeof(int32_t) * n, c.s));
            ck(cudaMemsetAsync(fill, 0, sizeof(int32_t) * n, c.s));
            ck(launch_pg_install(order + done, b, M, e_ids, e_dist, e_cnt, adj, nd, deg, cin, c.s));
            ck(scan_counts(cin, n, off, tmp, sb, c.s));
            ck(launch_pg_rev_fill(order + done, b, M, e_ids, e_dist, e_cnt, off, fill, rev, c.s));
            ck(launch_pos_flags(cin, n, flag, c.s));
            ck(compact_flags(flag, n, targets, toff, tmp, sb, c.s));
            const long long nt = c.read_ll(toff + n);
            // 3. every target keeps its list and its new edges, or the heuristic's M of them
            ck(cudaMemsetAsync(n_ov, 0, sizeof(int), c.s));
            ck(launch_pg_rev_merge(targets, nt, off, rev, M, M + (int)b, adj, nd, deg, ov_ids, ov_dist, ov_tgt, n_ov,
                                   c.s));
            const long long nov = c.read_i32(n_ov);
            if (nov > 0) {
                fgim_knng g2;
                std::memset(&g2, 0, sizeof(g2));
                g2.ids = ov_ids;
                g2.dist = ov_dist;
                g2.n = nov;
                g2.k = M + (int)b;
                ck(launch_prune(P.X, P.X8, P.inv, n, dim, metric, g2, zeros, M, heur, o_ids, o_dist, o_cnt, c.status,
                                c.s));
                ck(launch_pg_write_back(ov_tgt, nov, M, o_ids, o_dist, o_cnt, adj, nd, deg, c.s));
            }
            done += b;
        }
        c.finish(&t_stats);
        *entry_out = medoid;
    });
    end_call();
    return r;
}


fgim_status fgim_search_hnsw(const void* base, int64_t n, int32_t dim, int32_t dtype, int32_t metric,
                             const int32_t* graph_ids, int32_t R, const fgim_layer* layers, int32_t n_layers,
                             int32_t entry, const void* queries, int32_t nq, int32_t topk, int32_t beam, int32_t ef_up,
                             int32_t* out_ids, float* out_dist, int32_t* out_start, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        need(base && graph_ids && queries && out_ids && out_dist, FGIM_EINVAL, "NULL buffer");
        need(n >= 1 && n < 0x7fffffffLL, FGIM_EINVAL, "bad n");
        need(dim >= 4 && dim <= FGIM_MAX_DIM && dim % 4 == 0, FGIM_EINVAL, "dim must be a multiple of 4 in [4, 2048]");
        need(dtype == FGIM_F32 || dtype == FGIM_BF16, FGIM_EINVAL, "dtype must be FGIM_F32 or FGIM_BF16");
        need(metric == FGIM_L2SQ || metric == FGIM_IP || metric == FGIM_COSINE, FGIM_EINVAL, "unknown metric");
        need(R >= 1 && R <= FGIM_MAX_DEGREE, FGIM_EINVAL, "R must be in [1, 128]");
        need(entry >= 0 && entry < n, FGIM_EINVAL, "entry out of range");
        need(nq >= 0, FGIM_EINVAL, "nq must be >= 0");
        need(beam >= 1 && beam <= FGIM_MAX_L && topk >= 1 && topk <= beam, FGIM_EINVAL, "need 1 <= topk <= beam <= 128");
        need(ef_up >= 1 && ef_up <= FGIM_MAX_L, FGIM_EINVAL, "ef_up must be in [1, 128]");
        need(n_layers >= 0 && n_layers <= FGIM_MAX_LEVELS && (n_layers == 0 || layers), FGIM_EINVAL,
             "n_layers must be in [0, 16]");
        const uintptr_t am = dtype == FGIM_F32 ? 15u : 1u;
        need(((uintptr_t)base & am) == 0 && ((uintptr_t)queries & am) == 0, FGIM_EINVAL, "vectors misaligned");
        std::vector<int> live;   // the non-empty layers, top first
        for (int l = n_layers - 1; l >= 0; --l) {
            need(layers[l].n >= 0 && layers[l].n <= n && layers[l].M >= 1 && layers[l].M <= FGIM_MAX_DEGREE &&
                     (layers[l].n == 0 || (layers[l].members && layers[l].adj)),
                 FGIM_EINVAL, "bad layer");
            if (layers[l].n > 0) live.push_back(l);
        }
        if (nq == 0) return;
        Ctx c((cudaStream_t)stream);
        const float* X = f32_rows(c, base, n, dim, dtype);
        const float* Q = f32_rows(c, queries, nq, dim, dtype);
        float* inv = nullptr;
        float* qinv = nullptr;
        if (metric == FGIM_COSINE) {
            inv = c.alloc<float>(n);
            qinv = c.alloc<float>(nq);
            ck(launch_inv_norms(X, n, dim, inv, c.s));
            ck(launch_inv_norms(Q, nq, dim, qinv, c.s));
        }
        int32_t* start = out_start ? out_start : c.alloc<int32_t>(nq);
        int32_t* qpos = c.alloc<int32_t>(nq);
        int32_t* best = c.alloc<int32_t>(nq);
        float* bdist = c.alloc<float>(nq);
        if (live.empty()) {
            ck(launch_hnsw_next(nullptr, nullptr, 0, nullptr, 0, nq, 1, entry, qpos, start, c.status, c.s));
        } else {
            // every query starts at the entry's position in the top layer; each layer is searched
            // with Alg. 1 (pool ef_up) and its nearest result starts the layer below
            const fgim_layer& t0 = layers[live[0]];
            ck(launch_hnsw_next(nullptr, nullptr, 0, t0.members, t0.n, nq, 1, entry, qpos, start, c.status, c.s));
            for (size_t i = 0; i < live.size(); ++i) {
                const fgim_layer& ly = layers[live[i]];
                float* Xl = c.alloc<float>(ly.n * dim);
                ck(launch_gather_rows(X, ly.members, ly.n, dim, Xl, c.s));
                float* invl = nullptr;
                if (metric == FGIM_COSINE) {
                    invl = c.alloc<float>(ly.n);
                    ck(launch_inv_norms(Xl, ly.n, dim, invl, c.s));
                }
                ck(launch_search(Xl, nullptr, invl, ly.n, dim, metric, ly.adj, ly.M, 0, Q, qinv, nullptr, nq, 1, ef_up,
                                 best, bdist, c.ctr + 0, c.status, c.s, nullptr, qpos));
                const fgim_layer* nx = i + 1 < live.size() ? &layers[live[i + 1]] : nullptr;
                ck(launch_hnsw_next(best, ly.members, ly.n, nx ? nx->members : nullptr, nx ? nx->n : 0, nq, 0, entry,
                                    qpos, start, c.status, c.s));
            }
        }
        ck(launch_search(X, nullptr, inv, n, dim, metric, graph_ids, R, entry, Q, qinv, nullptr, nq, topk, beam, out_ids,
                         out_dist, c.ctr + 0, c.status, c.s,
                         dtype == FGIM_BF16 ? static_cast<const uint16_t*>(base) : nullptr, start));
        c.finish(&t_stats);
    });
    end_call();
    return r;
}

fgim_status fgim_search(const void* base, int64_t n, int32_t dim, int32_t dtype, int32_t metric,
                        const int32_t* graph_ids, int32_t R, int32_t entry, const void* queries, int32_t nq,
                        int32_t topk, int32_t beam, int32_t* out_ids, float* out_dist, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        need(base && graph_ids && queries && out_ids && out_dist, FGIM_EINVAL, "NULL buffer");
        need(n >= 1 && n < 0x7fffffffLL, FGIM_EINVAL, "bad n");
        need(dim >= 4 && dim <= FGIM_MAX_DIM && dim % 4 == 0, FGIM_EINVAL, "dim must be a multiple of 4 in [4, 2048]");
        need(dtype == FGIM_F32 || dtype == FGIM_BF16, FGIM_EINVAL, "dtype must be FGIM_F32 or FGIM_BF16");
        need(metric == FGIM_L2SQ || metric == FGIM_IP || metric == FGIM_COSINE, FGIM_EINVAL, "unknown metric");
        need(R >= 1 && R <= FGIM_MAX_DEGREE, FGIM_EINVAL, "R must be in [1, 128]");
        need(entry >= 0 && entry < n, FGIM_EINVAL, "entry out of range");
        need(nq >= 0, FGIM_EINVAL, "nq must be >= 0");
        need(beam >= 1 && beam <= FGIM_MAX_L && topk >= 1 && topk <= beam, FGIM_EINVAL, "need 1 <= topk <= beam <= 128");
        const uintptr_t am = dtype == FGIM_F32 ? 15u : 1u;
        need(((uintptr_t)base & am) == 0 && ((uintptr_t)queries & am) == 0, FGIM_EINVAL,
             "vectors must be 16-byte (FP32) or 2-byte (BF16) aligned");
        if (nq == 0) return;
        Ctx c((cudaStream_t)stream);
        const float* X = static_cast<const float*>(base);
        const float* Q = static_cast<const float*>(queries);
        if (dtype == FGIM_BF16) {
            float* Xf = c.alloc<float>(n * dim);
            float* Qf = c.alloc<float>((long long)nq * dim);
            ck(launch_bf16_to_f32(static_cast<const uint16_t*>(base), n * dim, Xf, c.s));
            ck(launch_bf16_to_f32(static_cast<const uint16_t*>(queries), (long long)nq * dim, Qf, c.s));
            X = Xf;
            Q = Qf;
        }
        float* inv = nullptr;
        float* qinv = nullptr;
        if (metric == FGIM_COSINE) {
            inv = c.alloc<float>(n);
            qinv = c.alloc<float>(nq);
            ck(launch_inv_norms(X, n, dim, inv, c.s));
            ck(launch_inv_norms(Q, nq, dim, qinv, c.s));
        }
        ck(launch_search(X, nullptr, inv, n, dim, metric, graph_ids, R, entry, Q, qinv, nullptr, nq, topk, beam, out_ids,
                         out_dist, c.ctr + 0, c.status, c.s,
                         dtype == FGIM_BF16 ? static_cast<const uint16_t*>(base) : nullptr));
        c.finish(&t_stats);
    });
    end_call();
    return r;
}

fgim_status fgim_graph_alloc(int64_t n, int32_t R, fgim_graph* g) {
    if (!g) return FGIM_EINVAL;
    std::memset(g, 0, sizeof(*g));
    if (n < 1 || n >= 0x7fffffffLL || R < 1 || R > FGIM_MAX_R) return FGIM_EINVAL;
    // ids, dist and deg in one block: ids first (the block's base), each part 256-byte aligned
    const size_t part = ((size_t)n * R * 4 + 255) & ~(size_t)255;
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, 2 * part + (size_t)n * 4);
    if (e != cudaSuccess) {
        cudaGetLastError();
        t_last_error = cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? FGIM_ENOMEM : FGIM_ECUDA;
    }
    g->ids = static_cast<int32_t*>(p);
    g->dist = reinterpret_cast<float*>(static_cast<char*>(p) + part);
    g->deg = reinterpret_cast<int32_t*>(static_cast<char*>(p) + 2 * part);
    g->n = n;
    g->R = R;
    g->entry = 0;
    return FGIM_OK;
}

void fgim_graph_free(fgim_graph* g) {
    if (!g) return;
    if (g->ids) cudaFree(g->ids);
    std::memset(g, 0, sizeof(*g));
}

fgim_status fgim_autotune(const fgim_shard* shards, int32_t h, const fgim_params* params, const char* cache_path,
                          int32_t* out_wpb, int32_t* out_ht_bits, float* out_ms, void* stream) {
    begin_call();
    fgim_status r = guarded([&] {
        check_params(params, true);
        check_shards(shards, h, params);
        need(!has_valid(shards, h), FGIM_EUNSUPPORTED, "tune on a merge without validity masks");
        Ctx c((cudaStream_t)stream);
        Problem P = make_problem(c, shards, h, params);
        const int L = resolve_L(params, h);
        need(L >= 1 && L <= FGIM_MAX_L, FGIM_EINVAL, "resolved L out of range");
        const bool bytes = P.X8 && byte_rows_ok(P.d);
        const bool bf16 = !bytes && P.Xh && P.d > 128 && (reinterpret_cast<uintptr_t>(P.Xh) & 7u) == 0;
        const unsigned long long key = beam_shape_key(P.metric, bytes ? 1 : bf16 ? 2 : 4, P.d, L);
        fgim_knng g;
        g.ids = c.alloc<int32_t>(P.N * params->k);
        g.dist = c.alloc<float>(P.N * params->k);
        g.flags = c.alloc<uint8_t>(P.N * params->k);
        g.n = P.N;
        g.k = params->k;
        cudaEvent_t e0, e1;
        ck(cudaEventCreate(&e0));
        ck(cudaEventCreate(&e1));
        const int ht0 = ht_bits_for(L);
        BeamShape best = {4, ht0};
        float best_ms = -1.f;
        bool had = false;
        BeamShape before = best;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                had = true;
                before = it->second;
            }
        }
        const int wpbs[3] = {1, 2, 4};
        for (int wi = 0; wi < 3; ++wi)
            for (int dh = -2; dh <= 1; ++dh) {
                const BeamShape cand = {wpbs[wi], std::min(13, std::max(6, ht0 + dh))};
                if ((size_t)warp_layout(P.d, L, cand.htbits, params->k, !bytes).bytes * cand.wpb > 227 * 1024) continue;
                {
                    std::lock_guard<std::mutex> lk(g_tune_mu);
                    g_tuned[key] = cand;
                }
                stage_a(c, P, params, h, &g);   // warm-up of this shape
                float ms = 0.f;
                for (int rep = 0; rep < 2; ++rep) {
                    ck(cudaEventRecord(e0, c.s));
                    stage_a(c, P, params, h, &g);
                    ck(cudaEventRecord(e1, c.s));
                    ck(cudaEventSynchronize(e1));
                    float t = 0.f;
                    ck(cudaEventElapsedTime(&t, e0, e1));
                    ms = rep == 0 ? t : std::min(ms, t);
                }
                if (best_ms < 0.f || ms < best_ms) {
                    best_ms = ms;
                    best = cand;
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            if (best_ms >= 0.f) g_tuned[key] = best;
            else if (had) g_tuned[key] = before;
            else g_tuned.erase(key);
        }
        c.finish(&t_stats);
        if (cache_path && best_ms >= 0.f) {
            FILE* f = std::fopen(cache_path, "a");
            need(f != nullptr, FGIM_EINVAL, "cannot open the autotune cache file");
            std::fprintf(f,
                         "{\"key\": %llu, \"wpb\": %d, \"ht_bits\": %d, \"ms\": %.4f, \"dim\": %d, \"L\": %d, "
                         "\"row_bytes\": %d, \"metric\": %d}\n",
                         key, best.wpb, best.htbits, best_ms, P.d, L, bytes ? 1 : bf16 ? 2 : 4, P.metric);
            std::fclose(f);
        }
        if (out_wpb) *out_wpb = best.wpb;
        if (out_ht_bits) *out_ht_bits = best.htbits;
        if (out_ms) *out_ms = best_ms;
    });
    end_call();
    return r;
}

fgim_status fgim_autotune_load(const char* cache_path) {
    if (!cache_path) return FGIM_EINVAL;
    FILE* f = std::fopen(cache_path, "r");
    if (!f) return FGIM_EINVAL;
    char line[512];
    int loaded = 0;
    while (std::fgets(line, sizeof(line), f)) {
        unsigned long long key = 0;
        int wpb = 0, hb = 0;
        if (std::sscanf(line, "{\"key\": %llu, \"wpb\": %d, \"ht_bits\": %d", &key, &wpb, &hb) == 3 &&
            (wpb == 1 || wpb == 2 || wpb == 4) && hb >= 6 && hb <= 13) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[key] = BeamShape{wpb, hb};   // a later line for the same key wins
            ++loaded;
        }
    }
    std::fclose(f);
    return loaded > 0 ? FGIM_OK : FGIM_EINVAL;
}

void fgim_autotune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
}

int32_t fgim_test_set(const char* knob, int64_t value) {
    if (!knob) return 0;
    const std::string k(knob);
    if (k == "prop_cap") {
        g_test_prop_cap.store(value > 0 ? (long long)value : 0);
        return 1;
    }
    if (k == "hop_budget") {
        g_test_hop_budget.store(value > 0 ? (int)std::min<int64_t>(value, 0x7fffffff) : 0);
        return 1;
    }
    if (k == "batch_union") {
        g_test_batch_union.store(value != 0 ? 1 : 0);
        return 1;
    }
    if (k == "join_sparse_nn") {
        g_test_sparse_nn.store(value >= 0 ? (int)std::min<int64_t>(value, 1 << 20) : -1);
        return 1;
    }
    if (k == "fail_alloc_after") {
        g_test_fail_after.store(value >= 0 ? (long long)value : -1);
        return 1;
    }
    return 0;
}

int64_t fgim_test_get(const char* what) {
    if (!what) return -1;
    if (std::string(what) == "scratch_allocs") return (int64_t)t_allocs;   // of the last call on this thread
    if (std::string(what) == "pool_used_bytes") {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        std::lock_guard<std::mutex> lk(g_pool_mu);
        auto it = g_pools.find(dev);
        if (it == g_pools.end()) return 0;
        uint64_t used = 0;
        if (cudaMemPoolGetAttribute(it->second, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        return (int64_t)used;
    }
    return -1;
}

void fgim_trim_memory(void) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto& kv : g_pools) cudaMemPoolTrimTo(kv.second, 0);
}

void fgim_last_stats(fgim_stats* out) {
    if (out) *out = t_stats;
}

const char* fgim_strerror(fgim_status s) {
    switch (s) {
        case FGIM_OK: return "ok";
        case FGIM_EINVAL: return "invalid argument";
        case FGIM_ENOMEM: return "out of memory";
        case FGIM_ECUDA: return "CUDA error";
        case FGIM_ETIMEOUT: return "device wait timed out";
        case FGIM_EUNSUPPORTED: return "unsupported configuration";
        case FGIM_EINTERNAL: return "internal error";
    }
    return "unknown status";
}

const char* fgim_last_error(void) { return t_last_error.c_str(); }

const char* fgim_version(void) { return "fgim-gb300 0.1.0 (sm_103a)"; }

int64_t fgim_launch_count(void) { return (int64_t)g_launches.load(); }

void fgim_prof_enable(int32_t on) { g_prof.store(on ? 1 : 0); }

void fgim_prof_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_table.clear();
}

int32_t fgim_prof_query(const char* kernel, int64_t* launches, double* total_ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    auto it = g_prof_table.find(kernel ? kernel : "");
    if (it == g_prof_table.end()) {
        if (launches) *launches = 0;
        if (total_ms) *total_ms = 0.0;
        return 0;
    }
    if (launches) *launches = it->second.launches;
    if (total_ms) *total_ms = it->second.ms;
    return 1;
}

int32_t fgim_prof_names(char* buf, int32_t buf_bytes) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::string all;
    for (auto& kv : g_prof_table) {
        if (!all.empty()) all += ",";
        all += kv.first;
    }
    if (buf && buf_bytes > 0) {
        const size_t n = std::min((size_t)(buf_bytes - 1), all.size());
        std::memcpy(buf, all.data(), n);
        buf[n] = 0;
    }
    return (int32_t)all.size();
}

}  // extern "C"
