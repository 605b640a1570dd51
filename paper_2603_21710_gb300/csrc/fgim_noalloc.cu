// fgim_search_noalloc: the search of fgim_search for callers that must not allocate.
//
// Some callers cannot allocate device memory while they run: code inside a memory-budgeted
// serving process that has handed all its memory to a pool it does not control, real-time
// paths where an allocation (and the implicit synchronisation it may bring) is not allowed,
// and plug-ins loaded into a host that forbids calls into the allocator. fgim_search takes
// its scratch (a status word, counters and, for cosine, inverse norms) from
// cudaMallocAsync on every call; this entry point takes it from one array that lives in the
// library for as long as the library is loaded.
//
// The array is file-scope device memory of fixed size. Host code cannot use its name as an
// address (on the host the name is only a stand-in), so the first call on each device does
// the set-up: it looks the address up with cudaGetSymbolAddress while that device is current
// (with lazy module loading this is also when the array comes into being) and remembers it.
// Make that first call outside any stream capture. Every call shares the array: calls that
// overlap on the GPU (other streams, other host threads) race on it and must be serialised
// by the caller. Nothing here allocates; failures return a status code and leave
// fgim_last_error() untouched. Keep launch profiling (fgim_prof_enable) off for these calls:
// its event bookkeeping allocates.
#include <cstring>
#include <mutex>
#include <string>

#include "fgim_launch.h"

namespace fgim {

// largest base set and query batch whose cosine norms fit the array
constexpr long long kNoAllocMaxBase = 1LL << 20;
constexpr long long kNoAllocMaxQueries = 1LL << 16;
constexpr size_t kNoAllocHeader = 256;   // status word (int) and two 64-bit counters, padded
constexpr size_t kNoAllocBytes = kNoAllocHeader + (size_t)(kNoAllocMaxBase + kNoAllocMaxQueries) * sizeof(float);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
constexpr int kNoAllocMaxDevices = 64;
static void* g_noalloc_ptr[kNoAllocMaxDevices] = {};   // per device ordinal

// Failures are reported by status code only: recording a message could allocate.
static fgim_status noalloc_fail(fgim_status st, const char* msg) {
    (void)msg;
    return st;
}

}  // namespace fgim

using namespace fgim;

extern "C" {

fgim_status fgim_search_noalloc(const void* base, int64_t n, int32_t dim, int32_t dtype, int32_t metric,
                                const int32_t* graph_ids, int32_t R, int32_t entry, const void* queries, int32_t nq,
                                int32_t topk, int32_t beam, int32_t* out_ids, float* out_dist, void* stream) {
    if (!base || !graph_ids || !queries || !out_ids || !out_dist) return noalloc_fail(FGIM_EINVAL, "NULL buffer");
    if (n < 1 || n >= 0x7fffffffLL) return noalloc_fail(FGIM_EINVAL, "bad n");
    if (dim < 4 || dim > FGIM_MAX_DIM || dim % 4 != 0)
        return noalloc_fail(FGIM_EINVAL, "dim must be a multiple of 4 in [4, 2048]");
    if (dtype != FGIM_F32) return noalloc_fail(FGIM_EUNSUPPORTED, "only FP32 vector storage is supported");
    if (metric != FGIM_L2SQ && metric != FGIM_IP && metric != FGIM_COSINE) return noalloc_fail(FGIM_EINVAL, "unknown metric");
    if (R < 1 || R > FGIM_MAX_DEGREE) return noalloc_fail(FGIM_EINVAL, "R must be in [1, 128]");
    if (entry < 0 || entry >= n) return noalloc_fail(FGIM_EINVAL, "entry out of range");
    if (nq < 0) return noalloc_fail(FGIM_EINVAL, "nq must be >= 0");
    if (beam < 1 || beam > FGIM_MAX_L || topk < 1 || topk > beam)
        return noalloc_fail(FGIM_EINVAL, "need 1 <= topk <= beam <= 128");
    if (((uintptr_t)base & 15u) != 0 || ((uintptr_t)queries & 15u) != 0)
        return noalloc_fail(FGIM_EINVAL, "vectors must be 16-byte aligned");
    if (metric == FGIM_COSINE && (n > kNoAllocMaxBase || nq > kNoAllocMaxQueries))
        return noalloc_fail(FGIM_EINVAL,
                            "cosine search without allocation holds at most 1,048,576 base vectors and 65,536 queries");
    if (nq == 0) return FGIM_OK;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
        return noalloc_fail(FGIM_ECUDA, "no current CUDA device");
    unsigned char* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return noalloc_fail(FGIM_ECUDA, "symbol lookup failed");
            g_noalloc_ptr[dev] = p;
        }
        scratch = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
    }
    cudaStream_t s = (cudaStream_t)stream;
    int* status = reinterpret_cast<int*>(scratch);
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(scratch + 64);
    float* inv = reinterpret_cast<float*>(scratch + kNoAllocHeader);
    float* qinv = inv + kNoAllocMaxBase;
    cudaError_t e = cudaMemsetAsync(scratch, 0, kNoAllocHeader, s);   // the status and counters start at zero
    const float* X = static_cast<const float*>(base);
    const float* Q = static_cast<const float*>(queries);
    if (e == cudaSuccess && metric == FGIM_COSINE) {
        e = launch_inv_norms(X, n, dim, inv, s);
        if (e == cudaSuccess) e = launch_inv_norms(Q, nq, dim, qinv, s);
    }
    if (e == cudaSuccess)
        e = launch_search(X, nullptr, metric == FGIM_COSINE ? inv : nullptr, n, dim, metric, graph_ids, R, entry, Q,
                          metric == FGIM_COSINE ? qinv : nullptr, nullptr, nq, topk, beam, out_ids, out_dist, counters,
                          status, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int hstatus = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return noalloc_fail(FGIM_ECUDA, "CUDA error");
    if (hstatus & kErrTimeout) return noalloc_fail(FGIM_ETIMEOUT, "a bounded device loop ran out");
    if (hstatus & kErrBounds) return noalloc_fail(FGIM_EINVAL, "an index is out of range (graph ids or entry)");
    return FGIM_OK;
}

}  // extern "C"
