// Stage (a), Alg. 2: the cross query over every vertex (the plain ID mapping), and the
// entry point that picks the form.
#include "k_cross.cuh"

namespace fgim {

cudaError_t launch_cross_query(const ShardTable& t, const float* X, const uint8_t* X8, const float* inv_norm,
                               long long N, int metric, int k, int L, fgim_knng* out, unsigned long long* counters,
                               int* status, cudaStream_t s, const int32_t* phi, const int32_t* src, long long nq,
                               const uint16_t* Xh) {
    if (nq < 0) nq = N;
    if ((phi == nullptr) != (src == nullptr)) return cudaErrorInvalidValue;
    if (phi)
        return launch_cross_query_t<true>(t, X, X8, inv_norm, N, metric, k, L, out, counters, status, s, phi, src, nq,
                                          Xh);
    return launch_cross_query_t<false>(t, X, X8, inv_norm, N, metric, k, L, out, counters, status, s, nullptr, nullptr,
                                       nq, Xh);
}

}  // namespace fgim
