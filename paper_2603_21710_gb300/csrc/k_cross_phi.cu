// Stage (a), Alg. 2 with the ID mapping of invalid vertices (Sec. 4.1.3): the PHI form of the
// cross query, compiled on its own.
#include "k_cross.cuh"

namespace fgim {

template cudaError_t launch_cross_query_t<true>(const ShardTable&, const float*, const uint8_t*, const float*,
                                                long long, int, int, int, fgim_knng*, unsigned long long*, int*,
                                                cudaStream_t, const int32_t*, const int32_t*, long long,
                                                const uint16_t*);

}  // namespace fgim
