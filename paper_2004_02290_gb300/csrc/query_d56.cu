// Query kernel instances for d = 5 and d = 6 (one translation unit per pair,
// so the build compiles them in parallel).
#include "query_kernel.cuh"

namespace ghn {

cudaError_t launch_query_d56(const QueryArgs& a, int blocks, cudaStream_t s)
{
    switch (a.g.d) {
    case 5: return qk::launch_d<5>(a, blocks, s);
    case 6: return qk::launch_d<6>(a, blocks, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ghn
