// Query kernel instances for d = 1 and d = 2 (one translation unit per pair,
// so the build compiles them in parallel).
#include "query_kernel.cuh"

namespace ghn {

cudaError_t launch_query_d12(const QueryArgs& a, int sms, cudaStream_t s)
{
    switch (a.g.d) {
    case 1: return qk::launch_d<1>(a, sms, s);
    case 2: return qk::launch_d<2>(a, sms, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_query_d12(const BatchArgs& g, int sms, cudaStream_t s)
{
    switch (g.d) {
    case 1: return qk::launch_batch_d<1>(g, sms, s);
    case 2: return qk::launch_batch_d<2>(g, sms, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ghn
