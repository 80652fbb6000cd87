// Query kernel instances for d = 3 and d = 4 (one translation unit per pair,
// so the build compiles them in parallel).
#include "query_kernel.cuh"

namespace ghn {

cudaError_t launch_query_d34(const QueryArgs& a, int sms, cudaStream_t s)
{
    switch (a.g.d) {
    case 3: return qk::launch_d<3>(a, sms, s);
    case 4: return qk::launch_d<4>(a, sms, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_query_d34(const BatchArgs& g, int sms, cudaStream_t s)
{
    switch (g.d) {
    case 3: return qk::launch_batch_d<3>(g, sms, s);
    case 4: return qk::launch_batch_d<4>(g, sms, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ghn
