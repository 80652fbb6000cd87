// Query kernel instances for d = 5 and d = 6 (one translation unit per pair,
// so the build compiles them in parallel).
#include "query_kernel.cuh"

namespace ghn {

cudaError_t launch_query_d56(const QueryArgs& a, int sms, cudaStream_t s)
{
    switch (a.g.d) {
    case 5: return qk::launch_d<5>(a, sms, s);
    case 6: return qk::launch_d<6>(a, sms, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_query_d56(const BatchArgs& g, int sms, cudaStream_t s)
{
    switch (g.d) {
    case 5: return qk::launch_batch_d<5>(g, sms, s);
    case 6: return qk::launch_batch_d<6>(g, sms, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ghn
