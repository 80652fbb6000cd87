// Query kernel instances for d = 7 and d = 8 (one translation unit per pair,
// so the build compiles them in parallel).
#include "query_kernel.cuh"

namespace ghn {

cudaError_t launch_query_d78(const QueryArgs& a, int sms, cudaStream_t s)
{
    switch (a.g.d) {
    case 7: return qk::launch_d<7>(a, sms, s);
    case 8: return qk::launch_d<8>(a, sms, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_query_d78(const BatchArgs& g, int sms, cudaStream_t s)
{
    switch (g.d) {
    case 7: return qk::launch_batch_d<7>(g, sms, s);
    case 8: return qk::launch_batch_d<8>(g, sms, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ghn
