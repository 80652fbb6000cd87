// knn_query_noalloc: batched query that allocates no memory.
//
// Some callers cannot allocate device memory when they query: a process whose
// own allocator has already reserved the GPU's memory (a cudaMalloc would fail
// or force it to release cached blocks), a serving loop that must not pay an
// allocation's latency or its implicit synchronisation, or code whose rules
// forbid allocation after start-up.  For them this entry point runs the same
// query kernels as knn_query, with the kernels' scratch memory (work counters,
// status word and the list of queries handed to the cooperative kernel) in a
// fixed array below instead of memory allocated per call.  Inputs and outputs
// are the caller's device buffers.
//
// The array is a file-scope __device__ variable, so every GPU that loads this
// library holds it (kNoAllocScratchBytes, about 4 MiB) until the process
// exits.  All calls share it: two calls whose kernels overlap on the GPU race
// on it, so calls must be ordered (one stream, or synchronised).  The
// counters are cleared at the start of every call; the rest is overwritten
// before it is read.

#include "ghn_internal.cuh"
#include "../../include/ghn_knn.h"

#include <string.h>

#include <mutex>

namespace {

constexpr unsigned int kNoAllocMaxQueries = 1u << 20;   // largest m accepted
constexpr size_t kCounterBytes = 32;                      // counter, status, deferral counters
constexpr size_t kNoAllocScratchBytes = kCounterBytes + 4ull * kNoAllocMaxQueries;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// The array's device address, taken once per device with that device current
// (in host code the symbol itself is only a host-side stand-in).
std::mutex g_setup_mutex;
void* g_scratch_addr[64] = {nullptr};

knn_status scratch_for(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= 64) {
        ghn::set_error("knn_query_noalloc: device ordinal out of range");
        return KNN_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            ghn::set_error("knn_query_noalloc: cudaGetSymbolAddress of the scratch array failed");
            return KNN_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return KNN_OK;
}

// Device memory of GPU `dev` (managed memory is reachable from every GPU).
// Memory of another GPU is refused: the kernels would reach it as a peer
// address, with no peer access set up.
bool on_device(const void* p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}

}  // namespace

extern "C" knn_status knn_query_noalloc(const ghn_index* index, const float* queries, int64_t m,
                                        int32_t k, int32_t mode, int32_t* ids, float* dist2,
                                        void* pred, int32_t flags, void* stream)
{
    if (!index) {
        ghn::set_error("knn_query_noalloc: index is NULL");
        return KNN_EINVAL;
    }
    if (m < 0 || m > (int64_t)kNoAllocMaxQueries) {
        ghn::set_error("knn_query_noalloc: m must be in [0, 1048576]; the fixed scratch array "
                       "holds at most 1048576 queries per call");
        return KNN_EINVAL;
    }
    if (k < 1 || k > ghn::kMaxK || mode < -1 || mode > 2) {
        ghn::set_error("knn_query_noalloc: k must be in [1, 64] and mode in {-1, 0, 1, 2}");
        return KNN_EINVAL;
    }
    if (mode >= 0 && !ghn::index_has_labels(index)) {
        ghn::set_error("knn_query_noalloc: a prediction needs labels, and the index has none");
        return KNN_EINVAL;
    }
    if (flags & ~(KNN_QUERY_CHECKED | KNN_QUERY_EXACT)) {
        ghn::set_error("knn_query_noalloc: only KNN_QUERY_CHECKED and KNN_QUERY_EXACT are "
                       "supported (the locality order needs sort buffers)");
        return KNN_EINVAL;
    }
    if (m == 0) return KNN_OK;
    if (!queries || !ids || (mode >= 0 && !pred)) {
        ghn::set_error("knn_query_noalloc: queries, ids (and pred for a prediction) are required");
        return KNN_EINVAL;
    }
    int prev = -1;
    const int dev = ghn::index_device(index);
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
    knn_status st = KNN_OK;
    do {
        if (!on_device(queries, dev) || !on_device(ids, dev) || (dist2 && !on_device(dist2, dev)) ||
            (mode >= 0 && !on_device(pred, dev))) {
            ghn::set_error("knn_query_noalloc: every buffer must be device memory of the index's "
                           "GPU (host data would need a staging allocation)");
            st = KNN_EINVAL;
            break;
        }
        unsigned char* scratch = nullptr;
        st = scratch_for(dev, &scratch);
        if (st != KNN_OK) break;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        // counters start at zero; the deferred list is written before it is read
        cudaError_t e = cudaMemsetAsync(scratch, 0, kCounterBytes, s);
        if (e == cudaSuccess) {
            ghn::QueryArgs a;
            memset(&a, 0, sizeof(a));
            ghn::index_query_args(index, a);
            a.q = queries;
            a.m = m;
            a.k = k;
            a.mode = mode;
            a.ids = ids;
            a.dist2 = dist2;
            a.pred = mode >= 0 ? pred : nullptr;
            a.exact = (flags & KNN_QUERY_EXACT) ? 1 : 0;
            a.counter = reinterpret_cast<unsigned long long*>(scratch);
            a.status = reinterpret_cast<unsigned int*>(scratch + 8);
            a.heavy_count = reinterpret_cast<unsigned int*>(scratch + 16);
            a.heavy_cursor = reinterpret_cast<unsigned int*>(scratch + 20);
            a.heavy_list = reinterpret_cast<unsigned int*>(scratch + kCounterBytes);
            e = ghn::launch_query(a, ghn::device_sms(dev), s);
        }
        if (e == cudaSuccess) ghn::index_mark_use(index, s);
        if (e == cudaSuccess && (flags & KNN_QUERY_CHECKED)) {
            unsigned int status = 0u;
            e = cudaMemcpyAsync(&status, scratch + 8, sizeof(status), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e == cudaSuccess && (status & ghn::kStatusNonFinite)) {
                ghn::set_error("knn_query_noalloc: a query coordinate is not finite");
                st = KNN_EINVAL;
            } else if (e == cudaSuccess && (status & ghn::kStatusLimit)) {
                ghn::set_error("knn_query_noalloc: a query reached its work bound (rows or layer cap)");
                st = KNN_ELIMIT;
            }
        }
        if (e != cudaSuccess) {
            ghn::set_error(cudaGetErrorString(e));
            st = KNN_ECUDA;
        }
    } while (false);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return st;
}
