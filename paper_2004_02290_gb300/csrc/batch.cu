// Batched indexes: build many independent indexes in one pass and query all
// of them in one persistent launch per dimension.
//
// The method is the same as for one index (Sec. III.A-B): each index has its
// own grid (origin, width, cells per dimension) and its own cell table.  The
// batch only changes how the work is laid out on the GPU:
//   - every stage of the build is one launch over the points of all indexes
//     (tiles of points tagged with their index), with a single host read of
//     all the boxes;
//   - the cell key carries the index in its high bits, so one stable radix
//     sort groups the points of every index by cell, index after index;
//   - dense tables and occupancy bitmaps are segments of shared buffers, and
//     the indexes with hash tables share one open-addressing table keyed by
//     (index, cell);
//   - queries of all indexes with the same dimension run in one persistent
//     launch; a plan captures those launches in a CUDA graph for replay.

#include "build_launch.cuh"
#include "ghn_internal.cuh"
#include "../../include/ghn_knn.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

using namespace ghn;

namespace {

constexpr int kTilePoints = 4096;
constexpr int kBoxThreads = 256;
constexpr int kPartStride = 2 * kMaxD + 1;  // floats per partial box

// Per-index data the build kernels need.
struct BuildDesc {
    const float* points;           // n * d, caller's device memory
    const unsigned int* labels;    // n or null
    long long n;
    long long off;                 // first point in the concatenation (and first sorted row)
    long long rows_off;            // first float of the index's rows
    long long dense_off;           // first entry of its dense table, or -1
    long long bitmap_off;          // first word of its occupancy bitmap, or -1
    int d;
    int p;                         // floats per stored row
    GridConst g;
};

// The part of a descriptor the row gather reads for every row (32 bytes).
struct __align__(16) GatherDesc {
    const float* points;
    long long off;
    long long rows_off;
    int d;
    int p;
};

struct Tile {
    int index;
    int count;
    long long first;  // first point (local to the index)
};

__global__ void __launch_bounds__(kBoxThreads)
    batch_box_partial_kernel(const BuildDesc* __restrict__ descs, const Tile* __restrict__ tiles,
                             float* __restrict__ partial)
{
    __shared__ float slo[kMaxD][kBoxThreads];
    __shared__ float shi[kMaxD][kBoxThreads];
    __shared__ int sbad;
    const Tile tile = tiles[blockIdx.x];
    const BuildDesc& ds = descs[tile.index];
    const int d = ds.d, t = threadIdx.x;
    if (t == 0) sbad = 0;
    float lo[kMaxD], hi[kMaxD];
#pragma unroll
    for (int j = 0; j < kMaxD; ++j) {
        lo[j] = INFINITY;
        hi[j] = -INFINITY;
    }
    bool bad = false;
    for (int i = t; i < tile.count; i += kBoxThreads) {
        const float* p = ds.points + (tile.first + i) * d;
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) {
            if (j < d) {
                const float v = __ldg(p + j);
                bad |= !isfinite(v);
                lo[j] = fminf(lo[j], v);
                hi[j] = fmaxf(hi[j], v);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kMaxD; ++j) {
        slo[j][t] = lo[j];
        shi[j][t] = hi[j];
    }
    __syncthreads();
    if (bad) sbad = 1;
    for (int half = kBoxThreads / 2; half > 0; half >>= 1) {
        if (t < half) {
#pragma unroll
            for (int j = 0; j < kMaxD; ++j) {
                slo[j][t] = fminf(slo[j][t], slo[j][t + half]);
                shi[j][t] = fmaxf(shi[j][t], shi[j][t + half]);
            }
        }
        __syncthreads();
    }
    if (t < kMaxD) {
        partial[(size_t)blockIdx.x * kPartStride + t] = slo[t][0];
        partial[(size_t)blockIdx.x * kPartStride + kMaxD + t] = shi[t][0];
    }
    if (t == 0) partial[(size_t)blockIdx.x * kPartStride + 2 * kMaxD] = sbad ? 1.0f : 0.0f;
}

// One block per index: fold the index's tiles, then cells per dimension.
__global__ void __launch_bounds__(kBoxThreads)
    batch_box_final_kernel(const BuildDesc* __restrict__ descs,
                           const int* __restrict__ tile_first, const float* __restrict__ partial,
                           const float* __restrict__ widths, BoxOut* __restrict__ out)
{
    __shared__ float slo[kMaxD][kBoxThreads];
    __shared__ float shi[kMaxD][kBoxThreads];
    __shared__ int sbad;
    const int i = blockIdx.x, t = threadIdx.x;
    const int d = descs[i].d;
    if (t == 0) sbad = 0;
    float lo[kMaxD], hi[kMaxD];
#pragma unroll
    for (int j = 0; j < kMaxD; ++j) {
        lo[j] = INFINITY;
        hi[j] = -INFINITY;
    }
    bool bad = false;
    for (int b = tile_first[i] + t; b < tile_first[i + 1]; b += kBoxThreads) {
        const float* p = partial + (size_t)b * kPartStride;
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) {
            lo[j] = fminf(lo[j], p[j]);
            hi[j] = fmaxf(hi[j], p[kMaxD + j]);
        }
        bad |= p[2 * kMaxD] != 0.0f;
    }
#pragma unroll
    for (int j = 0; j < kMaxD; ++j) {
        slo[j][t] = lo[j];
        shi[j][t] = hi[j];
    }
    __syncthreads();
    if (bad) sbad = 1;
    for (int half = kBoxThreads / 2; half > 0; half >>= 1) {
        if (t < half) {
#pragma unroll
            for (int j = 0; j < kMaxD; ++j) {
                slo[j][t] = fminf(slo[j][t], slo[j][t + half]);
                shi[j][t] = fmaxf(shi[j][t], shi[j][t + half]);
            }
        }
        __syncthreads();
    }
    if (t == 0) {
        unsigned int flags = 0u;
        const float w = widths[i];
        BoxOut& o = out[i];
        for (int j = 0; j < d; ++j) {
            const float l = slo[j][0], h = shi[j][0];
            o.lo[j] = l;
            o.hi[j] = h;
            long long ext = 0;
            if (sbad || !(l <= h)) {
                flags |= kStatusNonFinite;
            } else {
                // ext_j = floor((hi_j - lo_j) / w) + 1, Eq. 1 at the largest point
                const float q = __fdiv_rn(__fsub_rn(h, l), w);
                if (!(q < 2147483647.0f))
                    flags |= kStatusExtent;
                else
                    ext = (long long)floorf(q) + 1;
            }
            o.ext[j] = ext;
        }
        o.flags = flags;
    }
}

// Eq. 1 for every point of every index: key = index << shift | cell id.
__global__ void __launch_bounds__(256)
    batch_keys_kernel(const BuildDesc* __restrict__ descs, const Tile* __restrict__ tiles,
                      int shift, unsigned long long* __restrict__ keys,
                      unsigned int* __restrict__ vals)
{
    const Tile tile = tiles[blockIdx.x];
    const BuildDesc& ds = descs[tile.index];
    const int d = ds.d;
    const unsigned long long prefix = (unsigned long long)tile.index << shift;
    for (int i = threadIdx.x; i < tile.count; i += blockDim.x) {
        const long long local = tile.first + i;
        const float* p = ds.points + local * d;
        unsigned long long key = 0ull;
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) {
            if (j < d) {
                const float t = __fdiv_rn(__fsub_rn(__ldg(p + j), ds.g.lo[j]), ds.g.w[j]);
                key += (unsigned long long)(long long)floorf(t) * ds.g.stride[j];
            }
        }
        keys[ds.off + local] = prefix | key;
        vals[ds.off + local] = (unsigned int)(ds.off + local);
    }
}

// Dense tables: the row count of each cell at its id in the index's segment.
__global__ void batch_dense_counts_kernel(const BuildDesc* __restrict__ descs, int shift,
                                          const unsigned long long* __restrict__ cell_key,
                                          const unsigned int* __restrict__ cell_start,
                                          const GridDev* __restrict__ gdev,
                                          unsigned int* __restrict__ dense)
{
    const unsigned long long u = gdev->ncells;
    const unsigned long long low = (1ull << shift) - 1ull;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < (long long)u;
         c += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = cell_key[c];
        const BuildDesc& ds = descs[key >> shift];
        if (ds.dense_off >= 0)
            dense[ds.dense_off + (long long)(key & low)] = cell_start[c + 1] - cell_start[c];
    }
}

// After one exclusive scan over all dense segments, make each segment's
// entries local to its index: subtract the value at the segment's start.
__global__ void batch_seg_base_kernel(const long long* __restrict__ seg_off, int nseg,
                                      const unsigned int* __restrict__ dense,
                                      unsigned int* __restrict__ base)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nseg) base[k] = dense[seg_off[k]];
}

__global__ void batch_dense_fixup_kernel(const long long* __restrict__ seg_off, int nseg,
                                         const unsigned int* __restrict__ seg_base,
                                         long long total, unsigned int* __restrict__ dense)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = nseg - 1;  // the last segment starting at or before e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg_off[mid] <= e)
                lo = mid;
            else
                hi = mid - 1;
        }
        dense[e] -= seg_base[lo];
    }
}

// Cells of hash-table indexes into the shared table, with rows local to their
// index; occupancy bits of indexes that have a bitmap.
__global__ void batch_hash_insert_kernel(const BuildDesc* __restrict__ descs, int shift,
                                         const unsigned long long* __restrict__ cell_key,
                                         const unsigned int* __restrict__ cell_start,
                                         const GridDev* __restrict__ gdev, HashSlot* slots,
                                         unsigned int* __restrict__ bitmap)
{
    const unsigned long long u = gdev->ncells, mask = gdev->hmask;
    const unsigned long long low = (1ull << shift) - 1ull;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < (long long)u;
         c += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = cell_key[c];
        const BuildDesc& ds = descs[key >> shift];
        if (ds.dense_off >= 0) continue;
        if (ds.bitmap_off >= 0) {
            const unsigned long long id = key & low;
            atomicOr(bitmap + ds.bitmap_off + (long long)(id >> 5), 1u << (unsigned)(id & 31ull));
        }
        unsigned long long h = mix64(key) & mask;
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            const unsigned long long prev = atomicCAS(&slots[h].key, kEmptyKey, key);
            if (prev == kEmptyKey) {
                slots[h].start = cell_start[c] - (unsigned int)ds.off;
                slots[h].end = cell_start[c + 1] - (unsigned int)ds.off;
                break;
            }
            h = (h + 1ull) & mask;
        }
    }
}

// Rows into cell order, padded per index; the training index of each row
// local to its index; the labels of every index.
__global__ void __launch_bounds__(256)
    batch_gather_kernel(const GatherDesc* __restrict__ descs, int shift, long long total,
                        const unsigned long long* __restrict__ keys,
                        const unsigned int* __restrict__ vals, float* __restrict__ rows,
                        unsigned int* __restrict__ rid)
{
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < total;
         r += (long long)gridDim.x * blockDim.x) {
        const GatherDesc ds = descs[keys[r] >> shift];
        const long long local = r - ds.off;
        const long long src = (long long)vals[r] - ds.off;
        const float* p = ds.points + src * ds.d;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = j < ds.d ? __ldg(p + j) : 0.0f;
        // rows of every index start on 16 bytes: 8- or 16-byte stores
        float* o = rows + ds.rows_off + local * ds.p;
        if (ds.p == 2) {
            *reinterpret_cast<float2*>(o) = make_float2(v[0], v[1]);
        } else {
            reinterpret_cast<float4*>(o)[0] = make_float4(v[0], v[1], v[2], v[3]);
            if (ds.p == 8) reinterpret_cast<float4*>(o)[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
        rid[r] = (unsigned int)src;
    }
}

__global__ void __launch_bounds__(256)
    batch_labels_kernel(const BuildDesc* __restrict__ descs, const Tile* __restrict__ tiles,
                        unsigned int* __restrict__ labels)
{
    const Tile tile = tiles[blockIdx.x];
    const BuildDesc& ds = descs[tile.index];
    if (!ds.labels) return;
    for (int i = threadIdx.x; i < tile.count; i += blockDim.x)
        labels[ds.off + tile.first + i] = __ldg(ds.labels + tile.first + i);
}

int grid_blocks(long long work)
{
    long long b = (work + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// Device memory of the current GPU (the batch's), or managed memory.  Memory
// of another GPU is refused: the kernels would reach it as a peer address
// with no peer access set up.
bool is_device(const void* p)
{
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    int cur = -1;
    return at.type == cudaMemoryTypeDevice && cudaGetDevice(&cur) == cudaSuccess &&
           at.device == cur;
}

// Where a caller buffer lives.
enum { kOtherGpu = -1, kHostMem = 0, kDeviceMem = 1, kMappedHost = 2 };

// kDeviceMem: device memory of the current GPU, or managed memory;
// kMappedHost: pinned host memory the GPU addresses (NVLink-C2C on GB300),
// with its device address in *dptr; kHostMem: other host memory; kOtherGpu:
// device memory of another GPU (refused).
int pointer_kind(const void* p, void** dptr)
{
    if (dptr) *dptr = nullptr;
    if (!p) return kHostMem;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return kHostMem;
    }
    if (at.type == cudaMemoryTypeManaged) return kDeviceMem;
    if (at.type == cudaMemoryTypeDevice) {
        int cur = -1;
        return cudaGetDevice(&cur) == cudaSuccess && at.device == cur ? kDeviceMem : kOtherGpu;
    }
    if (at.type == cudaMemoryTypeHost && at.devicePointer) {
        if (dptr) *dptr = at.devicePointer;
        return kMappedHost;
    }
    return kHostMem;
}


}  // namespace

namespace ghn {

// Phase names of the batched query kernels (static strings for the timer).
const char* group_phase_name(int d, int ns, int dense, int exact, bool coop)
{
    static char names[kMaxD + 1][2][2][2][2][40];
    static std::once_flag once;
    std::call_once(once, [] {
        for (int dd = 0; dd <= kMaxD; ++dd)
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int c = 0; c < 2; ++c)
                        for (int h = 0; h < 2; ++h)
                            snprintf(names[dd][a][b][c][h], sizeof(names[dd][a][b][c][h]),
                                     "query.d%d.%s.%s%s%s", dd, a ? "k64" : "k32",
                                     b ? "dense" : "hash", c ? ".exact" : "", h ? ".coop" : "");
    });
    if (d < 0 || d > kMaxD) d = 0;
    return names[d][ns == 2 ? 1 : 0][dense ? 1 : 0][exact ? 1 : 0][coop ? 1 : 0];
}

}  // namespace ghn

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct ghn_batch {
    int device = 0;
    int count = 0;
    std::vector<knn_index_info_t> info;
    std::vector<QueryArgs> proto;  // the index part of each index's query arguments
    // storage shared by the indexes
    float* rows = nullptr;
    unsigned int* rid = nullptr;
    unsigned int* labels = nullptr;
    unsigned int* dense = nullptr;
    HashSlot* slots = nullptr;
    unsigned int* bitmap = nullptr;
    GridDev* gdev = nullptr;
    cudaEvent_t last_use = nullptr;
};

struct ghn_plan {
    const ghn_batch* batch = nullptr;
    int device = 0;
    void* dev_buf = nullptr;  // arguments, offsets, counters and deferred lists
    unsigned int* status = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<BatchArgs> groups;
    size_t counter_bytes = 0;
    unsigned long long* counters = nullptr;
};

namespace {

void free_batch(ghn_batch* b)
{
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaStream_t s = 0;
    if (b->last_use) cudaStreamWaitEvent(s, b->last_use, 0);
    device_free(b->rows, s);
    device_free(b->rid, s);
    device_free(b->labels, s);
    device_free(b->dense, s);
    device_free(b->slots, s);
    device_free(b->bitmap, s);
    device_free(b->gdev, s);
    if (b->last_use) cudaEventDestroy(b->last_use);
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    delete b;
}

// Device buffers of one build, freed on every exit path.
struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t s_) : s(s_) {}
    template <class T>
    knn_status alloc(T** p, size_t count, const char* what)
    {
        void* v = nullptr;
        knn_status st = device_alloc(&v, count * sizeof(T), s, what);
        *p = static_cast<T*>(v);
        if (st == KNN_OK) ptrs.push_back(v);
        return st;
    }
    ~Scratch()
    {
        for (void* p : ptrs) device_free(p, s);
    }
};

// Copies of pinned host inputs on the device's side stream, so that they
// overlap work already queued on the caller's stream (the host link is the
// bound of a host-buffer step).  begin() orders the side stream after
// everything queued on the caller's stream so far (the staging buffer's
// allocation, earlier copies); end() makes the caller's stream wait for the
// copies.  The destructor ends them too, so that no exit path frees a
// buffer that a copy still writes.
struct SideCopies {
    cudaStream_t s;
    cudaStream_t side = nullptr;
    cudaEvent_t ev = nullptr;
    bool pending = false;
    bool recorded = false;  // end() recorded the copies' event
    explicit SideCopies(cudaStream_t s_) : s(s_) {}
    // false: no side stream (the caller copies on its own stream)
    bool begin(int dev)
    {
        if (!open(dev)) return false;
        pending = false;
        if (cudaEventRecord(ev, s) != cudaSuccess || cudaStreamWaitEvent(side, ev, 0) != cudaSuccess) {
            cudaGetLastError();
            side = nullptr;
            return false;
        }
        return true;
    }
    // The side stream without ordering it after the caller's: for copies
    // into a buffer that is also allocated on the side stream.  The caller's
    // stream waits for the side stream at end() even if nothing is copied.
    bool open(int dev)
    {
        side = copy_stream(dev);
        if (side && !ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            ev = nullptr;
        }
        if (!side || !ev) {
            side = nullptr;
            return false;
        }
        pending = true;
        return true;
    }
    cudaError_t copy(void* dst, const void* src, size_t bytes)
    {
        pending = true;
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, side);
    }
    cudaError_t end()
    {
        if (!pending) return cudaSuccess;
        pending = false;
        cudaError_t e = cudaEventRecord(ev, side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
        if (e != cudaSuccess) cudaStreamSynchronize(side);
        recorded = e == cudaSuccess;
        return e;
    }
    // The host waits until the copies have read their sources, so that the
    // caller may reuse its pinned buffers once the call returns (the GPU
    // keeps the work queued on the caller's stream meanwhile).
    cudaError_t wait_host()
    {
        if (!recorded) return cudaSuccess;
        recorded = false;
        return cudaEventSynchronize(ev);
    }
    ~SideCopies()
    {
        end();
        if (ev) cudaEventDestroy(ev);
    }
};

knn_status fail(const char* msg, knn_status code)
{
    set_error(msg);
    return code;
}

knn_status cuda_error(cudaError_t e, const char* what)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    set_error(buf);
    return e == cudaErrorMemoryAllocation ? KNN_ENOMEM : KNN_ECUDA;
}

template <class T>
knn_status upload(Scratch& sc, const std::vector<T>& host, T** dev, const char* what)
{
    knn_status st = sc.alloc(dev, host.size() ? host.size() : 1, what);
    if (st != KNN_OK) return st;
    if (host.empty()) return KNN_OK;
    // A copy from pageable host memory returns once the source has been
    // staged (or copied), so the vector may go away right after: no wait,
    // and no bubble in the stream's work.
    const cudaError_t e = cudaMemcpyAsync(*dev, host.data(), host.size() * sizeof(T),
                                          cudaMemcpyHostToDevice, sc.s);
    return e == cudaSuccess ? KNN_OK : cuda_error(e, what);
}

knn_status batch_build_impl(int count, const float* const* points, const void* const* labels,
                            const int64_t* n, const int32_t* d, const float* width,
                            const int32_t* table, cudaStream_t s, ghn_batch** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    tune_device_pool(dev);
    ghn_batch* b = new ghn_batch();
    b->device = dev;
    b->count = count;
    auto bail = [&](knn_status code) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        free_batch(b);
        return code;
    };
    knn_status st = KNN_OK;
    phase_begin(s);
    {
        Scratch sc(s);
        SideCopies lab_copies(s);  // after sc: ends before sc frees the staging buffer
        struct LateCopy {
            void* dst;
            const void* src;
            size_t bytes;
        };
        std::vector<LateCopy> late_labels;
        // ---- host inputs: copied into one device buffer (16-byte aligned slices);
        // pinned host labels go over on the side stream once the boxes are
        // read back, while the sort, cells and table kernels run (issued
        // earlier, they held up the boxes' read-back on the copy engine) ----
        std::vector<const float*> pdev(points, points + count);
        std::vector<const void*> ldev(count, nullptr);
        if (labels) ldev.assign(labels, labels + count);
        {
            const size_t none = ~(size_t)0;
            std::vector<size_t> p_at(count, none), l_at(count, none);
            size_t words = 0;
            for (int i = 0; i < count; ++i) {
                if (pointer_kind(points[i], nullptr) != kDeviceMem) {
                    words = (words + 3) & ~(size_t)3;
                    p_at[i] = words;
                    words += (size_t)n[i] * (size_t)d[i];
                }
                if (ldev[i] && pointer_kind(ldev[i], nullptr) != kDeviceMem) {
                    words = (words + 3) & ~(size_t)3;
                    l_at[i] = words;
                    words += (size_t)n[i];
                }
            }
            if (words > 0) {
                float* stage = nullptr;
                if ((st = sc.alloc(&stage, words, "batch staged inputs")) != KNN_OK) return bail(st);
                for (int i = 0; i < count && e == cudaSuccess; ++i) {
                    if (p_at[i] != none) {
                        e = cudaMemcpyAsync(stage + p_at[i], points[i],
                                            (size_t)n[i] * (size_t)d[i] * 4, cudaMemcpyHostToDevice, s);
                        pdev[i] = stage + p_at[i];
                    }
                }
                for (int i = 0; i < count && e == cudaSuccess; ++i) {
                    if (l_at[i] == none) continue;
                    if (pointer_kind(ldev[i], nullptr) == kMappedHost)
                        late_labels.push_back(LateCopy{stage + l_at[i], ldev[i], (size_t)n[i] * 4});
                    else
                        e = cudaMemcpyAsync(stage + l_at[i], ldev[i], (size_t)n[i] * 4,
                                            cudaMemcpyHostToDevice, s);
                    ldev[i] = stage + l_at[i];
                }
                if (e != cudaSuccess) return bail(cuda_error(e, "batch staged inputs"));
            }
        }
        phase_mark("stage", s);
        // ---- per-index descriptors and tiles ----
        std::vector<BuildDesc> desc(count);
        std::vector<Tile> tiles;
        std::vector<int> tile_first(count + 1, 0);
        long long total = 0;
        for (int i = 0; i < count; ++i) {
            BuildDesc& ds = desc[i];
            memset(&ds, 0, sizeof(ds));
            ds.points = pdev[i];
            ds.labels = static_cast<const unsigned int*>(ldev[i]);
            ds.n = n[i];
            ds.d = d[i];
            ds.p = row_floats(d[i]);
            ds.off = total;
            total += n[i];
            tile_first[i] = (int)tiles.size();
            for (long long f = 0; f < n[i]; f += kTilePoints)
                tiles.push_back(Tile{i, (int)std::min<long long>(kTilePoints, n[i] - f), f});
        }
        tile_first[count] = (int)tiles.size();
        if (total >= (1ll << 31)) {
            set_error("knn_batch_build: more than 2^31 - 1 points in the batch");
            return bail(KNN_EINVAL);
        }
        BuildDesc* ddesc = nullptr;
        Tile* dtiles = nullptr;
        int* dtile_first = nullptr;
        float* dwidth = nullptr;
        float* partial = nullptr;
        BoxOut* dbox = nullptr;
        std::vector<float> wv(width, width + count);
        {
            // one copy for the tiles, their first entries and the widths
            std::vector<char> blob;
            auto put = [&blob](const void* p, size_t bytes) {
                const size_t at = (blob.size() + 255) & ~(size_t)255;
                blob.resize(at + bytes);
                memcpy(blob.data() + at, p, bytes);
                return at;
            };
            const size_t o_tiles = put(tiles.data(), tiles.size() * sizeof(Tile));
            const size_t o_first = put(tile_first.data(), tile_first.size() * sizeof(int));
            const size_t o_width = put(wv.data(), wv.size() * sizeof(float));
            char* dblob = nullptr;
            if ((st = upload(sc, blob, &dblob, "batch tiles")) != KNN_OK) return bail(st);
            dtiles = reinterpret_cast<Tile*>(dblob + o_tiles);
            dtile_first = reinterpret_cast<int*>(dblob + o_first);
            dwidth = reinterpret_cast<float*>(dblob + o_width);
        }
        if ((st = upload(sc, desc, &ddesc, "batch descriptors")) != KNN_OK) return bail(st);
        if ((st = sc.alloc(&partial, tiles.size() * kPartStride, "batch partial boxes")) != KNN_OK)
            return bail(st);
        if ((st = sc.alloc(&dbox, (size_t)count, "batch boxes")) != KNN_OK) return bail(st);
        // ---- every box, then the one host read of the build ----
        batch_box_partial_kernel<<<(unsigned)tiles.size(), kBoxThreads, 0, s>>>(ddesc, dtiles,
                                                                                partial);
        batch_box_final_kernel<<<count, kBoxThreads, 0, s>>>(ddesc, dtile_first, partial, dwidth,
                                                             dbox);
        count_launches(2);
        std::vector<BoxOut> box(count);
        e = cudaMemcpyAsync(box.data(), dbox, sizeof(BoxOut) * count, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bail(cuda_error(e, "batch boxes"));
        phase_mark("box", s);
        // the side stream may start the label copies from here on; they are
        // issued once the sort is launched, so that the GPU has work while
        // the host issues them
        const bool lab_side = !late_labels.empty() && lab_copies.begin(dev);

        // ---- layouts ----
        int shift = 0;
        long long rows_total = 0, dense_total = 0, bitmap_total = 0;
        bool any_hash = false, any_labels = false;
        std::vector<long long> dense_seg;
            b->info.resize(count);
        for (int i = 0; i < count; ++i) {
            BuildDesc& ds = desc[i];
            char msg[160];
            if (box[i].flags & kStatusNonFinite) {
                snprintf(msg, sizeof(msg), "knn_batch_build: index %d has a non-finite coordinate", i);
                set_error(msg);
                return bail(KNN_EINVAL);
            }
            if (box[i].flags & kStatusExtent) {
                snprintf(msg, sizeof(msg),
                         "knn_batch_build: index %d has more than 2^31 - 1 cells along one dimension", i);
                set_error(msg);
                return bail(KNN_EINVAL);
            }
            GridConst& g = ds.g;
            memset(&g, 0, sizeof(g));
            for (int j = 0; j < kMaxD; ++j) {
                g.w[j] = width[i];
                g.inv_w[j] = 1.0f / width[i];
            }
            g.d = d[i];
            unsigned long long space = 1ull;
            bool overflow = false;
            for (int j = 0; j < d[i]; ++j) {
                g.lo[j] = box[i].lo[j];
                g.cmax[j] = box[i].ext[j] - 1;
                const unsigned long long ext = (unsigned long long)box[i].ext[j];
                if (space > 0x7fffffffffffffffull / ext) overflow = true;
                space *= ext;
            }
            unsigned long long stride = 1ull;
            for (int j = d[i] - 1; j >= 0; --j) {
                g.stride[j] = stride;
                stride *= (unsigned long long)box[i].ext[j];
            }
            int bits = 0;
            while (bits < 64 && (1ull << bits) < space) ++bits;
            if (overflow) bits = 64;
            shift = std::max(shift, bits);
            int kind = table ? table[i] : KNN_TABLE_AUTO;
            if (kind == KNN_TABLE_AUTO)
                kind = space <= 4ull * (unsigned long long)n[i] + 1024ull ? KNN_TABLE_DENSE
                                                                          : KNN_TABLE_HASH;
            if (kind == KNN_TABLE_DENSE && (overflow || space + 1ull > 0x7fffffffull)) {
                snprintf(msg, sizeof(msg),
                         "knn_batch_build: the dense table of index %d is too large", i);
                set_error(msg);
                return bail(KNN_EINVAL);
            }
            // rows are read as 8/16-byte vectors: start each index on 16 bytes
            rows_total = (rows_total + 3) & ~3ll;
            ds.rows_off = rows_total;
            rows_total += n[i] * ds.p;
            ds.dense_off = -1;
            ds.bitmap_off = -1;
            if (kind == KNN_TABLE_DENSE) {
                ds.dense_off = dense_total;
                dense_seg.push_back(dense_total);
                dense_total += (long long)space + 1;
            } else {
                any_hash = true;
                if (!overflow && space <= (1ull << 33) && space / 8ull <= 64ull * (unsigned long long)n[i]) {
                    ds.bitmap_off = bitmap_total;
                    bitmap_total += (long long)((space + 31ull) / 32ull);
                }
            }
            any_labels |= ds.labels != nullptr;
            knn_index_info_t& inf = b->info[i];
            memset(&inf, 0, sizeof(inf));
            inf.n = n[i];
            inf.d = d[i];
            inf.table = kind;
            inf.cell_width = width[i];
            for (int j = 0; j < d[i]; ++j) {
                inf.origin[j] = g.lo[j];
                inf.extent[j] = box[i].ext[j];
            }
            inf.table_slots = kind == KNN_TABLE_DENSE ? (long long)space + 1 : 0;
            inf.row_floats = ds.p;
            inf.has_labels = ds.labels != nullptr;
        }
        int ib = 0;
        while ((1 << ib) < count) ++ib;
        if (shift + ib > 63) {
            set_error("knn_batch_build: the cell ids of the batch need more than 63 bits "
                      "(a grid too fine for a batch of this size)");
            return bail(KNN_EINVAL);
        }
        if ((st = upload(sc, desc, &ddesc, "batch descriptors")) != KNN_OK) return bail(st);

        // ---- keys, sort, cells ----
        unsigned long long *ka, *kb, *sk;
        unsigned int *va, *vb, *sv, *cell_start;
        unsigned long long* cell_key;
        void *rtmp, *stmp;
        const long long scan_n = std::max(total, dense_total);
        if ((st = sc.alloc(&ka, total, "batch keys")) != KNN_OK ||
            (st = sc.alloc(&kb, total, "batch keys")) != KNN_OK ||
            (st = sc.alloc(&va, total, "batch rows")) != KNN_OK ||
            (st = sc.alloc(&vb, total, "batch rows")) != KNN_OK ||
            (st = sc.alloc(reinterpret_cast<char**>(&rtmp), radix_temp_bytes(total), "batch sort")) != KNN_OK ||
            (st = sc.alloc(reinterpret_cast<char**>(&stmp), scan_temp_bytes(scan_n), "batch scan")) != KNN_OK ||
            (st = sc.alloc(&cell_key, total, "batch cell keys")) != KNN_OK ||
            (st = sc.alloc(&cell_start, total + 1, "batch cell starts")) != KNN_OK)
            return bail(st);
        void* gv = nullptr;
        if ((st = device_alloc(&gv, sizeof(GridDev), s, "batch grid")) != KNN_OK) return bail(st);
        b->gdev = static_cast<GridDev*>(gv);
        batch_keys_kernel<<<(unsigned)tiles.size(), 256, 0, s>>>(ddesc, dtiles, shift, ka, va);
        count_launches(1);
        phase_mark("keys", s);
        e = radix_sort_pairs(ka, va, kb, vb, total, shift + ib, rtmp, &sk, &sv, s);
        for (size_t c = 0; e == cudaSuccess && c < late_labels.size(); ++c) {
            const LateCopy& lc = late_labels[c];
            e = lab_side ? lab_copies.copy(lc.dst, lc.src, lc.bytes)
                         : cudaMemcpyAsync(lc.dst, lc.src, lc.bytes, cudaMemcpyHostToDevice, s);
        }
        phase_mark("sort", s);
        if (e == cudaSuccess)
            e = launch_cells(sk, total, stmp, cell_key, cell_start, b->gdev, s);
        if (e != cudaSuccess) return bail(cuda_error(e, "batch sort and staged labels"));
        phase_mark("cells", s);

        // ---- tables ----
        if (dense_total > 0) {
            if ((st = device_alloc(&gv, sizeof(unsigned int) * dense_total, s, "batch dense tables")) != KNN_OK)
                return bail(st);
            b->dense = static_cast<unsigned int*>(gv);
            e = cudaMemsetAsync(b->dense, 0, sizeof(unsigned int) * dense_total, s);
            batch_dense_counts_kernel<<<grid_blocks(total), 256, 0, s>>>(ddesc, shift, cell_key,
                                                                         cell_start, b->gdev, b->dense);
            count_launches(1);
            if (e == cudaSuccess) e = scan_exclusive(b->dense, b->dense, dense_total, stmp, s);
            long long* dseg = nullptr;
            unsigned int* sbase = nullptr;
            if ((st = upload(sc, dense_seg, &dseg, "batch dense segments")) != KNN_OK)
                return bail(st);
            if ((st = sc.alloc(&sbase, dense_seg.size(), "batch dense bases")) != KNN_OK)
                return bail(st);
            const int nseg = (int)dense_seg.size();
            batch_seg_base_kernel<<<(nseg + 255) / 256, 256, 0, s>>>(dseg, nseg, b->dense, sbase);
            batch_dense_fixup_kernel<<<grid_blocks(dense_total), 256, 0, s>>>(
                dseg, nseg, sbase, dense_total, b->dense);
            count_launches(2);
        }
        if (any_hash) {
            unsigned long long cap = 16ull;
            while (cap < 2ull * (unsigned long long)total) cap <<= 1;
            if ((st = device_alloc(&gv, sizeof(HashSlot) * cap, s, "batch hash table")) != KNN_OK)
                return bail(st);
            b->slots = static_cast<HashSlot*>(gv);
            if (bitmap_total > 0) {
                if ((st = device_alloc(&gv, sizeof(unsigned int) * bitmap_total, s, "batch bitmaps")) != KNN_OK)
                    return bail(st);
                b->bitmap = static_cast<unsigned int*>(gv);
                if (e == cudaSuccess)
                    e = cudaMemsetAsync(b->bitmap, 0, sizeof(unsigned int) * bitmap_total, s);
            }
            // the shared table's capacity comes from all cells (an upper bound)
            if (e == cudaSuccess) e = launch_hash_clear(b->slots, b->gdev, cap, s);
            batch_hash_insert_kernel<<<grid_blocks(total), 256, 0, s>>>(ddesc, shift, cell_key,
                                                                        cell_start, b->gdev,
                                                                        b->slots, b->bitmap);
            count_launches(1);
        }
        if (e != cudaSuccess) return bail(cuda_error(e, "batch tables"));
        phase_mark("table", s);

        // ---- rows, row ids, labels ----
        if ((st = device_alloc(&gv, sizeof(float) * rows_total, s, "batch rows")) != KNN_OK) return bail(st);
        b->rows = static_cast<float*>(gv);
        b->rid = sv;  // the sorted values become the rows' training indices
        // keep the sorted buffer: take it out of the scratch list
        sc.ptrs.erase(std::remove(sc.ptrs.begin(), sc.ptrs.end(), (void*)sv), sc.ptrs.end());
        if (any_labels) {
            if ((st = device_alloc(&gv, sizeof(unsigned int) * total, s, "batch labels")) != KNN_OK)
                return bail(st);
            b->labels = static_cast<unsigned int*>(gv);
        }
        std::vector<GatherDesc> gdesc(count);
        for (int i = 0; i < count; ++i)
            gdesc[i] = GatherDesc{desc[i].points, desc[i].off, desc[i].rows_off, desc[i].d, desc[i].p};
        GatherDesc* dgd = nullptr;
        if ((st = upload(sc, gdesc, &dgd, "batch gather descriptors")) != KNN_OK) return bail(st);
        batch_gather_kernel<<<grid_blocks(total), 256, 0, s>>>(dgd, shift, total, sk, sv, b->rows,
                                                               b->rid);
        count_launches(1);
        if (any_labels) {
            e = lab_copies.end();
            if (e != cudaSuccess) return bail(cuda_error(e, "batch staged labels"));
            batch_labels_kernel<<<(unsigned)tiles.size(), 256, 0, s>>>(ddesc, dtiles, b->labels);
            count_launches(1);
            e = lab_copies.wait_host();  // pinned labels may be reused after the call
            if (e != cudaSuccess) return bail(cuda_error(e, "batch staged labels"));
        }
        e = cudaGetLastError();
        phase_mark("gather", s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->last_use, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(b->last_use, s);
        if (e != cudaSuccess) return bail(cuda_error(e, "batch gather"));

        // ---- each index's part of its query arguments ----
        b->proto.resize(count);
        for (int i = 0; i < count; ++i) {
            QueryArgs& a = b->proto[i];
            memset(&a, 0, sizeof(a));
            const BuildDesc& ds = desc[i];
            a.g = ds.g;
            a.rows = b->rows + ds.rows_off;
            a.rid = b->rid + ds.off;
            a.labels = ds.labels && b->labels ? b->labels + ds.off : nullptr;
            a.dense = ds.dense_off >= 0;
            a.dstart = a.dense ? b->dense + ds.dense_off : nullptr;
            a.slots = a.dense ? nullptr : b->slots;
            a.bitmap = ds.bitmap_off >= 0 ? b->bitmap + ds.bitmap_off : nullptr;
            a.key_prefix = (unsigned long long)i << shift;
            a.gdev = b->gdev;
            a.max_layers = max_layers_default();
            a.max_rows = max_rows_default();
            a.heavy_rows = heavy_rows_default(ds.d);
            a.heavy_cands = heavy_cands_default();
        }
    }
    *out = b;
    return KNN_OK;
}

// The query arguments of a batch call, grouped by dimension.
struct Layout {
    std::vector<QueryArgs> args;              // all groups, group after group
    std::vector<unsigned long long> qoff;     // each group's count + 1 offsets
    std::vector<int> group_first;             // first args entry of each group
    std::vector<int> group_qoff;              // first qoff entry of each group
    std::vector<int> group_count;
    std::vector<int> group_d;
    std::vector<int> group_ns;     // 1: k <= 32, 2: k > 32
    std::vector<int> group_dense;  // dense tables
    std::vector<unsigned long long> group_total;
};

knn_status plan_layout(const ghn_batch* b, const float* const* queries, const int64_t* m,
                       const int32_t* k, const int32_t* mode, int32_t* const* ids,
                       float* const* dist2, void* const* pred, Layout& lay,
                       bool require_device = true)
{
    for (int i = 0; i < b->count; ++i) {
        char msg[160];
        if (m[i] < 0 || m[i] >= (1ll << 31) || k[i] < 1 || k[i] > kMaxK || mode[i] < -1 ||
            mode[i] > 2) {
            snprintf(msg, sizeof(msg), "knn_batch_query: index %d: bad m, k or mode", i);
            set_error(msg);
            return KNN_EINVAL;
        }
        if (mode[i] >= 0 && !b->proto[i].labels) {
            snprintf(msg, sizeof(msg), "knn_batch_query: index %d has no labels for a prediction", i);
            set_error(msg);
            return KNN_EINVAL;
        }
        if (m[i] > 0 && (!queries[i] || !ids[i] || (mode[i] >= 0 && (!pred || !pred[i])))) {
            snprintf(msg, sizeof(msg), "knn_batch_query: index %d: NULL queries or outputs", i);
            set_error(msg);
            return KNN_EINVAL;
        }
        if (require_device && m[i] > 0 &&
            (!is_device(queries[i]) || !is_device(ids[i]) ||
             (dist2 && dist2[i] && !is_device(dist2[i])) ||
             (mode[i] >= 0 && (!pred || !is_device(pred[i]))))) {
            snprintf(msg, sizeof(msg),
                     "knn_batch_query: index %d: queries and outputs must be device memory of the batch's GPU", i);
            set_error(msg);
            return KNN_EINVAL;
        }
    }
    // the deferred-query list holds 32-bit positions within a group
    unsigned long long all = 0ull;
    for (int i = 0; i < b->count; ++i) all += (unsigned long long)m[i];
    if (all >= (1ull << 32)) {
        set_error("knn_batch_query: more than 2^32 - 1 queries in one call");
        return KNN_EINVAL;
    }
    // one group per (dimension, buffer width, table kind): each launches a
    // kernel specialised for all three
    for (int key = 0; key < 4 * (kMaxD + 1); ++key) {
        const int dim = key / 4, ns = (key & 2) ? 2 : 1, dense = key & 1;
        std::vector<int> members;
        for (int i = 0; i < b->count; ++i)
            if (b->info[i].d == dim && m[i] > 0 && (k[i] > 32 ? 2 : 1) == ns &&
                (b->proto[i].dense ? 1 : 0) == dense)
                members.push_back(i);
        if (members.empty()) continue;
        lay.group_first.push_back((int)lay.args.size());
        lay.group_qoff.push_back((int)lay.qoff.size());
        lay.group_count.push_back((int)members.size());
        lay.group_d.push_back(dim);
        lay.group_ns.push_back(ns);
        lay.group_dense.push_back(dense);
        unsigned long long acc = 0ull;
        for (int i : members) {
            QueryArgs a = b->proto[i];
            a.q = queries[i];
            a.m = m[i];
            a.k = k[i];
            a.mode = mode[i];
            a.ids = ids[i];
            a.dist2 = dist2 ? dist2[i] : nullptr;
            a.pred = mode[i] >= 0 ? pred[i] : nullptr;
            lay.args.push_back(a);
            lay.qoff.push_back(acc);
            acc += (unsigned long long)m[i];
        }
        lay.qoff.push_back(acc);
        lay.group_total.push_back(acc);
    }
    return KNN_OK;
}

// Device image of a layout: arguments, offsets, counters, status, deferred lists.
knn_status make_plan(const ghn_batch* b, Layout& lay, cudaStream_t s, ghn_plan* p)
{
    const size_t ng = lay.group_d.size();
    unsigned long long heavy_total = 0ull;
    for (unsigned long long t : lay.group_total) heavy_total += t;
    const size_t args_bytes = (lay.args.size() * sizeof(QueryArgs) + 255) & ~(size_t)255;
    const size_t qoff_bytes = (lay.qoff.size() * 8 + 255) & ~(size_t)255;
    p->counter_bytes = (ng * 4 + 4) * sizeof(unsigned long long);
    const size_t heavy_bytes = heavy_total * sizeof(unsigned int);
    const size_t bytes = args_bytes + qoff_bytes + p->counter_bytes + heavy_bytes + 16;
    knn_status st = device_alloc(&p->dev_buf, bytes, s, "batch query plan");
    if (st != KNN_OK) return st;
    char* base = static_cast<char*>(p->dev_buf);
    QueryArgs* dargs = reinterpret_cast<QueryArgs*>(base);
    unsigned long long* dqoff = reinterpret_cast<unsigned long long*>(base + args_bytes);
    p->counters = reinterpret_cast<unsigned long long*>(base + args_bytes + qoff_bytes);
    unsigned int* heavy =
        reinterpret_cast<unsigned int*>(base + args_bytes + qoff_bytes + p->counter_bytes);
    // group g: counter at counters[2g], heavy count / cursor in counters[2g + 1];
    // the shared status word after the groups' counters
    p->status = reinterpret_cast<unsigned int*>(p->counters + 2 * ng);
    for (QueryArgs& a : lay.args) a.status = p->status;
    // pageable sources: each copy returns once its source is staged (no wait)
    cudaError_t e = cudaMemcpyAsync(dargs, lay.args.data(), lay.args.size() * sizeof(QueryArgs),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dqoff, lay.qoff.data(), lay.qoff.size() * 8, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "batch query arguments");
    unsigned long long hoff = 0ull;
    for (size_t g = 0; g < ng; ++g) {
        BatchArgs ba;
        memset(&ba, 0, sizeof(ba));
        ba.args = dargs + lay.group_first[g];
        ba.qoff = dqoff + lay.group_qoff[g];
        ba.count = lay.group_count[g];
        ba.d = lay.group_d[g];
        ba.total = lay.group_total[g];
        ba.counter = p->counters + 2 * g;
        ba.heavy_count = reinterpret_cast<unsigned int*>(p->counters + 2 * g + 1);
        ba.heavy_cursor = ba.heavy_count + 1;
        ba.heavy_list = heavy + hoff;
        ba.exact = lay.args[lay.group_first[g]].exact;  // one rule for the whole call
        ba.ns = lay.group_ns[g];
        ba.dense = lay.group_dense[g];
        hoff += lay.group_total[g];
        p->groups.push_back(ba);
    }
    p->batch = b;
    return KNN_OK;
}

// The launches of one batch query: clear the counters, then each group
// (each kernel marked for the phase timer when `timed`; never inside a capture).
cudaError_t launch_plan(const ghn_plan* p, cudaStream_t s, bool timed = false)
{
    cudaError_t e = cudaMemsetAsync(p->counters, 0, p->counter_bytes, s);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    set_kernel_marks(timed);
    for (size_t g = 0; e == cudaSuccess && g < p->groups.size(); ++g)
        e = launch_batch_query(p->groups[g], sms, s);
    set_kernel_marks(false);
    return e;
}

void free_plan(ghn_plan* p)
{
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->dev_buf) {
        cudaDeviceSynchronize();
        device_free(p->dev_buf, 0);
        cudaDeviceSynchronize();
    }
    delete p;
}

knn_status read_status(const ghn_plan* p, cudaStream_t s)
{
    unsigned int st = 0u;
    cudaError_t e = cudaMemcpyAsync(&st, p->status, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "batch status");
    if (st & kStatusNonFinite) return fail("knn_batch_query: a query coordinate is not finite", KNN_EINVAL);
    if (st & kStatusLimit) return fail("knn_batch_query: a query reached its work bound (rows or layer cap)", KNN_ELIMIT);
    return KNN_OK;
}

}  // namespace

extern "C" {

knn_status knn_batch_build(int32_t count, const float* const* points, const void* const* labels,
                           const int64_t* n, const int32_t* d, const float* cell_width,
                           const int32_t* table, void* stream, ghn_batch** out)
{
    if (!out) return fail("knn_batch_build: out is NULL", KNN_EINVAL);
    *out = nullptr;
    if (count < 1 || count > 65536 || !points || !n || !d || !cell_width)
        return fail("knn_batch_build: count must be in [1, 65536] and the arrays not NULL",
                    KNN_EINVAL);
    for (int i = 0; i < count; ++i) {
        char msg[160];
        if (n[i] < 1 || n[i] >= (1ll << 31) || d[i] < 1 || d[i] > kMaxD ||
            !(cell_width[i] > 0.0f) || !isfinite(cell_width[i]) ||
            (table && (table[i] < KNN_TABLE_AUTO || table[i] > KNN_TABLE_HASH))) {
            snprintf(msg, sizeof(msg), "knn_batch_build: index %d: bad n, d, width or table", i);
            return fail(msg, KNN_EINVAL);
        }
        if (!points[i] || pointer_kind(points[i], nullptr) == kOtherGpu ||
            (labels && labels[i] && pointer_kind(labels[i], nullptr) == kOtherGpu)) {
            snprintf(msg, sizeof(msg),
                     "knn_batch_build: index %d: points are NULL or on another GPU than the current one", i);
            return fail(msg, KNN_EINVAL);
        }
    }
    return batch_build_impl(count, points, labels, n, d, cell_width, table,
                            static_cast<cudaStream_t>(stream), out);
}

knn_status knn_batch_info(const ghn_batch* batch, int32_t i, knn_index_info_t* info)
{
    if (!batch || !info || i < 0 || i >= batch->count)
        return fail("knn_batch_info: bad argument", KNN_EINVAL);
    *info = batch->info[i];
    return KNN_OK;
}

knn_status knn_batch_query(const ghn_batch* batch, const float* const* queries, const int64_t* m,
                           const int32_t* k, const int32_t* mode, int32_t* const* ids,
                           float* const* dist2, void* const* pred, int32_t flags, void* stream)
{
    if (!batch || !queries || !m || !k || !mode || !ids)
        return fail("knn_batch_query: NULL argument", KNN_EINVAL);
    if (flags & ~(KNN_QUERY_CHECKED | KNN_QUERY_EXACT))
        return fail("knn_batch_query: only KNN_QUERY_CHECKED and KNN_QUERY_EXACT are supported",
                    KNN_EINVAL);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != batch->device) cudaSetDevice(batch->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int count = batch->count;
    phase_begin(s);
    // Host buffers.  Queries in host memory are copied into one device
    // buffer.  Outputs in pinned host memory that the GPU addresses are
    // written by the kernels directly; other host outputs get device space
    // and are copied out after the kernels.  Host outputs are complete when
    // the call returns.
    std::vector<const float*> qd(count, nullptr);
    std::vector<int32_t*> idd(count, nullptr);
    std::vector<float*> d2d(count, nullptr);
    std::vector<void*> pd(count, nullptr);
    struct Copy {
        void* dst;
        const void* src;
        size_t bytes;
    };
    std::vector<Copy> out_copies;
    void* stage = nullptr;
    SideCopies q_copies(s);
    cudaEvent_t q_read = nullptr;  // pinned queries copied on `s` have been read
    bool host_out = false;
    knn_status st = KNN_OK;
    {
        const size_t none = ~(size_t)0;
        std::vector<size_t> q_at(count, none), i_at(count, none), d_at(count, none),
            p_at(count, none);
        size_t words = 0;
        auto take = [&words](size_t count_words) {
            words = (words + 3) & ~(size_t)3;
            const size_t at = words;
            words += count_words;
            return at;
        };
        bool any_q = false, all_q_pinned = true, any_q_pinned = false;
        for (int i = 0; i < count && st == KNN_OK; ++i) {
            if (m[i] <= 0) continue;
            if (m[i] >= (1ll << 31) || k[i] < 1 || k[i] > kMaxK) break;  // plan_layout reports it
            const size_t mi = (size_t)m[i], ki = (size_t)k[i];
            const size_t di = (size_t)batch->info[i].d;
            void* dp = nullptr;
            int kind = pointer_kind(queries[i], &dp);
            if (kind == kOtherGpu) st = fail("knn_batch_query: a buffer is device memory of another GPU", KNN_EINVAL);
            qd[i] = queries[i];
            if (kind == kHostMem || kind == kMappedHost) q_at[i] = take(mi * di);
            any_q |= kind == kHostMem || kind == kMappedHost;
            all_q_pinned &= kind != kHostMem;
            any_q_pinned |= kind == kMappedHost;
            kind = pointer_kind(ids[i], &dp);
            if (kind == kOtherGpu) st = fail("knn_batch_query: a buffer is device memory of another GPU", KNN_EINVAL);
            idd[i] = kind == kMappedHost ? static_cast<int32_t*>(dp) : ids[i];
            if (kind == kHostMem) i_at[i] = take(mi * ki);
            host_out |= kind == kHostMem || kind == kMappedHost;
            if (dist2 && dist2[i]) {
                kind = pointer_kind(dist2[i], &dp);
                if (kind == kOtherGpu) st = fail("knn_batch_query: a buffer is device memory of another GPU", KNN_EINVAL);
                d2d[i] = kind == kMappedHost ? static_cast<float*>(dp) : dist2[i];
                if (kind == kHostMem) d_at[i] = take(mi * ki);
                host_out |= kind == kHostMem || kind == kMappedHost;
            }
            if (pred && pred[i] && mode[i] >= 0) {
                kind = pointer_kind(pred[i], &dp);
                if (kind == kOtherGpu) st = fail("knn_batch_query: a buffer is device memory of another GPU", KNN_EINVAL);
                pd[i] = kind == kMappedHost ? dp : pred[i];
                if (kind == kHostMem) p_at[i] = take(mi);
                host_out |= kind == kHostMem || kind == kMappedHost;
            }
        }
        // pinned host queries go over on the side stream, with the staging
        // buffer allocated there, so that the copies overlap work still
        // queued on the caller's stream (a build just launched); the kernels
        // wait for them
        const bool side = st == KNN_OK && words > 0 && any_q && all_q_pinned &&
                          q_copies.open(batch->device);
        if (st == KNN_OK && words > 0)
            st = device_alloc(&stage, words * 4, side ? q_copies.side : s, "batch query staging");
        cudaError_t e = cudaSuccess;
        float* sw = static_cast<float*>(stage);
        for (int i = 0; st == KNN_OK && i < count; ++i) {
            if (m[i] <= 0) continue;
            const size_t mi = (size_t)m[i], ki = (size_t)k[i];
            const size_t di = (size_t)batch->info[i].d;
            if (q_at[i] != none) {
                if (e == cudaSuccess)
                    e = side ? q_copies.copy(sw + q_at[i], queries[i], mi * di * 4)
                             : cudaMemcpyAsync(sw + q_at[i], queries[i], mi * di * 4,
                                               cudaMemcpyHostToDevice, s);
                qd[i] = sw + q_at[i];
            }
            if (i_at[i] != none) {
                idd[i] = reinterpret_cast<int32_t*>(sw + i_at[i]);
                out_copies.push_back(Copy{ids[i], idd[i], mi * ki * 4});
            }
            if (d_at[i] != none) {
                d2d[i] = sw + d_at[i];
                out_copies.push_back(Copy{dist2[i], d2d[i], mi * ki * 4});
            }
            if (p_at[i] != none) {
                pd[i] = sw + p_at[i];
                out_copies.push_back(Copy{pred[i], pd[i], mi * 4});
            }
        }
        const cudaError_t ee = q_copies.end();  // the kernels wait for the copies
        if (e == cudaSuccess) e = ee;
        // pinned queries copied on the caller's stream: an event, so that the
        // call can return once they have been read
        if (st == KNN_OK && e == cudaSuccess && !side && any_q_pinned &&
            cudaEventCreateWithFlags(&q_read, cudaEventDisableTiming) == cudaSuccess)
            e = cudaEventRecord(q_read, s);
        if (st == KNN_OK && e != cudaSuccess) st = cuda_error(e, "knn_batch_query: staging");
    }
    phase_mark("stage", s);
    Layout lay;
    if (st == KNN_OK)
        st = plan_layout(batch, qd.data(), m, k, mode, idd.data(), dist2 ? d2d.data() : nullptr,
                         pred ? pd.data() : nullptr, lay, false);
    for (QueryArgs& a : lay.args) a.exact = (flags & KNN_QUERY_EXACT) ? 1 : 0;
    ghn_plan p;
    p.device = batch->device;
    if (st == KNN_OK && !lay.args.empty()) {
        st = make_plan(batch, lay, s, &p);
        if (st == KNN_OK) {
            cudaError_t e = launch_plan(&p, s, true);
            for (size_t c = 0; e == cudaSuccess && c < out_copies.size(); ++c)
                e = cudaMemcpyAsync(out_copies[c].dst, out_copies[c].src, out_copies[c].bytes,
                                    cudaMemcpyDeviceToHost, s);
            if (!out_copies.empty()) phase_mark("copy", s);
            if (e == cudaSuccess) e = cudaEventRecord(batch->last_use, s);
            if (e != cudaSuccess) st = cuda_error(e, "knn_batch_query");
            if (st == KNN_OK && (flags & KNN_QUERY_CHECKED)) st = read_status(&p, s);
        }
        if (p.dev_buf) device_free(p.dev_buf, s);
        p.dev_buf = nullptr;
    }
    {
        // pinned queries may be reused after the call
        cudaError_t e = q_copies.wait_host();
        if (q_read) {
            const cudaError_t e2 = cudaEventSynchronize(q_read);
            if (e == cudaSuccess) e = e2;
            cudaEventDestroy(q_read);
        }
        if (st == KNN_OK && e != cudaSuccess) st = cuda_error(e, "knn_batch_query: staging");
    }
    if (stage) device_free(stage, s);
    if (host_out) {
        const cudaError_t e = cudaStreamSynchronize(s);
        if (st == KNN_OK && e != cudaSuccess) st = cuda_error(e, "knn_batch_query: synchronize");
    }
    if (prev >= 0 && prev != batch->device) cudaSetDevice(prev);
    return st;
}

knn_status knn_batch_plan(const ghn_batch* batch, const float* const* queries, const int64_t* m,
                          const int32_t* k, const int32_t* mode, int32_t* const* ids,
                          float* const* dist2, void* const* pred, ghn_plan** out)
{
    if (!out) return fail("knn_batch_plan: out is NULL", KNN_EINVAL);
    *out = nullptr;
    if (!batch || !queries || !m || !k || !mode || !ids)
        return fail("knn_batch_plan: NULL argument", KNN_EINVAL);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != batch->device) cudaSetDevice(batch->device);
    Layout lay;
    knn_status st = plan_layout(batch, queries, m, k, mode, ids, dist2, pred, lay);
    ghn_plan* p = new ghn_plan();
    p->device = batch->device;
    cudaStream_t cs = nullptr;
    if (st == KNN_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) st = cuda_error(e, "knn_batch_plan: stream");
    }
    if (st == KNN_OK) st = make_plan(batch, lay, cs, p);
    if (st == KNN_OK) {
        // the arguments must be on the device before any replay, which may
        // run on another stream
        const cudaError_t e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) st = cuda_error(e, "knn_batch_plan: arguments");
    }
    if (st == KNN_OK) {
        // capture the launches once; knn_batch_run replays them
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t le = launch_plan(p, cs);
            e = cudaStreamEndCapture(cs, &p->graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
        if (e != cudaSuccess) st = cuda_error(e, "knn_batch_plan: graph capture");
    }
    if (cs) cudaStreamDestroy(cs);
    if (prev >= 0 && prev != batch->device) cudaSetDevice(prev);
    if (st != KNN_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return KNN_OK;
}

knn_status knn_batch_run(ghn_plan* plan, int32_t flags, void* stream)
{
    if (!plan) return fail("knn_batch_run: plan is NULL", KNN_EINVAL);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != plan->device) cudaSetDevice(plan->device);
    knn_status st = KNN_OK;
    cudaError_t e = plan->exec ? cudaGraphLaunch(plan->exec, s) : cudaSuccess;
    if (e == cudaSuccess) e = cudaEventRecord(plan->batch->last_use, s);
    if (e != cudaSuccess) st = cuda_error(e, "knn_batch_run");
    if (st == KNN_OK && (flags & KNN_QUERY_CHECKED) && plan->exec) st = read_status(plan, s);
    if (prev >= 0 && prev != plan->device) cudaSetDevice(prev);
    return st;
}

void knn_plan_free(ghn_plan* plan) { free_plan(plan); }

knn_status knn_batch_set_deferral(ghn_batch* batch, int32_t i, int64_t heavy_rows,
                                  int64_t heavy_cands)
{
    if (!batch || i < 0 || i >= batch->count)
        return fail("knn_batch_set_deferral: bad argument", KNN_EINVAL);
    QueryArgs& a = batch->proto[i];
    a.heavy_rows = deferral_threshold(heavy_rows, heavy_rows_default(a.g.d));
    a.heavy_cands = deferral_threshold(heavy_cands, heavy_cands_default());
    return KNN_OK;
}

void knn_batch_free(ghn_batch* batch) { free_batch(batch); }

}  // extern "C"
