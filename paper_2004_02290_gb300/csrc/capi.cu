// C ABI of the GB300 grid-hashing KNN library: argument checks, device memory,
// host staging and the order of the build and query kernels on the caller's
// stream.  The entry points are declared, with their contracts, in
// include/ghn_knn.h.

#include "build_launch.cuh"
#include "ghn_internal.cuh"
#include "../../include/ghn_knn.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>

using namespace ghn;

struct ghn_index {
    int device = 0;
    long long n = 0;
    int d = 0;
    Widths wd{};  // cell measurement and split count of each dimension
    int table = KNN_TABLE_DENSE;
    GridConst g{};
    unsigned long long ncell_space = 0;  // cells in the box (prod of extents)
    int key_bits = 0;
    float* rows = nullptr;           // n * row_floats(d), cell order
    unsigned int* rid = nullptr;     // n training indices, cell order
    unsigned int* labels = nullptr;  // n outputs, training order (or null)
    unsigned int* dstart = nullptr;  // dense table
    HashSlot* slots = nullptr;       // hash table
    unsigned long long max_slots = 0;
    unsigned int* bitmap = nullptr;  // hash: occupancy bit per cell of the box, or null
    GridDev* gdev = nullptr;
    cudaEvent_t last_use = nullptr;
    // deferral to the cooperative kernel (knn_index_set_deferral): 0 = the
    // library's default, < 0 = never, > 0 = the threshold
    long long defer_rows = 0;
    long long defer_cands = 0;
    // filled on first inspection
    bool info_ready = false;
    GridDev host_gdev{};
};

namespace {

// Bits of the cell id that the locality order of the queries sorts by (the
// top ones): two 8-bit radix passes.
constexpr int kOrderBits = 16;

thread_local char g_err[512] = "";

void set_err(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

knn_status cuda_fail(cudaError_t e, const char* what)
{
    set_err("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? KNN_ENOMEM : KNN_ECUDA;
}

#define GHN_CHECK(call, what)                          \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ---- allocation (stream-ordered pool), with a host-side failure injector ----

std::atomic<long long> g_alloc_count{0};

long long fail_alloc_at()
{
    static long long v = [] {
        const char* s = getenv("GHN_FAIL_ALLOC_AT");
        return s ? atoll(s) : 0ll;
    }();
    return v;
}

// Deferral thresholds of the warp kernel (see query_kernel.cuh); a query
// with a layer of more rows, or a row batch of more candidates, goes to the
// cooperative kernel.  GHN_HEAVY_ROWS / GHN_HEAVY_CANDS override them.
unsigned int env_uint(const char* name, unsigned int dflt)
{
    const char* s = getenv(name);
    if (!s || !*s) return dflt;
    const long long v = atoll(s);
    return v <= 0 ? 0xffffffffu : (unsigned int)(v > 0xffffffffll ? 0xffffffffll : v);
}

// Defaults measured on GB300: a layer of more than 1024 rows (d <= 4) or 4096
// rows (d >= 5), or a row batch of more than 8192 candidates.
unsigned int heavy_rows_env(int d)
{
    static unsigned int v = env_uint("GHN_HEAVY_ROWS", 0u);  // 0: unset
    if (v != 0u) return v;  // a value, or all ones (no deferral) for a value <= 0
    return d <= 4 ? 1024u : 4096u;
}

// A deferral threshold as the kernels take it: the default, all ones
// (never), or the value.
unsigned int deferral(long long set, unsigned int dflt)
{
    if (set == 0) return dflt;
    if (set < 0) return 0xffffffffu;
    return set > 0xffffffffll ? 0xffffffffu : (unsigned int)set;
}

unsigned int heavy_cands_env()
{
    static unsigned int v = env_uint("GHN_HEAVY_CANDS", 8192u);
    return v;
}

// The one-launch build of small dense indexes (build_kernels.cu); GHN_SMALL_BUILD=0
// takes the multi-kernel path for every index (the two give the same index).
bool small_build_enabled()
{
    static const bool v = [] {
        const char* s = getenv("GHN_SMALL_BUILD");
        return !(s && s[0] == '0');
    }();
    return v;
}

long long max_layers_env()
{
    static long long v = [] {
        const char* s = getenv("GHN_MAX_LAYERS");
        return s ? atoll(s) : 0ll;
    }();
    return v;
}

// Default bound on a query's work: 2^22 cell rows enumerated over its layers
// (the rows of cube(L) clipped to the box, summed over the layers visited).
// A walk on a grid far finer than its k-th distance (e.g. a measured grid on
// dense data) needs thousands of layers of (2L + 1)^(d - 1) rows each; this
// bound ends such a query after a few hundred layers in d = 3, with -1 / +inf
// rows and KNN_ELIMIT, so that one call cannot run for minutes.  The bench
// and test workloads enumerate at most a few thousand rows per query.
// GHN_MAX_ROWS overrides it (0 or a negative value: no bound).
constexpr long long kDefaultMaxRows = 1ll << 22;

long long max_rows_env()
{
    static long long v = [] {
        const char* s = getenv("GHN_MAX_ROWS");
        if (!s || !*s) return kDefaultMaxRows;
        const long long x = atoll(s);
        return x > 0 ? x : 0ll;
    }();
    return v;
}

// ---- phase timing (knn_timing_enable / knn_timing_read) ----

std::atomic<int> g_timing_on{0};
std::atomic<long long> g_launches{0};

// The phase events of one call.
struct PhaseCall {
    static constexpr int kMax = 40;
    cudaEvent_t ev[kMax + 1] = {};
    const char* names[kMax] = {};
    int count = 0;  // phases recorded
    int device = -1;

    void ensure(int dev)
    {
        if (device == dev) return;
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        for (auto& e : ev) cudaEventCreate(&e);
        device = dev;
    }
};

// A ring of the calling thread's last calls, read oldest first, so that a
// caller can read them after a whole sequence of calls, without a
// synchronisation between the calls.
struct PhaseTimer {
    static constexpr int kRing = 32;
    PhaseCall calls[kRing];
    long long head = 0;  // calls begun
    long long tail = 0;  // calls read (or dropped)
    PhaseCall* cur = nullptr;

    void reset()
    {
        tail = head;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        for (auto& c : calls) c.ensure(dev);  // no event creation inside a timed loop
    }
    void begin(cudaStream_t s)
    {
        cur = nullptr;
        if (g_timing_on.load() == 0) return;
        if (head - tail == kRing) ++tail;  // the oldest unread call is dropped
        PhaseCall& c = calls[head % kRing];
        ++head;
        int dev = 0;
        cudaGetDevice(&dev);
        c.ensure(dev);
        c.count = 0;
        cudaEventRecord(c.ev[0], s);
        cur = &c;
    }
    void mark(const char* name, cudaStream_t s)
    {
        if (!cur || cur->count >= PhaseCall::kMax) return;
        cur->names[cur->count] = name;
        cudaEventRecord(cur->ev[cur->count + 1], s);
        ++cur->count;
    }
};

thread_local PhaseTimer g_timer;

std::once_flag g_pool_once[64];

void tune_pool(int dev)
{
    if (dev < 0 || dev >= 64) return;
    std::call_once(g_pool_once[dev], [dev] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            unsigned long long keep = ~0ull;  // keep freed blocks for reuse
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    });
}

template <class T>
knn_status dalloc(T** p, size_t count, cudaStream_t s, const char* what)
{
    *p = nullptr;
    const long long nth = ++g_alloc_count;
    const long long at = fail_alloc_at();
    if (at > 0 && nth == at) {
        set_err("%s: allocation %lld failed (injected by GHN_FAIL_ALLOC_AT)", what, nth);
        return KNN_ENOMEM;
    }
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(p), bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_err("%s: cudaMallocAsync of %zu bytes failed: %s", what, bytes, cudaGetErrorString(e));
        return KNN_ENOMEM;
    }
    return KNN_OK;
}

template <class T>
void dfree(T*& p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
}

// Frees every registered temporary on scope exit.
struct Temps {
    cudaStream_t s;
    void* ptrs[24];
    int n = 0;
    explicit Temps(cudaStream_t s_) : s(s_) {}
    template <class T>
    knn_status alloc(T** p, size_t count, const char* what)
    {
        knn_status st = dalloc(p, count, s, what);
        if (st == KNN_OK) ptrs[n++] = *p;
        return st;
    }
    ~Temps()
    {
        for (int i = 0; i < n; ++i) cudaFreeAsync(ptrs[i], s);
    }
};

// Where a caller buffer lives: 1 device memory of the current GPU (or managed
// memory), 0 host memory, -1 device memory of another GPU.  The kernels would
// reach another GPU's memory as a peer address with no peer access set up, so
// such buffers are refused.
int pointer_kind(const void* p)
{
    if (!p) return 0;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (at.type == cudaMemoryTypeManaged) return 1;
    if (at.type != cudaMemoryTypeDevice) return 0;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return -1;
    return at.device == cur ? 1 : -1;
}

knn_status other_gpu(const char* what)
{
    set_err("%s: device memory of another GPU than the index's", what);
    return KNN_EINVAL;
}

// Device view of a caller buffer: the pointer itself when it is device memory,
// else a temporary (copied in when `in` is set).
template <class T>
knn_status device_view(const T* user, size_t count, bool in, Temps& tmp, T** out,
                       const char* what)
{
    if (!user) {
        *out = nullptr;
        return KNN_OK;
    }
    const int kind = pointer_kind(user);
    if (kind < 0) return other_gpu(what);
    if (kind > 0) {
        *out = const_cast<T*>(user);
        return KNN_OK;
    }
    knn_status st = tmp.alloc(out, count, what);
    if (st != KNN_OK) return st;
    if (in) GHN_CHECK(cudaMemcpyAsync(*out, user, count * sizeof(T), cudaMemcpyHostToDevice, tmp.s),
                      what);
    return KNN_OK;
}

// An output buffer as the kernels see it.  Device memory is used as is.
// Pinned host memory that the GPU can address (NVLink-C2C on GB300, mapped
// memory elsewhere) is written by the kernels directly, so the results cross
// to the host while the search runs.  Any other host memory gets a temporary
// that is copied out after the kernels.
template <class T>
struct OutView {
    T* dev = nullptr;     // what the kernels write
    bool staged = false;  // dev is a temporary: copy it to the caller's buffer
    bool host = false;    // the caller's buffer is host memory: synchronize before returning
};

template <class T>
knn_status output_view(T* user, size_t count, Temps& tmp, OutView<T>* v, const char* what)
{
    *v = OutView<T>{};
    if (!user) return KNN_OK;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, user) != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
        at.devicePointer = nullptr;
    }
    if (at.type == cudaMemoryTypeManaged) {
        v->dev = user;
        return KNN_OK;
    }
    if (at.type == cudaMemoryTypeDevice) {
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess || at.device != cur) return other_gpu(what);
        v->dev = user;
        return KNN_OK;
    }
    v->host = true;
    if (at.type == cudaMemoryTypeHost && at.devicePointer) {
        v->dev = static_cast<T*>(at.devicePointer);
        return KNN_OK;
    }
    v->staged = true;
    return tmp.alloc(&v->dev, count, what);
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int num_sms(int dev)
{
    static int cache[64] = {0};
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 1;
    if (dev >= 0 && dev < 64) cache[dev] = v;
    return v;
}

// A non-blocking stream per device for copies that overlap a build (created
// on first use, kept for the life of the process), or null.
cudaStream_t side_stream(int dev)
{
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

bool pinned_host(const void* p)
{
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

void free_index(ghn_index* x)
{
    if (!x) return;
    DeviceGuard dg(x->device);
    cudaStream_t s = 0;
    if (x->last_use) cudaStreamWaitEvent(s, x->last_use, 0);
    dfree(x->rows, s);
    dfree(x->rid, s);
    dfree(x->labels, s);
    dfree(x->dstart, s);
    dfree(x->slots, s);
    dfree(x->bitmap, s);
    dfree(x->gdev, s);
    if (x->last_use) cudaEventDestroy(x->last_use);
    delete x;
}

knn_status build_impl(const float* points_user, const void* labels_user, long long n, int d,
                      const Widths& wd, int table, cudaStream_t s, ghn_index** out)
{
    int dev = 0;
    GHN_CHECK(cudaGetDevice(&dev), "cudaGetDevice");
    tune_pool(dev);
    ghn_index* x = new ghn_index();
    cudaEvent_t lab_done = nullptr;  // the side-stream copy of pinned host labels
    // on failure: wait for the work already queued (on the stream and the
    // side stream), then release
    auto fail = [&](knn_status code) {
        cudaStreamSynchronize(s);
        if (lab_done) {
            cudaEventSynchronize(lab_done);
            cudaEventDestroy(lab_done);
            lab_done = nullptr;
        }
        cudaGetLastError();
        free_index(x);
        return code;
    };
    x->device = dev;
    x->n = n;
    x->d = d;
    x->wd = wd;
    knn_status st = KNN_OK;
    g_timer.begin(s);
    {
        Temps tmp(s);
        const float* pts = nullptr;
        float* pts_dev = nullptr;
        st = device_view(points_user, (size_t)(n * d), true, tmp, &pts_dev, "points");
        pts = pts_dev;
        // labels: a caller's device buffer is copied into the index at the
        // end; pinned host labels go straight into the index on a side stream,
        // overlapping the build (joined before the build returns); other
        // host labels are staged first
        const unsigned int* lab_in = nullptr;
        if (st == KNN_OK && labels_user) {
            const auto* lu = static_cast<const unsigned int*>(labels_user);
            cudaStream_t side = pinned_host(lu) ? side_stream(dev) : nullptr;
            cudaEvent_t ready = nullptr;
            if (side && dalloc(&x->labels, (size_t)n, s, "labels") == KNN_OK &&
                cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&lab_done, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventRecord(ready, s) == cudaSuccess &&
                cudaStreamWaitEvent(side, ready, 0) == cudaSuccess &&
                cudaMemcpyAsync(x->labels, lu, (size_t)n * 4, cudaMemcpyHostToDevice, side) ==
                    cudaSuccess &&
                cudaEventRecord(lab_done, side) == cudaSuccess) {
                cudaEventDestroy(ready);
            } else {
                cudaGetLastError();
                if (ready) cudaEventDestroy(ready);
                if (lab_done) {
                    // a copy may have been queued: wait for the side stream
                    // before the labels buffer is used or freed
                    if (side) cudaStreamSynchronize(side);
                    cudaEventDestroy(lab_done);
                    lab_done = nullptr;
                }
                if (x->labels) {
                    dfree(x->labels, s);
                    x->labels = nullptr;
                }
                unsigned int* lv = nullptr;
                st = device_view(lu, (size_t)n, true, tmp, &lv, "labels");
                lab_in = lv;
            }
        }
        g_timer.mark("stage", s);
        // ---- box of the training points and cells per dimension (one sync) ----
        const int pb = box_partial_blocks(n);
        float* partial = nullptr;
        BoxOut* box_dev = nullptr;
        if (st == KNN_OK) st = tmp.alloc(&partial, (size_t)pb * (2 * d + 1), "box partials");
        if (st == KNN_OK) st = tmp.alloc(&box_dev, 1, "box");
        if (st != KNN_OK) {
            return fail(st);
        }
        BoxOut box;
        cudaError_t e = launch_box(pts, n, d, wd, partial, pb, box_dev, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&box, box_dev, sizeof(box), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            return fail(cuda_fail(e, "box"));
        }
        g_timer.mark("box", s);
        if (box.flags & kStatusNonFinite) {
            set_err("knn_build: a training coordinate is not finite");
            return fail(KNN_EINVAL);
        }
        if (box.flags & kStatusExtent) {
            set_err("knn_build: more than 2^31 - 1 cells along one dimension (cell width too small)");
            return fail(KNN_EINVAL);
        }
        GridConst& g = x->g;
        memset(&g, 0, sizeof(g));
        for (int j = 0; j < d; ++j) {
            g.w[j] = wd.w[j];
            g.inv_w[j] = 1.0f / wd.w[j];
            g.split[j] = wd.split[j];
        }
        g.d = d;
        unsigned long long space = 1ull;
        bool overflow = false;
        for (int j = 0; j < d; ++j) {
            g.lo[j] = box.lo[j];
            g.cmax[j] = box.ext[j] - 1;
            const unsigned long long ext = (unsigned long long)box.ext[j];
            if (space > (0x7fffffffffffffffull / ext)) overflow = true;
            space *= ext;
        }
        if (overflow) {
            set_err("knn_build: more than 2^63 cells in the box of the points (cell width too small)");
            return fail(KNN_EINVAL);
        }
        unsigned long long stride = 1ull;
        for (int j = d - 1; j >= 0; --j) {
            g.stride[j] = stride;
            stride *= (unsigned long long)box.ext[j];
        }
        x->ncell_space = space;
        int bits = 0;
        while (bits < 64 && (1ull << bits) < space) ++bits;
        x->key_bits = bits;
        if (table == KNN_TABLE_AUTO)
            table = space <= 4ull * (unsigned long long)n + 1024ull ? KNN_TABLE_DENSE : KNN_TABLE_HASH;
        if (table == KNN_TABLE_DENSE && space + 1ull > 0x7fffffffull) {
            set_err("knn_build: a dense table over %llu cells is too large; use KNN_TABLE_HASH",
                    space);
            return fail(KNN_EINVAL);
        }
        x->table = table;

        if (table == KNN_TABLE_DENSE && n <= kSmallMaxN && space <= kSmallMaxCells &&
            small_build_enabled()) {
            // ---- small dense index: ids, sort, rows, table in one launch ----
            st = dalloc(&x->rid, (size_t)n, s, "row ids");
            if (st == KNN_OK) st = dalloc(&x->gdev, 1, s, "grid");
            if (st == KNN_OK) st = dalloc(&x->dstart, (size_t)space + 1, s, "dense table");
            if (st == KNN_OK) st = dalloc(&x->rows, (size_t)n * row_floats(d), s, "rows");
            if (st == KNN_OK && lab_in) st = dalloc(&x->labels, (size_t)n, s, "labels");
            if (st != KNN_OK) return fail(st);
            e = launch_small_build(pts, n, d, g, space, x->rid, x->rows, x->dstart, x->gdev, s);
            g_timer.mark("small", s);
            if (e == cudaSuccess && lab_in)
                e = cudaMemcpyAsync(x->labels, lab_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
            if (lab_done) {
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s, lab_done, 0);
                cudaEventDestroy(lab_done);
                lab_done = nullptr;
            }
            g_timer.mark("gather", s);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x->last_use, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(x->last_use, s);
            if (e != cudaSuccess) return fail(cuda_fail(e, "small build"));
            *out = x;
            return KNN_OK;
        }

        // ---- Eq. 1 keys, stable sort by cell, cell offsets, table, row gather ----
        // 32-bit keys when every cell id of the box fits (space <= 2^32)
        const bool narrow = bits <= 32;
        char *ka = nullptr, *kb = nullptr;
        unsigned int *va = nullptr, *vb = nullptr;
        void* rtmp = nullptr;
        void* stmp = nullptr;
        unsigned long long* cell_key = nullptr;
        unsigned int* cell_start = nullptr;
        const size_t key_bytes = narrow ? sizeof(unsigned int) : sizeof(unsigned long long);
        st = tmp.alloc(&ka, (size_t)n * key_bytes, "keys");
        if (st == KNN_OK) st = tmp.alloc(&kb, (size_t)n * key_bytes, "keys");
        if (st == KNN_OK) st = dalloc(&va, (size_t)n, s, "row ids");
        if (st == KNN_OK) st = dalloc(&vb, (size_t)n, s, "row ids");
        if (st == KNN_OK) st = tmp.alloc(reinterpret_cast<char**>(&rtmp), radix_temp_bytes(n), "sort temp");
        if (st != KNN_OK) {
            dfree(va, s);
            dfree(vb, s);
            return fail(st);
        }
        void* sk = nullptr;
        unsigned int* sv = nullptr;
        if (narrow) {
            auto k32a = reinterpret_cast<unsigned int*>(ka), k32b = reinterpret_cast<unsigned int*>(kb);
            unsigned int* sk32 = nullptr;
            e = launch_cell_keys(pts, n, g, k32a, s);
            g_timer.mark("keys", s);
            if (e == cudaSuccess)
                e = radix_sort_pairs(k32a, va, k32b, vb, n, bits, rtmp, &sk32, &sv, s, true);
            sk = sk32;
        } else {
            auto k64a = reinterpret_cast<unsigned long long*>(ka);
            auto k64b = reinterpret_cast<unsigned long long*>(kb);
            unsigned long long* sk64 = nullptr;
            e = launch_cell_keys(pts, n, g, k64a, s);
            g_timer.mark("keys", s);
            if (e == cudaSuccess)
                e = radix_sort_pairs(k64a, va, k64b, vb, n, bits, rtmp, &sk64, &sv, s, true);
            sk = sk64;
        }
        g_timer.mark("sort", s);
        if (e != cudaSuccess) {
            dfree(va, s);
            dfree(vb, s);
            return fail(cuda_fail(e, "sort by cell"));
        }
        // the sorted values are the training index of every row, in cell order
        x->rid = sv;
        if (sv == va)
            dfree(vb, s);
        else
            dfree(va, s);

        const unsigned long long scan_n =
            table == KNN_TABLE_DENSE && space + 1ull > (unsigned long long)n ? space + 1ull
                                                                           : (unsigned long long)n;
        st = tmp.alloc(reinterpret_cast<char**>(&stmp), scan_temp_bytes((long long)scan_n), "scan temp");
        if (st == KNN_OK) st = tmp.alloc(&cell_key, (size_t)n, "cell keys");
        if (st == KNN_OK) st = tmp.alloc(&cell_start, (size_t)n + 1, "cell starts");
        if (st == KNN_OK) st = dalloc(&x->gdev, 1, s, "grid");
        if (st != KNN_OK) {
            return fail(st);
        }
        e = narrow ? launch_cells(static_cast<const unsigned int*>(sk), n, stmp, cell_key, cell_start,
                                  x->gdev, s)
                   : launch_cells(static_cast<const unsigned long long*>(sk), n, stmp, cell_key,
                                  cell_start, x->gdev, s);
        if (e != cudaSuccess) {
            return fail(cuda_fail(e, "cells"));
        }
        g_timer.mark("cells", s);
        if (table == KNN_TABLE_DENSE) {
            st = dalloc(&x->dstart, (size_t)space + 1, s, "dense table");
            if (st != KNN_OK) {
                return fail(st);
            }
            e = launch_dense_table(cell_key, cell_start, x->gdev, space, x->dstart, stmp, s);
        } else {
            unsigned long long cap = 16ull;
            while (cap < 2ull * (unsigned long long)n) cap <<= 1;
            x->max_slots = cap;
            st = dalloc(&x->slots, (size_t)cap, s, "hash table");
            if (st != KNN_OK) {
                return fail(st);
            }
            e = launch_hash_table(cell_key, cell_start, x->gdev, x->slots, cap, s);
            // an occupancy bitmap over the box when it is small next to the
            // points (at most 64 bytes per point, 1 GiB): a row's occupied
            // cells then cost one word load, and only two of them are probed
            if (e == cudaSuccess && space <= (1ull << 33) && space / 8ull <= 64ull * (unsigned long long)n) {
                const unsigned long long words = (space + 31ull) / 32ull;
                st = dalloc(&x->bitmap, (size_t)words, s, "occupancy bitmap");
                if (st != KNN_OK) return fail(st);
                e = launch_bitmap(cell_key, x->gdev, x->bitmap, words, s);
            }
        }
        if (e != cudaSuccess) {
            return fail(cuda_fail(e, "cell table"));
        }
        g_timer.mark("table", s);
        st = dalloc(&x->rows, (size_t)n * row_floats(d), s, "rows");
        if (st == KNN_OK && lab_in) st = dalloc(&x->labels, (size_t)n, s, "labels");
        if (st != KNN_OK) {
            return fail(st);
        }
        e = launch_gather(pts, n, d, x->rid, x->rows, s);
        if (e == cudaSuccess && lab_in)
            e = cudaMemcpyAsync(x->labels, lab_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
        if (lab_done) {
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, lab_done, 0);
            cudaEventDestroy(lab_done);
            lab_done = nullptr;
        }
        g_timer.mark("gather", s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x->last_use, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(x->last_use, s);
        if (e != cudaSuccess) {
            return fail(cuda_fail(e, "gather"));
        }
    }  // temporaries are freed here, ordered on the stream
    *out = x;
    return KNN_OK;
}

knn_status query_impl(const ghn_index* x, const float* queries_user, long long m, int k, int mode,
                      int* ids_user, float* dist2_user, void* pred_user, long long* stats_user,
                      int flags, cudaStream_t s)
{
    DeviceGuard dg(x->device);
    const int d = x->d;
    knn_status st = KNN_OK;
    unsigned int status_host = 0u;
    bool host_out = false;
    g_timer.begin(s);
    {
        Temps tmp(s);
        float* q = nullptr;
        OutView<int> v_ids;
        OutView<float> v_d2;
        OutView<unsigned int> v_pred;
        OutView<long long> v_stats;
        st = device_view(queries_user, (size_t)(m * d), true, tmp, &q, "queries");
        if (st == KNN_OK) st = output_view(ids_user, (size_t)(m * k), tmp, &v_ids, "ids");
        if (st == KNN_OK) st = output_view(dist2_user, (size_t)(m * k), tmp, &v_d2, "dist2");
        if (st == KNN_OK && mode >= 0)
            st = output_view(static_cast<unsigned int*>(pred_user), (size_t)m, tmp, &v_pred, "pred");
        if (st == KNN_OK) st = output_view(stats_user, (size_t)(m * 3), tmp, &v_stats, "stats");
        if (st != KNN_OK) return st;
        int* ids = v_ids.dev;
        float* dist2 = v_d2.dev;
        unsigned int* pred = v_pred.dev;
        long long* stats = v_stats.dev;
        host_out = v_ids.host || v_d2.host || v_pred.host || v_stats.host;

        g_timer.mark("stage", s);
        // scratch: work counter, status word, deferral counters, deferred list
        unsigned long long* scratch = nullptr;
        st = tmp.alloc(&scratch, 4, "query scratch");
        if (st != KNN_OK) return st;
        GHN_CHECK(cudaMemsetAsync(scratch, 0, 4 * sizeof(unsigned long long), s), "memset");
        unsigned int* heavy = nullptr;
        if (!stats) {
            st = tmp.alloc(&heavy, (size_t)m, "deferred queries");
            if (st != KNN_OK) return st;
        }

        const unsigned int* order = nullptr;
        if ((flags & KNN_QUERY_SORTED) && m > 1 && x->key_bits > 0) {
            // the order only has to bring queries of nearby cells together:
            // sort by the top kOrderBits bits of the cell id (two 8-bit passes)
            const int shift = x->key_bits > kOrderBits ? x->key_bits - kOrderBits : 0;
            unsigned int *ka = nullptr, *kb = nullptr;
            unsigned int *va = nullptr, *vb = nullptr;
            char* rtmp = nullptr;
            st = tmp.alloc(&ka, (size_t)m, "query keys");
            if (st == KNN_OK) st = tmp.alloc(&kb, (size_t)m, "query keys");
            if (st == KNN_OK) st = tmp.alloc(&va, (size_t)m, "query order");
            if (st == KNN_OK) st = tmp.alloc(&vb, (size_t)m, "query order");
            if (st == KNN_OK) st = tmp.alloc(&rtmp, radix_temp_bytes(m), "sort temp");
            if (st != KNN_OK) return st;
            unsigned int *sk, *sv;
            GHN_CHECK(launch_query_keys(q, m, x->g, shift, ka, s), "query keys");
            GHN_CHECK(radix_sort_pairs(ka, va, kb, vb, m, x->key_bits - shift, rtmp, &sk, &sv, s,
                                       true),
                      "query order");
            order = sv;
        }

        g_timer.mark("order", s);
        QueryArgs a;
        memset(&a, 0, sizeof(a));
        a.g = x->g;
        a.q = q;
        a.m = m;
        a.k = k;
        a.mode = mode;
        a.ids = ids;
        a.dist2 = dist2;
        a.pred = pred;
        a.rows = x->rows;
        a.rid = x->rid;
        a.labels = x->labels;
        a.dstart = x->dstart;
        a.slots = x->slots;
        a.bitmap = x->bitmap;
        a.gdev = x->gdev;
        a.counter = scratch;
        a.status = reinterpret_cast<unsigned int*>(scratch + 1);
        a.heavy_count = reinterpret_cast<unsigned int*>(scratch + 2);
        a.heavy_cursor = reinterpret_cast<unsigned int*>(scratch + 2) + 1;
        a.heavy_list = heavy;
        a.heavy_rows = deferral(x->defer_rows, heavy_rows_env(x->d));
        a.heavy_cands = deferral(x->defer_cands, heavy_cands_env());
        a.stats = stats;
        a.order = order;
        a.max_layers = max_layers_env();
        a.max_rows = max_rows_env();
        a.dense = x->table == KNN_TABLE_DENSE;
        a.exact = (flags & KNN_QUERY_EXACT) ? 1 : 0;
        // the launcher marks "search" (warp kernel) and "coop" (cooperative kernel)
        set_kernel_marks(true);
        const cudaError_t le = launch_query(a, num_sms(x->device), s);
        set_kernel_marks(false);
        GHN_CHECK(le, "query kernel");

        if (v_ids.staged)
            GHN_CHECK(cudaMemcpyAsync(ids_user, ids, (size_t)(m * k) * 4, cudaMemcpyDeviceToHost, s), "ids");
        if (v_d2.staged)
            GHN_CHECK(cudaMemcpyAsync(dist2_user, dist2, (size_t)(m * k) * 4, cudaMemcpyDeviceToHost, s), "dist2");
        if (v_pred.staged)
            GHN_CHECK(cudaMemcpyAsync(pred_user, pred, (size_t)m * 4, cudaMemcpyDeviceToHost, s), "pred");
        if (v_stats.staged)
            GHN_CHECK(cudaMemcpyAsync(stats_user, stats, (size_t)(m * 3) * 8, cudaMemcpyDeviceToHost, s), "stats");
        if ((flags & KNN_QUERY_CHECKED) || stats_user)
            GHN_CHECK(cudaMemcpyAsync(&status_host, scratch + 1, 4, cudaMemcpyDeviceToHost, s), "status");
        g_timer.mark("copy", s);
        GHN_CHECK(cudaEventRecord(x->last_use, s), "event");
    }
    if (host_out || (flags & KNN_QUERY_CHECKED) || stats_user)
        GHN_CHECK(cudaStreamSynchronize(s), "synchronize");
    if ((flags & KNN_QUERY_CHECKED) || stats_user) {
        if (status_host & kStatusNonFinite) {
            set_err("knn_query: a query coordinate is not finite");
            return KNN_EINVAL;
        }
        if (status_host & kStatusLimit) {
            set_err("knn_query: a query reached its work bound (rows or layer cap)");
            return KNN_ELIMIT;
        }
    }
    return KNN_OK;
}

knn_status check_query_args(const ghn_index* x, const float* queries, long long m, int k, int mode,
                            const int* ids, const void* pred)
{
    if (!x) {
        set_err("knn_query: index is NULL");
        return KNN_EINVAL;
    }
    if (m < 0 || m >= (1ll << 31)) {
        set_err("knn_query: m = %lld outside [0, 2^31)", m);
        return KNN_EINVAL;
    }
    if (k < 1 || k > kMaxK) {
        set_err("knn_query: k = %d outside [1, %d]", k, kMaxK);
        return KNN_EINVAL;
    }
    if (mode < -1 || mode > 2) {
        set_err("knn_query: unknown mode %d", mode);
        return KNN_EINVAL;
    }
    if (mode >= 0 && !x->labels) {
        set_err("knn_query: a prediction needs labels, and the index has none");
        return KNN_EINVAL;
    }
    if (m > 0 && (!queries || !ids)) {
        set_err("knn_query: queries and ids must not be NULL");
        return KNN_EINVAL;
    }
    if (m > 0 && mode >= 0 && !pred) {
        set_err("knn_query: pred must not be NULL for a prediction");
        return KNN_EINVAL;
    }
    return KNN_OK;
}

}  // namespace

namespace ghn {

void count_launches(long long k) { g_launches += k; }

void phase_begin(cudaStream_t s) { g_timer.begin(s); }
void phase_mark(const char* name, cudaStream_t s) { g_timer.mark(name, s); }

thread_local bool g_kernel_marks = false;
void set_kernel_marks(bool on) { g_kernel_marks = on; }
void kernel_mark(const char* name, cudaStream_t s)
{
    if (g_kernel_marks) g_timer.mark(name, s);
}

// Accessors for entry points defined in other translation units.
void set_error(const char* msg) { set_err("%s", msg); }

int index_device(const ghn_index* x) { return x->device; }

int device_sms(int dev) { return num_sms(dev); }

bool index_has_labels(const ghn_index* x) { return x->labels != nullptr; }

int index_dims(const ghn_index* x) { return x->d; }

void index_query_args(const ghn_index* x, QueryArgs& a)
{
    a.g = x->g;
    a.rows = x->rows;
    a.rid = x->rid;
    a.labels = x->labels;
    a.dstart = x->dstart;
    a.slots = x->slots;
    a.bitmap = x->bitmap;
    a.gdev = x->gdev;
    a.max_layers = max_layers_env();
    a.max_rows = max_rows_env();
    a.heavy_rows = deferral(x->defer_rows, heavy_rows_env(x->d));
    a.heavy_cands = deferral(x->defer_cands, heavy_cands_env());
    a.dense = x->table == KNN_TABLE_DENSE;
}

void index_mark_use(const ghn_index* x, cudaStream_t s) { cudaEventRecord(x->last_use, s); }

long long index_bytes(const ghn_index* x)
{
    long long b = x->n * (long long)row_floats(x->d) * 4 + x->n * 4;  // rows, rid
    if (x->labels) b += x->n * 4;
    if (x->dstart) b += ((long long)x->ncell_space + 1) * 4;
    if (x->slots) b += (long long)x->max_slots * (long long)sizeof(HashSlot);
    if (x->bitmap) b += (long long)((x->ncell_space + 31ull) / 32ull) * 4;
    return b + (long long)sizeof(GridDev);
}

cudaError_t launch_batch_query(const BatchArgs& g, int sms, cudaStream_t s)
{
    count_launches(1);
    if (g.d <= 2) return launch_batch_query_d12(g, sms, s);
    if (g.d <= 4) return launch_batch_query_d34(g, sms, s);
    if (g.d <= 6) return launch_batch_query_d56(g, sms, s);
    return launch_batch_query_d78(g, sms, s);
}

knn_status device_alloc(void** p, size_t bytes, cudaStream_t s, const char* what)
{
    char* c = nullptr;
    knn_status st = dalloc(&c, bytes, s, what);
    *p = c;
    return st;
}

void device_free(void* p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

cudaStream_t copy_stream(int dev) { return side_stream(dev); }
unsigned int heavy_rows_default(int d) { return heavy_rows_env(d); }
unsigned int deferral_threshold(long long set, unsigned int dflt) { return deferral(set, dflt); }
unsigned int heavy_cands_default() { return heavy_cands_env(); }
long long max_layers_default() { return max_layers_env(); }
long long max_rows_default() { return max_rows_env(); }
void tune_device_pool(int dev) { tune_pool(dev); }

cudaError_t launch_query(const QueryArgs& a, int sms, cudaStream_t s)
{
    const int d = a.g.d;
    count_launches(1);
    if (d <= 2) return launch_query_d12(a, sms, s);
    if (d <= 4) return launch_query_d34(a, sms, s);
    if (d <= 6) return launch_query_d56(a, sms, s);
    return launch_query_d78(a, sms, s);
}

}  // namespace ghn

extern "C" {

knn_status knn_build(const float* points, const void* labels, int64_t n, int32_t d,
                     float cell_width, int32_t table, void* stream, ghn_index** out)
{
    float widths[kMaxD];
    for (int j = 0; j < kMaxD; ++j) widths[j] = cell_width;
    return knn_build_grid(points, labels, n, d, widths, nullptr, table, stream, out);
}

knn_status knn_build_grid(const float* points, const void* labels, int64_t n, int32_t d,
                          const float* cell_widths, const int64_t* splits, int32_t table,
                          void* stream, ghn_index** out)
{
    if (!out) {
        set_err("knn_build: out is NULL");
        return KNN_EINVAL;
    }
    *out = nullptr;
    if (!points) {
        set_err("knn_build: points is NULL");
        return KNN_EINVAL;
    }
    if (n < 1 || n >= (1ll << 31)) {
        set_err("knn_build: n = %lld outside [1, 2^31)", (long long)n);
        return KNN_EINVAL;
    }
    if (d < 1 || d > kMaxD) {
        set_err("knn_build: d = %d outside [1, %d]", d, kMaxD);
        return KNN_EINVAL;
    }
    if (!cell_widths) {
        set_err("knn_build: cell widths are NULL");
        return KNN_EINVAL;
    }
    Widths wd{};
    for (int j = 0; j < d; ++j) {
        if (!(cell_widths[j] > 0.0f) || !isfinite(cell_widths[j])) {
            set_err("knn_build: cell width must be a positive finite number");
            return KNN_EINVAL;
        }
        if (splits && (splits[j] < 1 || splits[j] >= (1ll << 31))) {
            set_err("knn_build: split counts must be in [1, 2^31)");
            return KNN_EINVAL;
        }
        wd.w[j] = cell_widths[j];
        wd.split[j] = splits ? splits[j] : 0;
    }
    if (table < KNN_TABLE_AUTO || table > KNN_TABLE_HASH) {
        set_err("knn_build: unknown table kind %d", table);
        return KNN_EINVAL;
    }
    return build_impl(points, labels, n, d, wd, table, static_cast<cudaStream_t>(stream), out);
}

knn_status knn_index_grid(const ghn_index* index, float* cell_widths, int64_t* splits)
{
    if (!index) {
        set_err("knn_index_grid: index is NULL");
        return KNN_EINVAL;
    }
    for (int j = 0; j < index->d; ++j) {
        if (cell_widths) cell_widths[j] = index->wd.w[j];
        if (splits) splits[j] = index->wd.split[j];
    }
    return KNN_OK;
}

knn_status knn_query(const ghn_index* index, const float* queries, int64_t m, int32_t k,
                     int32_t mode, int32_t* ids, float* dist2, void* pred, int32_t flags,
                     void* stream)
{
    knn_status st = check_query_args(index, queries, m, k, mode, ids, pred);
    if (st != KNN_OK) return st;
    if (m == 0) return KNN_OK;
    return query_impl(index, queries, m, k, mode, ids, dist2, mode >= 0 ? pred : nullptr, nullptr,
                      flags, static_cast<cudaStream_t>(stream));
}

knn_status knn_query_stats(const ghn_index* index, const float* queries, int64_t m, int32_t k,
                           int32_t* ids, float* dist2, int64_t* stats, void* stream)
{
    knn_status st = check_query_args(index, queries, m, k, -1, ids, nullptr);
    if (st != KNN_OK) return st;
    if (m > 0 && !stats) {
        set_err("knn_query_stats: stats must not be NULL");
        return KNN_EINVAL;
    }
    if (m == 0) return KNN_OK;
    return query_impl(index, queries, m, k, -1, ids, dist2, nullptr,
                      reinterpret_cast<long long*>(stats), 0, static_cast<cudaStream_t>(stream));
}

knn_status knn_index_info(const ghn_index* index, knn_index_info_t* info)
{
    if (!index || !info) {
        set_err("knn_index_info: NULL argument");
        return KNN_EINVAL;
    }
    ghn_index* x = const_cast<ghn_index*>(index);
    if (!x->info_ready) {
        DeviceGuard dg(x->device);
        GHN_CHECK(cudaEventSynchronize(x->last_use), "synchronize");
        GHN_CHECK(cudaMemcpy(&x->host_gdev, x->gdev, sizeof(GridDev), cudaMemcpyDeviceToHost),
                  "read grid");
        x->info_ready = true;
    }
    memset(info, 0, sizeof(*info));
    info->n = x->n;
    info->d = x->d;
    info->table = x->table;
    info->cell_width = x->wd.w[0];
    for (int j = 0; j < x->d; ++j) {
        info->origin[j] = x->g.lo[j];
        info->extent[j] = x->g.cmax[j] + 1;
    }
    info->num_cells = (int64_t)x->host_gdev.ncells;
    info->table_slots = x->table == KNN_TABLE_DENSE ? (int64_t)x->ncell_space + 1
                                                    : (int64_t)(x->host_gdev.hmask + 1ull);
    info->row_floats = row_floats(x->d);
    info->has_labels = x->labels != nullptr;
    return KNN_OK;
}

knn_status knn_index_export(const ghn_index* index, uint64_t* cell_keys, uint32_t* cell_start,
                            int32_t* rows)
{
    knn_index_info_t info;
    knn_status st = knn_index_info(index, &info);
    if (st != KNN_OK) return st;
    const ghn_index* x = index;
    DeviceGuard dg(x->device);
    GHN_CHECK(cudaDeviceSynchronize(), "synchronize");
    const long long n = x->n, u = info.num_cells;
    if (rows) GHN_CHECK(cudaMemcpy(rows, x->rid, (size_t)n * 4, cudaMemcpyDeviceToHost), "rows");
    if (!cell_keys && !cell_start) return KNN_OK;
    // rebuild the cell list from the table
    uint64_t* keys = cell_keys;
    uint32_t* starts = cell_start;
    uint64_t* kbuf = nullptr;
    uint32_t* sbuf = nullptr;
    if (!keys) keys = kbuf = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(u > 0 ? u : 1));
    if (!starts) starts = sbuf = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(u + 1));
    if (!keys || !starts) {
        free(kbuf);
        free(sbuf);
        set_err("knn_index_export: out of host memory");
        return KNN_ENOMEM;
    }
    long long c = 0;
    if (x->table == KNN_TABLE_DENSE) {
        const size_t cnt = (size_t)x->ncell_space + 1;
        uint32_t* ds = (uint32_t*)malloc(sizeof(uint32_t) * cnt);
        if (!ds) {
            free(kbuf);
            free(sbuf);
            set_err("knn_index_export: out of host memory");
            return KNN_ENOMEM;
        }
        cudaError_t e = cudaMemcpy(ds, x->dstart, sizeof(uint32_t) * cnt, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            free(ds);
            free(kbuf);
            free(sbuf);
            return cuda_fail(e, "read table");
        }
        for (unsigned long long id = 0; id < x->ncell_space; ++id) {
            if (ds[id + 1] > ds[id] && c < u) {
                keys[c] = id;
                starts[c] = ds[id];
                ++c;
            }
        }
        free(ds);
    } else {
        const size_t cap = (size_t)(x->host_gdev.hmask + 1ull);
        HashSlot* hs = (HashSlot*)malloc(sizeof(HashSlot) * cap);
        if (!hs) {
            free(kbuf);
            free(sbuf);
            set_err("knn_index_export: out of host memory");
            return KNN_ENOMEM;
        }
        cudaError_t e = cudaMemcpy(hs, x->slots, sizeof(HashSlot) * cap, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            free(hs);
            free(kbuf);
            free(sbuf);
            return cuda_fail(e, "read table");
        }
        for (size_t i = 0; i < cap; ++i) {
            if (hs[i].key != kEmptyKey && c < u) {
                keys[c] = hs[i].key;
                starts[c] = hs[i].start;
                ++c;
            }
        }
        // order the occupied slots by cell id
        struct P {
            uint64_t k;
            uint32_t s;
        };
        P* ps = (P*)malloc(sizeof(P) * (size_t)(c > 0 ? c : 1));
        if (!ps) {
            free(hs);
            free(kbuf);
            free(sbuf);
            set_err("knn_index_export: out of host memory");
            return KNN_ENOMEM;
        }
        for (long long i = 0; i < c; ++i) ps[i] = P{keys[i], starts[i]};
        qsort(ps, (size_t)c, sizeof(P), [](const void* a, const void* b) {
            const uint64_t x1 = ((const P*)a)->k, x2 = ((const P*)b)->k;
            return x1 < x2 ? -1 : (x1 > x2 ? 1 : 0);
        });
        for (long long i = 0; i < c; ++i) {
            keys[i] = ps[i].k;
            starts[i] = ps[i].s;
        }
        free(ps);
        free(hs);
    }
    starts[c] = (uint32_t)n;
    free(kbuf);
    free(sbuf);
    if (c != u) {
        set_err("knn_index_export: table holds %lld cells, expected %lld", c, u);
        return KNN_ECUDA;
    }
    return KNN_OK;
}

knn_status knn_timing_enable(int32_t on)
{
    g_timing_on = on ? 1 : 0;
    if (on) g_timer.reset();
    return KNN_OK;
}

int32_t knn_timing_read(const char** names, float* ms, int32_t cap)
{
    PhaseTimer& t = g_timer;
    if (t.tail == t.head) return 0;
    PhaseCall& c = t.calls[t.tail % PhaseTimer::kRing];
    ++t.tail;
    if (c.count == 0) return 0;
    if (cudaEventSynchronize(c.ev[c.count]) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int n = c.count < cap ? c.count : cap;
    for (int i = 0; i < n; ++i) {
        if (names) names[i] = c.names[i];
        if (ms) {
            float v = 0.0f;
            cudaEventElapsedTime(&v, c.ev[i], c.ev[i + 1]);
            ms[i] = v;
        }
    }
    return c.count;
}

int64_t knn_kernel_launches(void) { return g_launches.load(); }

knn_status knn_index_set_deferral(ghn_index* index, int64_t heavy_rows, int64_t heavy_cands)
{
    if (!index) {
        set_err("knn_index_set_deferral: index is NULL");
        return KNN_EINVAL;
    }
    index->defer_rows = heavy_rows;
    index->defer_cands = heavy_cands;
    return KNN_OK;
}

void knn_free(ghn_index* index) { free_index(index); }

const char* knn_last_error(void) { return g_err; }

int32_t knn_abi_version(void) { return 1; }

}  // extern "C"
