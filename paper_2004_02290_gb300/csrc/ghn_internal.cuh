// Internal declarations of the GB300 grid-hashing KNN library (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ghn {

constexpr int kMaxD = 8;
constexpr int kMaxK = 64;
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr float kQueryClamp = 1099511627776.0f;  // 2^40

// Status bits a kernel ORs into a device word.
constexpr unsigned int kStatusNonFinite = 1u;  // a non-finite point or query
constexpr unsigned int kStatusLimit = 2u;      // a query reached its work bound
constexpr unsigned int kStatusExtent = 4u;     // too many cells along one dimension

// Grid geometry, passed by value to the kernels.
struct GridConst {
    float lo[kMaxD];                 // origin: per-dimension minimum
    float w[kMaxD];                  // cell measurement of each dimension
    float inv_w[kMaxD];              // 1 / w_j rounded (bounds only, never Eq. 1)
    int d;
    long long cmax[kMaxD];           // largest occupied cell coordinate (extent - 1)
    unsigned long long stride[kMaxD];  // linear id = sum c_j * stride_j, stride_{d-1} = 1
    long long split[kMaxD];          // training cells clamped to split_j - 1 (0: no clamp)
};

// Cell measurements of a build: a width and an optional split count per dimension.
struct Widths {
    float w[kMaxD];
    long long split[kMaxD];  // 0: no clamp
};

// Results of the build that only the device knows without a sync.
struct GridDev {
    unsigned long long ncells;  // occupied cells U
    unsigned long long hmask;   // hash capacity - 1 (capacity: power of two >= 2U)
};

// Box of the training points, read back once by the host during build.
struct BoxOut {
    float lo[kMaxD];
    float hi[kMaxD];
    long long ext[kMaxD];
    unsigned int flags;
    unsigned int pad;
};

// One open-addressing slot: a linear cell id and its row range [start, end).
struct __align__(16) HashSlot {
    unsigned long long key;
    unsigned int start;
    unsigned int end;
};

// SplitMix64 finaliser (Steele, Lea, Flood 2014; constants as published by
// Vigna): a 64-bit bijective mixer used to spread cell ids over the table.
__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Floats per stored row: 2 for d <= 2, 4 for d <= 4, 8 otherwise.
__host__ __device__ constexpr int row_floats(int d) { return d <= 2 ? 2 : (d <= 4 ? 4 : 8); }

// Count of kernels launched by this library (read by knn_kernel_launches).
void count_launches(long long k);

// Phase timing of knn_timing_enable: a call begins, then marks the end of
// each phase with a static name (no effect while timing is off).
void phase_begin(cudaStream_t s);
void phase_mark(const char* name, cudaStream_t s);
// While set on the calling thread, the query launchers mark the end of each
// kernel they launch (knn_query, and knn_batch_query outside a graph capture).
void set_kernel_marks(bool on);
void kernel_mark(const char* name, cudaStream_t s);
// Phase name of a batched query group's warp kernel, or of its cooperative
// kernel (`coop`): "query.d<d>.<k32|k64>.<dense|hash>[.exact][.coop]".
const char* group_phase_name(int d, int ns, int dense, int exact, bool coop);

// ---- query ----
struct QueryArgs {
    GridConst g;
    const float* q;                 // m*d queries
    long long m;
    int k;
    int mode;                       // -1 none, 0 vote, 1 mean
    int* ids;                       // m*k
    float* dist2;                   // m*k or null
    void* pred;                     // m or null
    const float* rows;              // n rows of row_floats(d) floats, cell order
    const unsigned int* rid;        // n training indices, cell order
    const unsigned int* labels;     // n raw 32-bit outputs, training order, or null
    const unsigned int* dstart;     // dense: ncell_space + 1 row offsets
    const HashSlot* slots;          // hash table
    const unsigned int* bitmap;     // hash: one bit per cell of the box, or null
    unsigned long long key_prefix;  // hash keys are key_prefix | cell id (0 for one index)
    const GridDev* gdev;
    unsigned long long* counter;    // work counter, zero at launch
    unsigned int* status;           // status bits
    unsigned int* heavy_list;       // deferred queries (m entries), or null: no deferral
    unsigned int* heavy_count;      // deferred queries so far, zero at launch
    unsigned int* heavy_cursor;     // cooperative kernel's work counter, zero at launch
    unsigned int heavy_rows;        // defer a query whose layer has more rows than this
    unsigned int heavy_cands;       // or whose row batch holds more candidates than this
    long long* stats;               // m*3 or null (exhaustive counting walk)
    const unsigned int* order;      // visiting order of queries or null
    long long max_layers;           // 0 = no cap
    long long max_rows;             // cap on the cell rows a query enumerates, over its layers (0 = none)
    int dense;
    int exact;                      // certified stop instead of the paper's rule
};

cudaError_t launch_query(const QueryArgs& a, int num_sms, cudaStream_t s);

// A group of indexes queried in one persistent launch: the queries of index i
// are the group's queries qoff[i] .. qoff[i+1]-1.  Every index of a group has
// the same dimension, buffer width (ns: 1 for k <= 32, 2 above), table kind
// and stop rule.
struct BatchArgs {
    const QueryArgs* args;           // device: one per index of the group
    const unsigned long long* qoff;  // device: count + 1 prefix offsets
    int count;
    int d;
    unsigned long long total;        // queries of the group
    unsigned long long* counter;     // zero at launch
    unsigned int* heavy_list;        // total entries, or null: no deferral
    unsigned int* heavy_count;       // zero at launch
    unsigned int* heavy_cursor;      // zero at launch
    int exact;                       // certified stop for every index of the group
    int ns;                          // 1: k <= 32 for every index; 2: k > 32
    int dense;                       // every index has a dense table
};

cudaError_t launch_batch_query(const BatchArgs& g, int num_sms, cudaStream_t s);
cudaError_t launch_batch_query_d12(const BatchArgs& g, int sms, cudaStream_t s);
cudaError_t launch_batch_query_d34(const BatchArgs& g, int sms, cudaStream_t s);
cudaError_t launch_batch_query_d56(const BatchArgs& g, int sms, cudaStream_t s);
cudaError_t launch_batch_query_d78(const BatchArgs& g, int sms, cudaStream_t s);

}  // namespace ghn

struct ghn_index;

namespace ghn {

// Accessors of the index for entry points outside capi.cu.
void set_error(const char* msg);
int index_device(const ghn_index* x);
int device_sms(int dev);
bool index_has_labels(const ghn_index* x);
int index_dims(const ghn_index* x);
void index_query_args(const ghn_index* x, QueryArgs& a);  // the index's part of QueryArgs
void index_mark_use(const ghn_index* x, cudaStream_t s);
long long index_bytes(const ghn_index* x);  // device bytes the index holds

// Allocation through the library's pool (with the GHN_FAIL_ALLOC_AT injector).
int device_alloc(void** p, size_t bytes, cudaStream_t s, const char* what);
void device_free(void* p, cudaStream_t s);
unsigned int heavy_rows_default(int d);
unsigned int heavy_cands_default();
// A per-index deferral setting (0 default, < 0 never, > 0 threshold) as kernels take it.
unsigned int deferral_threshold(long long set, unsigned int dflt);
long long max_layers_default();
long long max_rows_default();
void tune_device_pool(int dev);

// Persistent launch: as many blocks as fit on `sms` SMs (fewer when m is small).
cudaError_t launch_query_d12(const QueryArgs& a, int sms, cudaStream_t s);
cudaError_t launch_query_d34(const QueryArgs& a, int sms, cudaStream_t s);
cudaError_t launch_query_d56(const QueryArgs& a, int sms, cudaStream_t s);
cudaError_t launch_query_d78(const QueryArgs& a, int sms, cudaStream_t s);

}  // namespace ghn
