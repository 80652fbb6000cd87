/*
 * ghn_knn.h: C ABI of the GB300 grid-hashing nearest-neighbour library.
 *
 * The method is GHN ("Grid Hashing Neighborhood", Tchaye-Kondi, Zhai, Zhu,
 * arXiv 2004.02290).  Training points are hashed to the cells of a virtual
 * grid (Sec. III.A, Eq. 1, Algorithm 1).  A query starts from its own cell and
 * visits the surrounding cells layer by layer, keeping the k nearest points
 * seen so far, until a layer brings no update (Sec. III.B, Algorithm 2).  The
 * neighbours' outputs then give a majority vote (classification) or a mean
 * (regression) (Sec. I, Sec. III.D).
 *
 * Conventions shared by every entry point:
 *   - Pointers are plain host or device pointers.  Arguments documented as
 *     "host or device" may point to either; the library asks the CUDA driver
 *     which one it is and stages host data through device memory itself.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Device work is ordered on it.
 *   - Inputs are borrowed: the library copies what it keeps before the call's
 *     work on `stream` completes.  Outputs are owned by the caller.
 *   - Every function returns a knn_status; on failure knn_last_error() holds
 *     a message for the calling thread.
 *   - One device per index: the device current at knn_build time.
 *
 * Readings of points the paper leaves open, fixed by this library:
 *   - origin: per-dimension minimum of the training points; a cell width per
 *     dimension (knn_build_grid) or one for all (knn_build), given by the
 *     caller or measured by the paper's rule (knn_measure_cells).
 *   - cell id (Eq. 1): c_j = floor((p_j - o_j) / w_j) in IEEE single
 *     precision, round to nearest; cells are half-open; on a grid with split
 *     counts, training cells are clamped to s_j - 1 (the last split is
 *     closed); query cells are clamped to [-2^40, 2^40].
 *   - layer L: the cells at Chebyshev distance L from the central cell.
 *   - stop: after layer L when the k-buffer is full and no point of layer L
 *     entered it, or when the layers so far cover every occupied cell.
 *   - order: (squared distance, training index) ascending; squared distance
 *     in single precision, dimension order, no fused multiply-add.
 *   - fewer than k points found: ids padded with -1, distances with +inf.
 *   - vote: largest count, ties to the smallest label.  mean: double-precision
 *     sum in neighbour order divided by the count, rounded to single.
 */
#ifndef GHN_KNN_H
#define GHN_KNN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define KNN_OK 0
#define KNN_EINVAL 1 /* bad argument or input outside what the index can hold */
#define KNN_ENOMEM 2 /* device or host allocation failed */
#define KNN_ECUDA 3  /* a CUDA call failed; knn_last_error() has its text */
#define KNN_ELIMIT 4 /* a query reached its work bound; its rows are -1 / +inf */
#define KNN_ETIMEDOUT 5 /* a wait ended before the request completed (ghn_serve.h) */
typedef int32_t knn_status;

/* Prediction modes (Sec. I and Sec. III.D: majority class, or the average
 * or the median of the outputs). */
#define KNN_NONE -1  /* neighbours only; pred is ignored and may be NULL */
#define KNN_VOTE 0   /* labels are int32 classes; pred receives int32 */
#define KNN_MEAN 1   /* labels are float targets; pred receives float */
#define KNN_MEDIAN 2 /* labels are float targets; pred receives float: the
                        middle output under IEEE total order (-0 < +0), or
                        the two middle ones a, b averaged as
                        (double(a) + double(b)) / 2 for an even count */

/* Cell tables (Sec. III.A: a hash table keyed by the cell id, no empty cells). */
#define KNN_TABLE_AUTO 0  /* dense when the cell box has at most 4n + 1024 cells */
#define KNN_TABLE_DENSE 1 /* direct table over the bounding box of occupied cells */
#define KNN_TABLE_HASH 2  /* open addressing over occupied cells only */

/* knn_query flags. */
#define KNN_QUERY_CHECKED 1 /* synchronize `stream` and return the kernel's status */
#define KNN_QUERY_SORTED 2  /* visit queries grouped by cell (locality in L2): ordered by the
                              top 16 bits of their clamped cell id; results do not change */
#define KNN_QUERY_EXACT 4   /* certified stop instead of the paper's rule: stop after
                               layer L once the k-th squared distance is below the
                               squared distance from the query to every cell outside
                               cube(L), less rounding margins; the neighbours then
                               equal exhaustive KNN's */

typedef struct ghn_index ghn_index; /* opaque; owns all of its device memory */

/* Shape of a built index, for inspection (knn_index_info). */
typedef struct {
    int64_t n;           /* training points */
    int32_t d;           /* dimensions */
    int32_t table;       /* KNN_TABLE_DENSE or KNN_TABLE_HASH */
    float cell_width;    /* w */
    float origin[8];     /* per-dimension minimum of the training points */
    int64_t extent[8];   /* cells per dimension in the box of occupied cells */
    int64_t num_cells;   /* occupied cells (at most n) */
    int64_t table_slots; /* dense entries or hash slots in use */
    int32_t row_floats;  /* floats per stored point row (2, 4 or 8) */
    int32_t has_labels;  /* 1 when labels were given */
} knn_index_info_t;

/*
 * knn_build: cell sampling (Sec. III.A, Eq. 1, Algorithm 1).
 *   points      host or device, n*d float32, row-major (point i at points[i*d]).
 *   labels      host or device, n 32-bit outputs (int32 classes or float
 *               targets, kept as raw bits), or NULL (neighbours only).
 *   n           1 <= n < 2^31.
 *   d           1 <= d <= 8.
 *   cell_width  w > 0, finite.
 *   table       KNN_TABLE_AUTO / _DENSE / _HASH.
 *   stream      cudaStream_t or NULL.
 *   out         receives the new index; NULL on failure.
 * Errors: KNN_EINVAL for a bad argument, a non-finite coordinate, more than
 * 2^31 - 1 cells along one dimension, more than 2^63 cells in the box, or a
 * dense table of more than 2^31 entries; KNN_ENOMEM; KNN_ECUDA.
 * The call synchronizes `stream` once, to read the box of occupied cells.
 * Host inputs are copied to the device; labels in pinned host memory are
 * copied on a library-owned side stream while the build runs, and the build
 * waits for that copy before it returns.
 */
knn_status knn_build(const float* points, const void* labels, int64_t n, int32_t d,
                     float cell_width, int32_t table, void* stream, ghn_index** out);

/*
 * knn_build_grid: knn_build with one cell measurement per dimension (Sec.
 * III.A: all cells have one shape, which need not be a cube).
 *   cell_widths  host, d positive finite widths.
 *   splits       host, d split counts in [1, 2^31), or NULL: training cells
 *                are clamped to splits[j] - 1, so that the largest value lies
 *                in the last split (the grid of knn_measure_cells).
 * Other arguments, errors and synchronisation as knn_build (which is
 * knn_build_grid with every width equal and no splits).
 */
knn_status knn_build_grid(const float* points, const void* labels, int64_t n, int32_t d,
                          const float* cell_widths, const int64_t* splits, int32_t table,
                          void* stream, ghn_index** out);

/*
 * knn_measure_cells: the paper's cell measurement (Sec. III.A).  For each
 * dimension, the largest number s of equal splits of the range of values
 * [min, max] such that every split holds a training point, and the split
 * width w = (max - min) / s in single precision.  A point's split is its
 * Eq. 1 coordinate with width w, the last split closed (coordinates clamped
 * to s - 1).  s is at most 2^21 (finer splits than single precision resolves
 * over a range); a dimension with one value gets s = 1, w = 1.
 *   points   host or device, n*d float32.
 *   splits   host, d int64; cell_widths host, d float32 (receive the result).
 * Synchronizes `stream`.  KNN_EINVAL for bad arguments or a non-finite value.
 */
knn_status knn_measure_cells(const float* points, int64_t n, int32_t d, int64_t* splits,
                             float* cell_widths, void* stream);

/* The widths and split counts an index was built with (host, d entries each;
 * splits are 0 for a grid without them).  Either pointer may be NULL. */
knn_status knn_index_grid(const ghn_index* index, float* cell_widths, int64_t* splits);

/*
 * knn_query: exploration and prediction (Sec. III.B, Algorithm 2; Sec. I).
 *   index    from knn_build.
 *   queries  host or device, m*d float32, row-major.
 *   m        0 <= m < 2^31 (0 is a no-op; KNN_EINVAL beyond).
 *   k        1 <= k <= 64.
 *   mode     KNN_NONE / KNN_VOTE / KNN_MEAN / KNN_MEDIAN (all but NONE need
 *            labels).
 *   ids      host or device, m*k int32: training indices, nearest first.
 *   dist2    host or device, m*k float32 squared distances (may be NULL).
 *   pred     host or device, m int32 (VOTE) or float32 (MEAN, MEDIAN), or
 *            NULL; NaN for MEAN / MEDIAN when no neighbour was found.
 *   flags    KNN_QUERY_CHECKED | KNN_QUERY_SORTED | KNN_QUERY_EXACT.
 *   stream   cudaStream_t or NULL.
 * Device outputs are written asynchronously on `stream`; host outputs are
 * filled before the call returns.  Pinned host outputs (page-locked memory the
 * GPU can address, e.g. over NVLink-C2C) are written by the kernels directly;
 * other host outputs are staged in device memory and copied out.  A query
 * with a non-finite coordinate gets -1 / +inf rows (KNN_EINVAL under
 * KNN_QUERY_CHECKED).
 * Work bound: a query that would enumerate more than 2^22 cell rows over the
 * layers it visits (the rows of cube(L) clipped to the box of occupied cells,
 * summed over L) stops there with -1 / +inf rows (KNN_ELIMIT under
 * KNN_QUERY_CHECKED).  Only grids far finer than the k-th neighbour distance
 * reach it (their walks need hundreds of layers); it keeps such a call from
 * running for minutes.  The environment variable GHN_MAX_ROWS replaces the
 * bound (0 or negative: none), and GHN_MAX_LAYERS adds a cap on the layers
 * visited from the first one that reaches the box (0 or unset: none).  The
 * bound and the cap apply to every query entry point of this library (batches,
 * the server and knn_query_noalloc included).
 */
knn_status knn_query(const ghn_index* index, const float* queries, int64_t m, int32_t k,
                     int32_t mode, int32_t* ids, float* dist2, void* pred, int32_t flags,
                     void* stream);

/*
 * knn_query_stats: the same walk with every cell of every visited layer
 * looked up (no geometric skipping), reporting per query the work the method
 * defines (Sec. III.C: exploration depth and points processed).
 *   ids, dist2  as knn_query (device or host; dist2 may be NULL).
 *   stats       host or device, m*3 int64: {layers visited (L* + 1),
 *               occupied cells looked up, training points examined}.
 * Synchronizes `stream` and returns the kernel's status.
 */
knn_status knn_query_stats(const ghn_index* index, const float* queries, int64_t m, int32_t k,
                           int32_t* ids, float* dist2, int64_t* stats, void* stream);

/*
 * knn_query_noalloc: knn_query for callers that cannot allocate device memory
 * while they query (an allocator that already holds the GPU's memory, a loop
 * that must not pay an allocation's latency or synchronisation, rules that
 * forbid allocation after start-up).  The paper has no counterpart: this is
 * a deployment variant of the same query kernels.
 *   Same arguments and results as knn_query, except:
 *   - queries, ids, dist2 and pred must be device memory (KNN_EINVAL if not);
 *   - 0 <= m <= 1048576 (KNN_EINVAL beyond);
 *   - flags: KNN_QUERY_CHECKED and KNN_QUERY_EXACT only (the locality order
 *     needs sort buffers).
 * The kernels' scratch lives in a fixed device array of the library (about
 * 4 MiB, held by every GPU that loads the library until exit).  The first call
 * on a device looks up that array's address, with the index's device current;
 * make that first call before any stream capture.  The address is kept for the
 * life of the process: a cudaDeviceReset in between invalidates it (and every
 * index on that device), so do not use the library across a device reset.
 * Queries, ids, dist2 and pred must be device memory of the index's GPU
 * (KNN_EINVAL otherwise).  All calls share the array:
 * calls whose work overlaps on the GPU race on it and must be ordered (one
 * stream, or synchronised).  No memory is allocated or freed by this call.
 */
knn_status knn_query_noalloc(const ghn_index* index, const float* queries, int64_t m, int32_t k,
                             int32_t mode, int32_t* ids, float* dist2, void* pred, int32_t flags,
                             void* stream);

/*
 * Batches of independent indexes (many small and large problems at once).
 * Each index of a batch is the method of knn_build / knn_query on its own
 * points with its own cell width (Sec. III.A-B); the batch builds all of them
 * in one pass over their points (one host synchronisation for all boxes) and
 * queries all of them in one persistent launch per dimension.  Results equal
 * those of knn_build + knn_query on each index.
 */
typedef struct ghn_batch ghn_batch; /* opaque; owns the device memory of its indexes */
typedef struct ghn_plan ghn_plan;   /* a captured batch query (CUDA graph) */

/*
 * knn_batch_build: build `count` indexes (1 <= count <= 65536).
 *   points[i]      host or device, n[i]*d[i] float32, row-major.
 *   labels         NULL, or an array whose entry i points to n[i] 32-bit
 *                  outputs (host or device), or is NULL for index i.
 *   Host inputs are copied into one device buffer.  Points are copied on
 *   `stream`; labels in pinned host memory on a library-owned side stream,
 *   once the boxes are read back, while the build's kernels run (`stream`
 *   waits for them before it reads them).  The call returns once every host
 *   input has been read, so the caller may reuse those buffers then.
 *   n, d, cell_width, table   host arrays of count entries, as in knn_build
 *                  (table may be NULL: KNN_TABLE_AUTO for every index).
 * The total number of points must be below 2^31.  Errors as knn_build, and
 * KNN_EINVAL when the cell ids of the batch need more than 63 bits.
 */
knn_status knn_batch_build(int32_t count, const float* const* points, const void* const* labels,
                           const int64_t* n, const int32_t* d, const float* cell_width,
                           const int32_t* table, void* stream, ghn_batch** out);

/* Shape of index i of the batch (table_slots: dense entries, 0 for hash). */
knn_status knn_batch_info(const ghn_batch* batch, int32_t i, knn_index_info_t* info);

/*
 * knn_batch_query: query every index of the batch (host arrays of count
 * entries; m[i] may be 0; the sum of the m[i] must be below 2^32).  Outputs
 * of index i as knn_query's.  flags: KNN_QUERY_CHECKED, KNN_QUERY_EXACT.
 * Data pointers are host or device memory, as for knn_query: host queries
 * are copied into one device buffer (when every host query array is pinned,
 * on a library-owned side stream that starts at once, so that the copies
 * overlap work already queued on `stream`, which waits for them; the call
 * returns once every host query has been read, so the caller may reuse
 * those buffers then); outputs in pinned host memory are written by the
 * kernels directly, other host outputs are staged on the device and copied
 * out; host outputs are complete when the call returns.
 * With knn_timing_enable on, the call records its phases (stage, one per
 * kernel group "query.d<d>.<k32|k64>.<dense|hash>", copy); knn_batch_build
 * records stage, box, keys, sort, cells, table, gather.
 */
knn_status knn_batch_query(const ghn_batch* batch, const float* const* queries, const int64_t* m,
                           const int32_t* k, const int32_t* mode, int32_t* const* ids,
                           float* const* dist2, void* const* pred, int32_t flags, void* stream);

/*
 * knn_batch_plan / knn_batch_run: the same query captured once in a CUDA
 * graph (the buffers are fixed at plan time and must be device memory) and
 * replayed by each run.
 * A plan must be freed before its batch.  knn_batch_run flags:
 * KNN_QUERY_CHECKED (synchronize and return the status) or 0.
 */
knn_status knn_batch_plan(const ghn_batch* batch, const float* const* queries, const int64_t* m,
                          const int32_t* k, const int32_t* mode, int32_t* const* ids,
                          float* const* dist2, void* const* pred, ghn_plan** out);
knn_status knn_batch_run(ghn_plan* plan, int32_t flags, void* stream);
void knn_plan_free(ghn_plan* plan);   /* NULL-safe */
void knn_batch_free(ghn_batch* batch); /* NULL-safe; waits for work that uses it */

/* Shape of the index.  Synchronizes the index's build stream on first use. */
knn_status knn_index_info(const ghn_index* index, knn_index_info_t* info);

/*
 * knn_index_export: the grid as built, for inspection and tests.
 *   cell_keys   host, num_cells uint64: linear cell ids, ascending; the id of
 *               cell c is sum_j c_j * prod_{i>j} extent_i.
 *   cell_start  host, num_cells + 1 uint32: first stored row of each cell.
 *   rows        host, n int32: training index of each stored row (cell order,
 *               ascending index inside a cell).
 * Any pointer may be NULL.  Synchronizes the device.
 */
knn_status knn_index_export(const ghn_index* index, uint64_t* cell_keys, uint32_t* cell_start,
                            int32_t* rows);

/*
 * Phase timing, for profiling.  While enabled, knn_build and knn_query record
 * a CUDA event on the call's stream at each phase boundary (build: stage, box,
 * keys, sort, cells, table, gather; query: stage, order, search (the warp
 * kernel), coop (the cooperative kernel, when it runs), copy).
 * The calling thread keeps its last 32 calls (up to 40 phases each); enabling
 * clears them.
 * knn_timing_read takes the calling thread's oldest unread call, waits for
 * its events, and writes up to `cap` phase names (static strings) and device
 * milliseconds; it returns the number of phases (0 when no call is unread).
 * Reading after a sequence of calls, rather than between them, adds no
 * synchronisation between the calls.
 */
knn_status knn_timing_enable(int32_t on);
int32_t knn_timing_read(const char** names, float* ms, int32_t cap);

/* Kernels this library has launched in this process (all threads). */
int64_t knn_kernel_launches(void);

/*
 * Deferral of heavy queries (a tuning choice; results do not depend on it).
 * The warp kernel walks a query with one warp; a query whose layer has more
 * than `heavy_rows` cell rows, or whose batch of 32 rows holds more than
 * `heavy_cands` points, is handed to the cooperative kernel, which walks it
 * with a block of 256 threads.  0 keeps the library default (1024 rows for
 * d <= 4, 4096 above; 8192 points; the environment variables GHN_HEAVY_ROWS
 * and GHN_HEAVY_CANDS replace these defaults), a negative value never defers
 * on that test, a positive value is the threshold.  knn_index_set_deferral
 * sets it for later queries of an index, knn_batch_set_deferral for index i
 * of a batch (later knn_batch_query and knn_batch_plan calls).
 */
knn_status knn_index_set_deferral(ghn_index* index, int64_t heavy_rows, int64_t heavy_cands);
knn_status knn_batch_set_deferral(ghn_batch* batch, int32_t i, int64_t heavy_rows,
                                  int64_t heavy_cands);

/* Release the index (NULL is a no-op).  Waits for work that uses it. */
void knn_free(ghn_index* index);

/* Message of the last failure on the calling thread ("" if none). */
const char* knn_last_error(void);

/* ABI version: 1. */
int32_t knn_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GHN_KNN_H */
