// Build-side launchers (build_kernels.cu): the index build of Sec. III.A,
// Eq. 1 and Algorithm 1 as a sequence of streaming kernels, and the keys of
// the queries' locality order.  Shared by the single build (capi.cu), the
// batched build (batch.cu) and the cell measurement (measure.cu).
#pragma once

#include "ghn_internal.cuh"

namespace ghn {

// A non-blocking stream per device for host-to-device copies that overlap
// work on the caller's stream (created on first use; capi.cu), or null.
cudaStream_t copy_stream(int dev);

// Box of the points: per-block partials, then one block computes the extents.
cudaError_t launch_box(const float* pts, long long n, int d, const Widths& w, float* partial,
                       int partial_blocks, BoxOut* out, cudaStream_t s);
int box_partial_blocks(long long n);

// Eq. 1 cell id of every training point (32-bit keys only when every id of
// the box fits).
cudaError_t launch_cell_keys(const float* pts, long long n, const GridConst& g,
                             unsigned long long* keys, cudaStream_t s);
cudaError_t launch_cell_keys(const float* pts, long long n, const GridConst& g, unsigned int* keys,
                             cudaStream_t s);

// LSD radix sort of (key, value) by the low `bits` bits of the key; stable.
// Returns in *result_keys / *result_vals the buffers that hold the sorted data.
// With identity_vals the values are taken to be 0..n-1 and vals_a is not read
// (it is still written, as one of the two value buffers).
size_t radix_temp_bytes(long long n);
cudaError_t radix_sort_pairs(unsigned long long* keys_a, unsigned int* vals_a,
                             unsigned long long* keys_b, unsigned int* vals_b, long long n,
                             int bits, void* temp, unsigned long long** result_keys,
                             unsigned int** result_vals, cudaStream_t s,
                             bool identity_vals = false);
cudaError_t radix_sort_pairs(unsigned int* keys_a, unsigned int* vals_a, unsigned int* keys_b,
                             unsigned int* vals_b, long long n, int bits, void* temp,
                             unsigned int** result_keys, unsigned int** result_vals,
                             cudaStream_t s, bool identity_vals = false);

// Exclusive prefix sum of n uint32 values (out may alias in).
size_t scan_temp_bytes(long long n);
cudaError_t scan_exclusive(const unsigned int* in, unsigned int* out, long long n, void* temp,
                           cudaStream_t s);

// Cells of n sorted keys: cell_key[c] / cell_start[c] for every cell c,
// cell_start[U] = n, and gdev->ncells / hmask.  scan_tmp: scan_temp_bytes(n).
cudaError_t launch_cells(const unsigned long long* sorted_keys, long long n, void* scan_tmp,
                         unsigned long long* cell_key, unsigned int* cell_start, GridDev* gdev,
                         cudaStream_t s);
cudaError_t launch_cells(const unsigned int* sorted_keys, long long n, void* scan_tmp,
                         unsigned long long* cell_key, unsigned int* cell_start, GridDev* gdev,
                         cudaStream_t s);

// Dense table: dstart[id] = first row of cell id, for every id of the box, and
// dstart[ncell_space] = n.  scan_tmp: scan_temp_bytes(ncell_space + 1).
cudaError_t launch_dense_table(const unsigned long long* cell_key, const unsigned int* cell_start,
                               const GridDev* gdev, unsigned long long ncell_space,
                               unsigned int* dstart, void* scan_tmp, cudaStream_t s);

cudaError_t launch_hash_table(const unsigned long long* cell_key, const unsigned int* cell_start,
                              const GridDev* gdev, HashSlot* slots, unsigned long long max_slots,
                              cudaStream_t s);

// Empty every slot of a table whose capacity the device computed (gdev->hmask + 1).
cudaError_t launch_hash_clear(HashSlot* slots, const GridDev* gdev, unsigned long long max_slots,
                              cudaStream_t s);

// Occupancy bitmap over the box (bit id set when cell id holds a point);
// `words` 32-bit words, zeroed here.
cudaError_t launch_bitmap(const unsigned long long* cell_key, const GridDev* gdev,
                          unsigned int* bitmap, unsigned long long words, cudaStream_t s);

cudaError_t launch_gather(const float* pts, long long n, int d, const unsigned int* order,
                          float* rows, cudaStream_t s);

// Small dense build (one block, shared memory): for n <= kSmallMaxN points in a
// box of at most kSmallMaxCells cells, the row ids, rows in cell order, dense
// table (space + 1 entries) and occupied-cell count, in one launch.
constexpr int kSmallMaxN = 16384;
constexpr unsigned long long kSmallMaxCells = 32767;
cudaError_t launch_small_build(const float* pts, long long n, int d, const GridConst& g,
                               unsigned long long space, unsigned int* rid, float* rows,
                               unsigned int* dstart, GridDev* gdev, cudaStream_t s);

// Query keys for the locality order: the cell id of each query, clamped into
// the box, shifted right by `shift` bits (the caller keeps it below 2^32).
cudaError_t launch_query_keys(const float* q, long long m, const GridConst& g, int shift,
                              unsigned int* keys, cudaStream_t s);

}  // namespace ghn
