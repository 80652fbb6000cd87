// Index build kernels: cell sampling (Sec. III.A, Eq. 1, Algorithm 1) on the GPU.
//
// Algorithm 1 appends every training point to the list of its cell in a
// dictionary keyed by the cell id.  Here the same grouping is a stable sort of
// the points by a linear cell id, followed by run-length cell offsets, a cell
// table (dense over the box of occupied cells, or open addressing over the
// occupied cells only: "no information about empty cells", Sec. III.A) and a
// gather of the point rows into cell order.  Stable sorting keeps the points
// of a cell in ascending training index, which is Algorithm 1's append order.
//
// Every kernel is a streaming pass bound by HBM bandwidth; none is a dense
// contraction, so tensor cores have no role here.

#include "build_launch.cuh"
#include "ghn_internal.cuh"

#include <math.h>

namespace ghn {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// Box of the training points: per-dimension min / max and a finiteness check.
// A block has 64*d threads and the grid stride is a multiple of d, so every
// thread always sees the same dimension (threadIdx.x % d) of the row-major
// array, and the loads of a warp are contiguous.
// ---------------------------------------------------------------------------
constexpr int kBoxUnroll = 8;

__global__ void box_partial_kernel(const float* __restrict__ pts, long long total, int d,
                                   float* __restrict__ partial)
{
    extern __shared__ float sm[];
    float* slo = sm;
    float* shi = sm + blockDim.x;
    __shared__ int sbad;
    const int t = threadIdx.x;
    if (t == 0) sbad = 0;
    float lo = INFINITY, hi = -INFINITY;
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long e = (long long)blockIdx.x * blockDim.x + t;
    // kBoxUnroll independent loads in flight per thread, all of one dimension
    for (; e + (kBoxUnroll - 1) * stride < total; e += kBoxUnroll * stride) {
        float v[kBoxUnroll];
#pragma unroll
        for (int r = 0; r < kBoxUnroll; ++r) v[r] = __ldg(pts + e + r * stride);
#pragma unroll
        for (int r = 0; r < kBoxUnroll; ++r) {
            bad |= !isfinite(v[r]);
            lo = fminf(lo, v[r]);
            hi = fmaxf(hi, v[r]);
        }
    }
    for (; e < total; e += stride) {
        const float v = __ldg(pts + e);
        bad |= !isfinite(v);
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    slo[t] = lo;
    shi[t] = hi;
    __syncthreads();
    if (bad) sbad = 1;
    if (t < d) {
        for (int u = t + d; u < (int)blockDim.x; u += d) {
            lo = fminf(lo, slo[u]);
            hi = fmaxf(hi, shi[u]);
        }
    }
    __syncthreads();
    float* out = partial + (size_t)blockIdx.x * (2 * d + 1);
    if (t < d) {
        out[t] = lo;
        out[d + t] = hi;
    }
    if (t == 0) out[2 * d] = sbad ? 1.0f : 0.0f;
}

// Reduce the partial boxes (one block: each thread folds a slice of the
// partials, then a tree over the block); compute the number of cells per
// dimension from the largest point: ext_j = floor((hi_j - lo_j) / w_j) + 1 (Eq. 1
// is monotone in the coordinate, so no training point has a larger cell),
// at most split_j when the grid clamps training cells into split_j splits.
constexpr int kBoxFinalThreads = 256;

__global__ void __launch_bounds__(kBoxFinalThreads)
    box_final_kernel(const float* __restrict__ partial, int nblocks, int d, const Widths w,
                     BoxOut* __restrict__ out)
{
    __shared__ float slo[kMaxD][kBoxFinalThreads];
    __shared__ float shi[kMaxD][kBoxFinalThreads];
    __shared__ int sbad;
    const int t = threadIdx.x;
    if (t == 0) sbad = 0;
    float lo[kMaxD], hi[kMaxD];
#pragma unroll
    for (int j = 0; j < kMaxD; ++j) {
        lo[j] = INFINITY;
        hi[j] = -INFINITY;
    }
    bool bad = false;
    for (int b = t; b < nblocks; b += kBoxFinalThreads) {
        const float* p = partial + (size_t)b * (2 * d + 1);
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) {
            if (j < d) {
                lo[j] = fminf(lo[j], p[j]);
                hi[j] = fmaxf(hi[j], p[d + j]);
            }
        }
        bad |= p[2 * d] != 0.0f;
    }
#pragma unroll
    for (int j = 0; j < kMaxD; ++j) {
        slo[j][t] = lo[j];
        shi[j][t] = hi[j];
    }
    __syncthreads();
    if (bad) sbad = 1;
    for (int half = kBoxFinalThreads / 2; half > 0; half >>= 1) {
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
        for (int j = 0; j < d; ++j) {
            const float l = slo[j][0], h = shi[j][0];
            out->lo[j] = l;
            out->hi[j] = h;
            long long ext = 0;
            if (sbad || !(l <= h)) {
                flags |= kStatusNonFinite;
            } else {
                const float q = __fdiv_rn(__fsub_rn(h, l), w.w[j]);
                if (!(q < 2147483647.0f))
                    flags |= kStatusExtent;
                else
                    ext = (long long)floorf(q) + 1;
                if (w.split[j] > 0 && ext > w.split[j]) ext = w.split[j];
            }
            out->ext[j] = ext;
        }
        out->flags = flags;
    }
}

// ---------------------------------------------------------------------------
// Eq. 1 for every training point: c_j = floor((p_j - o_j) / w_j) in single
// precision (subtract and divide rounded to nearest, as IEEE operations),
// clamped to split_j - 1 on a grid with splits, then the linear id
// sum_j c_j * stride_j; the value is the point's index.
// ---------------------------------------------------------------------------
constexpr int kKeyUnroll = 4;

template <int D, class K>
__global__ void cell_keys_kernel(const float* __restrict__ pts, long long n, GridConst g,
                                 K* __restrict__ keys)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    // kKeyUnroll points a thread per round, all of their loads issued first
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n;
         i0 += kKeyUnroll * stride) {
        float p[kKeyUnroll][D];
#pragma unroll
        for (int u = 0; u < kKeyUnroll; ++u) {
            const long long i = i0 + u * stride;
#pragma unroll
            for (int j = 0; j < D; ++j) p[u][j] = i < n ? __ldg(pts + i * D + j) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kKeyUnroll; ++u) {
            const long long i = i0 + u * stride;
            if (i >= n) break;
            unsigned long long key = 0;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const float t = __fdiv_rn(__fsub_rn(p[u][j], g.lo[j]), g.w[j]);
                long long c = (long long)floorf(t);
                if (g.split[j] > 0 && c > g.split[j] - 1) c = g.split[j] - 1;
                key += (unsigned long long)c * g.stride[j];
            }
            keys[i] = (K)key;  // 32-bit K only when every id of the box fits
        }
    }
}

// ---------------------------------------------------------------------------
// Vector forms of the box and of the cell keys, for 16-byte aligned points.
// A thread takes chunks of 4 points: that is D float4 loads whatever D is,
// and the dimension of every float is known at compile time.  Up to two
// chunks per round (d <= 4) keep 96 to 128 bytes in flight per thread.  The
// n mod 4 points after the last chunk are done one by one by block 0.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void load_chunk(const float* __restrict__ pts, long long c,
                                           float (&v)[4 * D])
{
    const float4* p = reinterpret_cast<const float4*>(pts) + c * D;
#pragma unroll
    for (int h = 0; h < D; ++h) {
        const float4 x = __ldg(p + h);
        v[4 * h] = x.x;
        v[4 * h + 1] = x.y;
        v[4 * h + 2] = x.z;
        v[4 * h + 3] = x.w;
    }
}

template <int D>
struct VecRounds {
    static constexpr int value = D <= 4 ? 2 : 1;
};

constexpr int kVecThreads = 256;

template <int D>
__global__ void __launch_bounds__(kVecThreads)
    box_partial_vec_kernel(const float* __restrict__ pts, long long n, float* __restrict__ partial)
{
    constexpr int U = VecRounds<D>::value;
    constexpr int W = kVecThreads / 32;
    __shared__ float wlo[W][D], whi[W][D];
    __shared__ int wbad[W];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float lo[D], hi[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        lo[j] = INFINITY;
        hi[j] = -INFINITY;
    }
    bool bad = false;
    const long long chunks = n / 4;
    const long long stride = (long long)gridDim.x * kVecThreads;
    for (long long c0 = (long long)blockIdx.x * kVecThreads + t; c0 < chunks; c0 += U * stride) {
        float v[U][4 * D];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (c0 + u * stride < chunks) load_chunk<D>(pts, c0 + u * stride, v[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (c0 + u * stride >= chunks) break;
#pragma unroll
            for (int f = 0; f < 4 * D; ++f) {
                bad |= !isfinite(v[u][f]);
                lo[f % D] = fminf(lo[f % D], v[u][f]);
                hi[f % D] = fmaxf(hi[f % D], v[u][f]);
            }
        }
    }
    if (blockIdx.x == 0) {
        for (long long i = 4 * chunks + t; i < n; i += kVecThreads) {
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const float x = __ldg(pts + i * D + j);
                bad |= !isfinite(x);
                lo[j] = fminf(lo[j], x);
                hi[j] = fmaxf(hi[j], x);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[j] = fminf(lo[j], __shfl_xor_sync(FULL, lo[j], o));
            hi[j] = fmaxf(hi[j], __shfl_xor_sync(FULL, hi[j], o));
        }
    }
    bad = __any_sync(FULL, bad);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            wlo[warp][j] = lo[j];
            whi[warp][j] = hi[j];
        }
        wbad[warp] = bad ? 1 : 0;
    }
    __syncthreads();
    if (t < D) {
        float l = wlo[0][t], h = whi[0][t];
        for (int w = 1; w < W; ++w) {
            l = fminf(l, wlo[w][t]);
            h = fmaxf(h, whi[w][t]);
        }
        float* out = partial + (size_t)blockIdx.x * (2 * D + 1);
        out[t] = l;
        out[D + t] = h;
    }
    if (t == 0) {
        int b = 0;
        for (int w = 0; w < W; ++w) b |= wbad[w];
        partial[(size_t)blockIdx.x * (2 * D + 1) + 2 * D] = b ? 1.0f : 0.0f;
    }
}

// Eq. 1 for one coordinate of a training point, as in cell_keys_kernel.
__device__ __forceinline__ unsigned long long key_part(float p, const GridConst& g, int j)
{
    const float t = __fdiv_rn(__fsub_rn(p, g.lo[j]), g.w[j]);
    long long c = (long long)floorf(t);
    if (g.split[j] > 0 && c > g.split[j] - 1) c = g.split[j] - 1;
    return (unsigned long long)c * g.stride[j];
}

__device__ __forceinline__ void store4(unsigned int* keys, long long c, const unsigned long long (&k)[4])
{
    reinterpret_cast<uint4*>(keys)[c] =
        make_uint4((unsigned)k[0], (unsigned)k[1], (unsigned)k[2], (unsigned)k[3]);
}
__device__ __forceinline__ void store4(unsigned long long* keys, long long c,
                                       const unsigned long long (&k)[4])
{
    ulonglong2* p = reinterpret_cast<ulonglong2*>(keys) + 2 * c;
    p[0] = make_ulonglong2(k[0], k[1]);
    p[1] = make_ulonglong2(k[2], k[3]);
}

template <int D, class K>
__global__ void __launch_bounds__(kVecThreads)
    cell_keys_vec_kernel(const float* __restrict__ pts, long long n, GridConst g,
                         K* __restrict__ keys)
{
    constexpr int U = VecRounds<D>::value;
    const long long chunks = n / 4;
    const long long stride = (long long)gridDim.x * kVecThreads;
    for (long long c0 = (long long)blockIdx.x * kVecThreads + threadIdx.x; c0 < chunks;
         c0 += U * stride) {
        float v[U][4 * D];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (c0 + u * stride < chunks) load_chunk<D>(pts, c0 + u * stride, v[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (c0 + u * stride >= chunks) break;
            unsigned long long k[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
            for (int f = 0; f < 4 * D; ++f) k[f / D] += key_part(v[u][f], g, f % D);
            store4(keys, c0 + u * stride, k);  // 32-bit K only when every id fits
        }
    }
    if (blockIdx.x == 0) {
        for (long long i = 4 * chunks + threadIdx.x; i < n; i += kVecThreads) {
            unsigned long long key = 0ull;
#pragma unroll
            for (int j = 0; j < D; ++j) key += key_part(__ldg(pts + i * D + j), g, j);
            keys[i] = (K)key;
        }
    }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8- or 9-bit digits (256 or 512 buckets), 2048-element
// tiles (256 threads x 8), of 64-bit keys or, when every key fits, 32-bit ones
// (20 bytes a pass per element instead of 32).  Per pass: a digit histogram per tile, an exclusive
// scan of the digit-major histogram table, and a scatter that ranks each tile
// stably in shared memory and writes it out in digit runs.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadixMax = 512;

// Lanes of the warp whose digit (BITS bits) equals this lane's, among the
// lanes in `valid`: one ballot per digit bit.
template <int BITS>
__device__ __forceinline__ unsigned match_digit(unsigned d, unsigned valid)
{
    unsigned m = valid;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned bal = __ballot_sync(FULL, bit);
        m &= bit ? bal : ~bal;
    }
    return m;
}
template <int R>
struct DigitBits {
    static constexpr int value = R == 512 ? 9 : 8;
};

template <class K, int R>
__global__ void __launch_bounds__(kSortThreads)
    radix_hist_kernel(const K* __restrict__ keys, long long n, int shift,
                      unsigned int* __restrict__ hist, unsigned int nb)
{
    constexpr int W = kSortThreads / 32;
    __shared__ unsigned int cnt[W][R];  // one histogram per warp
    const int t = threadIdx.x, warp = t >> 5;
    for (int e = t; e < W * R; e += kSortThreads) (&cnt[0][0])[e] = 0u;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
    K kv[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const long long i = base + r * kSortThreads + t;
        kv[r] = i < n ? keys[i] : (K)0;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const long long i = base + r * kSortThreads + t;
        if (i < n) atomicAdd(&cnt[warp][(unsigned)((kv[r] >> shift) & (K)(R - 1))], 1u);
    }
    __syncthreads();
    for (int e = t; e < R; e += kSortThreads) {
        unsigned int c = 0u;
#pragma unroll
        for (int w = 0; w < W; ++w) c += cnt[w][e];
        hist[(size_t)e * nb + blockIdx.x] = c;
    }
}

template <class K, int R>
__global__ void __launch_bounds__(kSortThreads, (sizeof(K) == 4 ? 5 : 4))
    radix_scatter_kernel(const K* __restrict__ kin, const unsigned int* __restrict__ vin,
                         K* __restrict__ kout, unsigned int* __restrict__ vout,
                         long long n, int shift, const unsigned int* __restrict__ scanned,
                         unsigned int nb)
{
    constexpr int W = kSortThreads / 32;
    constexpr int DPT = R / kSortThreads;  // digits per thread in the digit scan
    constexpr K MASK = (K)(R - 1);
    __shared__ unsigned int wcnt[W][R];
    __shared__ unsigned int dig_off[R];
    __shared__ unsigned int gbase[R];
    __shared__ unsigned int wsum[W];
    __shared__ K skey[kSortTile];
    __shared__ unsigned int sval[kSortTile];

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // this thread's digits' global bases, loaded now and stored after the
    // ranking so that their latency overlaps it
    unsigned int gb[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) gb[q] = scanned[(size_t)(t * DPT + q) * nb + blockIdx.x];
    for (int e = t; e < W * R; e += kSortThreads) (&wcnt[0][0])[e] = 0u;

    const long long tile = (long long)blockIdx.x * kSortTile;
    const long long count = n - tile < kSortTile ? n - tile : kSortTile;
    K k[kSortItems];
    unsigned int v[kSortItems], rank[kSortItems], dg[kSortItems];
    // warp `warp` ranks elements [warp*256, warp*256+256) of the tile, in
    // order; all of its loads are issued first
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int local = warp * (32 * kSortItems) + r * 32 + lane;
        const bool valid = local < count;
        k[r] = valid ? kin[tile + local] : (K)0;
        v[r] = valid ? (vin ? vin[tile + local] : (unsigned int)(tile + local)) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int local = warp * (32 * kSortItems) + r * 32 + lane;
        const bool valid = local < count;
        const unsigned d = valid ? (unsigned)((k[r] >> shift) & MASK) : R + lane;
        const unsigned peers =
            match_digit<DigitBits<R>::value>(d & (unsigned)(R - 1), __ballot_sync(FULL, valid));
        const unsigned before = __popc(peers & lanemask_lt());
        unsigned int b = 0u;
        if (valid) b = wcnt[warp][d];
        __syncwarp();
        if (valid && before == 0u) wcnt[warp][d] = b + __popc(peers);
        __syncwarp();
        rank[r] = b + before;
        dg[r] = d;
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, and the tile's total; thread t
    // owns the consecutive digits t*DPT .. t*DPT + DPT - 1
    unsigned int run[DPT];
    unsigned int mine = 0u;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int e = t * DPT + q;
        unsigned int acc = 0u;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const unsigned int c = wcnt[w][e];
            wcnt[w][e] = acc;
            acc += c;
        }
        run[q] = acc;
        mine += acc;
    }
    // exclusive scan of the digit totals over the threads
    unsigned int x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    unsigned int wpre = 0u;
    for (int w = 0; w < warp; ++w) wpre += wsum[w];
    unsigned int off = wpre + x - mine;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        dig_off[t * DPT + q] = off;
        gbase[t * DPT + q] = gb[q];
        off += run[q];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (dg[r] < (unsigned)R) {
            const unsigned int p = dig_off[dg[r]] + wcnt[warp][dg[r]] + rank[r];
            skey[p] = k[r];
            sval[p] = v[r];
        }
    }
    __syncthreads();
    for (int i = t; i < count; i += kSortThreads) {
        const K key = skey[i];
        const unsigned d = (unsigned)((key >> shift) & MASK);
        const unsigned int g = gbase[d] + (unsigned int)i - dig_off[d];
        kout[g] = key;
        vout[g] = sval[i];
    }
}

// vals[i] = i: the values of a sort whose first pass did not run.
__global__ void iota_kernel(unsigned int* __restrict__ vals, long long n)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        vals[i] = (unsigned int)i;
}

// ---------------------------------------------------------------------------
// Exclusive prefix sum of uint32: reduce per 1024-element block, scan the
// block sums in one block, then scan each block and add its offset.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

// Inclusive block scan of one value per thread; returns the inclusive value
// and writes the block total to *total.
__device__ __forceinline__ unsigned int block_scan_incl(unsigned int x, unsigned int* wsum,
                                                        unsigned int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned int s = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) wsum[lane] = s;
    }
    __syncthreads();
    const unsigned int pre = warp > 0 ? wsum[warp - 1] : 0u;
    *total = wsum[nw - 1];
    __syncthreads();
    return x + pre;
}

__global__ void __launch_bounds__(kScanThreads)
    scan_reduce_kernel(const unsigned int* __restrict__ in, long long n,
                       unsigned int* __restrict__ sums)
{
    __shared__ unsigned int wsum[32];
    const long long base = (long long)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
    unsigned int s = 0u;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r)
        if (base + r < n) s += in[base + r];
    unsigned int total;
    block_scan_incl(s, wsum, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_spine_kernel(unsigned int* __restrict__ sums,
                                                          long long nb)
{
    __shared__ unsigned int wsum[32];
    unsigned int carry = 0u;
    for (long long base = 0; base < nb; base += blockDim.x) {
        const long long i = base + threadIdx.x;
        const unsigned int x = i < nb ? sums[i] : 0u;
        unsigned int total;
        const unsigned int incl = block_scan_incl(x, wsum, &total);
        if (i < nb) sums[i] = carry + incl - x;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads)
    scan_down_kernel(const unsigned int* in, unsigned int* out, long long n,
                     const unsigned int* __restrict__ sums)
{
    __shared__ unsigned int wsum[32];
    const long long base = (long long)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
    unsigned int v[kScanItems];
    unsigned int s = 0u;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        v[r] = base + r < n ? in[base + r] : 0u;
        s += v[r];
    }
    unsigned int total;
    unsigned int run = block_scan_incl(s, wsum, &total) - s + sums[blockIdx.x];
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        if (base + r < n) out[base + r] = run;
        run += v[r];
    }
}

// ---------------------------------------------------------------------------
// Cells: a head where the sorted id changes (and at row 0); the exclusive
// scan of the heads numbers the cells, and each head writes its cell's id and
// first row.  Both passes of the scan (per-block head counts, then the
// scan proper) recompute the heads from the sorted keys, so no flag or cell
// index array is written.  Blocks of kScanBlock rows, kScanItems consecutive
// rows a thread.
// ---------------------------------------------------------------------------
template <class K>
__device__ __forceinline__ unsigned int heads_of(const K* __restrict__ keys, long long n,
                                                 long long base, K (&kv)[kScanItems],
                                                 unsigned int (&head)[kScanItems])
{
    K prev = base > 0 && base <= n ? keys[base - 1] : (K)0;
    unsigned int cnt = 0u;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) kv[r] = base + r < n ? keys[base + r] : (K)0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const long long i = base + r;
        head[r] = i < n && (i == 0 || kv[r] != prev) ? 1u : 0u;
        prev = kv[r];
        cnt += head[r];
    }
    return cnt;
}

template <class K>
__global__ void __launch_bounds__(kScanThreads)
    cells_count_kernel(const K* __restrict__ keys, long long n, unsigned int* __restrict__ sums)
{
    __shared__ unsigned int wsum[32];
    const long long base = (long long)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
    K kv[kScanItems];
    unsigned int head[kScanItems];
    const unsigned int cnt = heads_of(keys, n, base, kv, head);
    unsigned int total;
    block_scan_incl(cnt, wsum, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <class K>
__global__ void __launch_bounds__(kScanThreads)
    cells_write_kernel(const K* __restrict__ keys, long long n,
                       const unsigned int* __restrict__ sums,
                       unsigned long long* __restrict__ cell_key,
                       unsigned int* __restrict__ cell_start, GridDev* gdev)
{
    __shared__ unsigned int wsum[32];
    const long long base = (long long)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
    K kv[kScanItems];
    unsigned int head[kScanItems];
    const unsigned int cnt = heads_of(keys, n, base, kv, head);
    unsigned int total;
    // the first cell this thread's rows open
    unsigned int c = block_scan_incl(cnt, wsum, &total) - cnt + sums[blockIdx.x];
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const long long i = base + r;
        if (head[r]) {
            cell_key[c] = (unsigned long long)kv[r];
            cell_start[c] = (unsigned int)i;
            ++c;
        }
        if (i == n - 1) {
            // c is now the number of cells
            cell_start[c] = (unsigned int)n;
            unsigned long long cap = 16ull;
            while (cap < 2ull * c) cap <<= 1;
            gdev->ncells = c;
            gdev->hmask = cap - 1ull;
        }
    }
}

// Dense table: the row count of every occupied cell at its linear id, zeros
// elsewhere; an exclusive scan of that array gives each cell's first row.
__global__ void dense_counts_kernel(const unsigned long long* __restrict__ cell_key,
                                    const unsigned int* __restrict__ cell_start,
                                    const GridDev* __restrict__ gdev,
                                    unsigned int* __restrict__ dstart)
{
    const unsigned long long u = gdev->ncells;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < (long long)u;
         c += stride)
        dstart[cell_key[c]] = cell_start[c + 1] - cell_start[c];
}

// Open addressing with linear probing over a power-of-two table at most half
// full, so every insert finds an empty slot.
__global__ void hash_clear_kernel(HashSlot* __restrict__ slots, const GridDev* __restrict__ gdev)
{
    const unsigned long long cap = gdev->hmask + 1ull;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < (long long)cap;
         s += stride) {
        HashSlot e;
        e.key = kEmptyKey;
        e.start = 0u;
        e.end = 0u;
        slots[s] = e;
    }
}

__global__ void hash_insert_kernel(const unsigned long long* __restrict__ cell_key,
                                   const unsigned int* __restrict__ cell_start,
                                   const GridDev* __restrict__ gdev, HashSlot* slots)
{
    const unsigned long long u = gdev->ncells, mask = gdev->hmask;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < (long long)u;
         c += stride) {
        const unsigned long long key = cell_key[c];
        unsigned long long h = mix64(key) & mask;
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            const unsigned long long prev = atomicCAS(&slots[h].key, kEmptyKey, key);
            if (prev == kEmptyKey) {
                slots[h].start = cell_start[c];
                slots[h].end = cell_start[c + 1];
                break;
            }
            h = (h + 1ull) & mask;
        }
    }
}

// Occupancy bitmap: one bit per linear cell id of the box.
__global__ void bitmap_kernel(const unsigned long long* __restrict__ cell_key,
                              const GridDev* __restrict__ gdev, unsigned int* __restrict__ bm)
{
    const unsigned long long u = gdev->ncells;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < (long long)u;
         c += stride) {
        const unsigned long long id = cell_key[c];
        atomicOr(bm + (id >> 5), 1u << (unsigned)(id & 31ull));
    }
}

// ---------------------------------------------------------------------------
// Gather the point rows into cell order, padded to 2, 4 or 8 floats so that a
// row is one 8-, 16- or two 16-byte loads in the query kernel.
// ---------------------------------------------------------------------------
template <int D>
__global__ void gather_kernel(const float* __restrict__ pts, long long n,
                              const unsigned int* __restrict__ order, float* __restrict__ rows)
{
    constexpr int P = row_floats(D);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const long long i = order[r];
        float v[P];
#pragma unroll
        for (int j = 0; j < P; ++j) v[j] = j < D ? __ldg(pts + i * D + j) : 0.0f;
        if constexpr (P == 2) {
            reinterpret_cast<float2*>(rows)[r] = make_float2(v[0], v[1]);
        } else {
#pragma unroll
            for (int h = 0; h < P / 4; ++h)
                reinterpret_cast<float4*>(rows)[r * (P / 4) + h] =
                    make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
        }
    }
}

// ---------------------------------------------------------------------------
// Small dense build: one block of 1024 threads builds a whole index of at most
// kSmallMaxN points whose box holds at most kSmallMaxCells cells (ids fit 16
// bits), with everything between the box and the outputs in shared memory:
//   - Eq. 1 ids of every point (the arithmetic of cell_keys_kernel);
//   - a stable LSD radix sort of (id, index) by id, 8-bit digits, one or two
//     passes.  Warp w ranks the 512 consecutive points w*512 .. w*512+511 in
//     index order (item j of lane l is point w*512 + 32j + l); a digit-major,
//     warp-minor scan of the warps' digit counts then places every point, so
//     points of one cell keep ascending index, as the multi-kernel sort does;
//   - the training index of every row, the rows gathered in cell order, the
//     dense table (each cell's first row: the number of rows with a smaller
//     id, by binary search) and the occupied-cell count.
// The result is the same index as the multi-kernel path builds.
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 1024;
constexpr int kSmallItems = kSmallMaxN / kSmallThreads;  // points a lane ranks per pass
static_assert(kSmallMaxN % kSmallThreads == 0, "whole items per lane");

struct SmallSmem {
    unsigned short key[2][kSmallMaxN];
    unsigned short idx[2][kSmallMaxN];
    unsigned int cnt[32][256];  // per warp and digit: counts, then first positions
    unsigned int wsum[32];
    unsigned int total;
};

size_t small_build_smem_bytes() { return sizeof(SmallSmem); }

template <int D>
__global__ void __launch_bounds__(kSmallThreads, 1)
    small_build_kernel(const float* __restrict__ pts, int n, GridConst g, unsigned int space,
                       unsigned int* __restrict__ rid, float* __restrict__ rows,
                       unsigned int* __restrict__ dstart, GridDev* __restrict__ gdev)
{
    extern __shared__ __align__(16) unsigned char small_raw[];
    SmallSmem& sm = *reinterpret_cast<SmallSmem*>(small_raw);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const unsigned int lt = (1u << lane) - 1u;
    constexpr int P = row_floats(D);
    // ---- Eq. 1 ids ----
#pragma unroll 4
    for (int j = 0; j < kSmallItems; ++j) {
        const int e = w * (32 * kSmallItems) + j * 32 + lane;
        if (e < n) {
            unsigned long long key = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const float tq =
                    __fdiv_rn(__fsub_rn(__ldg(pts + (long long)e * D + c), g.lo[c]), g.w[c]);
                long long cc = (long long)floorf(tq);
                if (g.split[c] > 0 && cc > g.split[c] - 1) cc = g.split[c] - 1;
                key += (unsigned long long)cc * g.stride[c];
            }
            sm.key[0][e] = (unsigned short)key;
            sm.idx[0][e] = (unsigned short)e;
        }
    }
    __syncthreads();
    // ---- stable radix sort by id ----
    const int passes = space <= 256u ? 1 : 2;
    int cur = 0;
    for (int pass = 0; pass < passes; ++pass) {
        const int sh = 8 * pass;
        for (int i = t; i < 32 * 256; i += kSmallThreads) (&sm.cnt[0][0])[i] = 0u;
        __syncthreads();
        unsigned int rd[kSmallItems];  // digit << 16 | rank within the warp (rank < 2^14)
#pragma unroll
        for (int j = 0; j < kSmallItems; ++j) {
            const int e = w * (32 * kSmallItems) + j * 32 + lane;
            const bool valid = e < n;
            const unsigned int d = valid ? ((unsigned int)sm.key[cur][e] >> sh) & 255u : 0u;
            // the lanes with the same digit (and validity): one ballot per bit
            unsigned int peers = __ballot_sync(FULL, valid);
            if (!valid) peers = ~peers;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const bool bit = (d >> b) & 1u;
                const unsigned int m = __ballot_sync(FULL, bit);
                peers &= bit ? m : ~m;
            }
            const unsigned int base = valid ? sm.cnt[w][d] : 0u;
            __syncwarp();
            if (valid && (peers & lt) == 0u) sm.cnt[w][d] = base + (unsigned int)__popc(peers);
            __syncwarp();
            rd[j] = (d << 16) | (base + (unsigned int)__popc(peers & lt));
        }
        __syncthreads();
        {
            // thread t owns digit t / 4 and warps 8 (t % 4) .. 8 (t % 4) + 7
            const int d = t >> 2, w0 = (t & 3) * 8;
            unsigned int sum = 0u;
#pragma unroll
            for (int i = 0; i < 8; ++i) sum += sm.cnt[w0 + i][d];
            unsigned int tot;
            unsigned int pre = block_scan_incl(sum, sm.wsum, &tot) - sum;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const unsigned int v = sm.cnt[w0 + i][d];
                sm.cnt[w0 + i][d] = pre;
                pre += v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSmallItems; ++j) {
            const int e = w * (32 * kSmallItems) + j * 32 + lane;
            if (e < n) {
                const unsigned int dst = sm.cnt[w][rd[j] >> 16] + (rd[j] & 0xffffu);
                sm.key[cur ^ 1][dst] = sm.key[cur][e];
                sm.idx[cur ^ 1][dst] = sm.idx[cur][e];
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    const unsigned short* sk = sm.key[cur];
    const unsigned short* si = sm.idx[cur];
    // ---- rows in cell order, their training indices, occupied cells ----
    unsigned int heads = 0u;
    for (int r = t; r < n; r += kSmallThreads) {
        const int i = si[r];
        rid[r] = (unsigned int)i;
        float v[P];
#pragma unroll
        for (int c = 0; c < P; ++c) v[c] = c < D ? __ldg(pts + (long long)i * D + c) : 0.0f;
        if constexpr (P == 2) {
            reinterpret_cast<float2*>(rows)[r] = make_float2(v[0], v[1]);
        } else {
#pragma unroll
            for (int h = 0; h < P / 4; ++h)
                reinterpret_cast<float4*>(rows)[r * (P / 4) + h] =
                    make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
        }
        heads += (r == 0 || sk[r] != sk[r - 1]) ? 1u : 0u;
    }
    // ---- dense table: the first row of cell c is the count of smaller ids ----
    for (unsigned int c = (unsigned int)t; c <= space; c += kSmallThreads) {
        int lo = 0, hi = n;  // first row whose id is >= c
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((unsigned int)sk[mid] < c)
                lo = mid + 1;
            else
                hi = mid;
        }
        dstart[c] = (unsigned int)lo;
    }
    unsigned int u;
    block_scan_incl(heads, sm.wsum, &u);
    if (t == 0) {
        unsigned long long cap = 16ull;
        while (cap < 2ull * u) cap <<= 1;
        gdev->ncells = u;
        gdev->hmask = cap - 1ull;
    }
}

// Cell id of each query clamped into the box (for the locality order only).
template <int D, class K>
__global__ void query_keys_kernel(const float* __restrict__ q, long long m, GridConst g, int shift,
                                  K* __restrict__ keys)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        unsigned long long key = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float t = floorf(__fdiv_rn(__fsub_rn(__ldg(q + i * D + j), g.lo[j]), g.w[j]));
            t = fminf(fmaxf(t, 0.0f), (float)g.cmax[j]);  // NaN becomes 0
            long long c = (long long)t;
            if (c > g.cmax[j]) c = g.cmax[j];
            key += (unsigned long long)c * g.stride[j];
        }
        keys[i] = (K)(key >> shift);  // 32-bit K only when every shifted id fits
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0u; }

int grid_for(long long work, int threads)
{
    long long b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

int box_partial_blocks(long long n)
{
    long long b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 8) b = 152 * 8;
    return (int)b;
}

cudaError_t launch_box(const float* pts, long long n, int d, const Widths& w, float* partial,
                       int partial_blocks, BoxOut* out, cudaStream_t s)
{
    if (aligned16(pts)) {
        const int pb = partial_blocks;
        switch (d) {
        case 1: box_partial_vec_kernel<1><<<pb, kVecThreads, 0, s>>>(pts, n, partial); break;
        case 2: box_partial_vec_kernel<2><<<pb, kVecThreads, 0, s>>>(pts, n, partial); break;
        case 3: box_partial_vec_kernel<3><<<pb, kVecThreads, 0, s>>>(pts, n, partial); break;
        case 4: box_partial_vec_kernel<4><<<pb, kVecThreads, 0, s>>>(pts, n, partial); break;
        case 5: box_partial_vec_kernel<5><<<pb, kVecThreads, 0, s>>>(pts, n, partial); break;
        case 6: box_partial_vec_kernel<6><<<pb, kVecThreads, 0, s>>>(pts, n, partial); break;
        case 7: box_partial_vec_kernel<7><<<pb, kVecThreads, 0, s>>>(pts, n, partial); break;
        case 8: box_partial_vec_kernel<8><<<pb, kVecThreads, 0, s>>>(pts, n, partial); break;
        default: return cudaErrorInvalidValue;
        }
    } else {
        const int threads = 64 * d;
        box_partial_kernel<<<partial_blocks, threads, 2 * threads * sizeof(float), s>>>(
            pts, n * d, d, partial);
    }
    box_final_kernel<<<1, kBoxFinalThreads, 0, s>>>(partial, partial_blocks, d, w, out);
    count_launches(2);
    return cudaGetLastError();
}

namespace {
template <class K>
cudaError_t launch_cell_keys_t(const float* pts, long long n, const GridConst& g, K* keys,
                               cudaStream_t s)
{
    count_launches(1);
    if (aligned16(pts) && aligned16(keys)) {
        const int b = grid_for((n + 3) / 4, kVecThreads);
        switch (g.d) {
        case 1: cell_keys_vec_kernel<1, K><<<b, kVecThreads, 0, s>>>(pts, n, g, keys); break;
        case 2: cell_keys_vec_kernel<2, K><<<b, kVecThreads, 0, s>>>(pts, n, g, keys); break;
        case 3: cell_keys_vec_kernel<3, K><<<b, kVecThreads, 0, s>>>(pts, n, g, keys); break;
        case 4: cell_keys_vec_kernel<4, K><<<b, kVecThreads, 0, s>>>(pts, n, g, keys); break;
        case 5: cell_keys_vec_kernel<5, K><<<b, kVecThreads, 0, s>>>(pts, n, g, keys); break;
        case 6: cell_keys_vec_kernel<6, K><<<b, kVecThreads, 0, s>>>(pts, n, g, keys); break;
        case 7: cell_keys_vec_kernel<7, K><<<b, kVecThreads, 0, s>>>(pts, n, g, keys); break;
        case 8: cell_keys_vec_kernel<8, K><<<b, kVecThreads, 0, s>>>(pts, n, g, keys); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    const int b = grid_for(n, 256);
    switch (g.d) {
    case 1: cell_keys_kernel<1, K><<<b, 256, 0, s>>>(pts, n, g, keys); break;
    case 2: cell_keys_kernel<2, K><<<b, 256, 0, s>>>(pts, n, g, keys); break;
    case 3: cell_keys_kernel<3, K><<<b, 256, 0, s>>>(pts, n, g, keys); break;
    case 4: cell_keys_kernel<4, K><<<b, 256, 0, s>>>(pts, n, g, keys); break;
    case 5: cell_keys_kernel<5, K><<<b, 256, 0, s>>>(pts, n, g, keys); break;
    case 6: cell_keys_kernel<6, K><<<b, 256, 0, s>>>(pts, n, g, keys); break;
    case 7: cell_keys_kernel<7, K><<<b, 256, 0, s>>>(pts, n, g, keys); break;
    case 8: cell_keys_kernel<8, K><<<b, 256, 0, s>>>(pts, n, g, keys); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_cell_keys(const float* pts, long long n, const GridConst& g,
                             unsigned long long* keys, cudaStream_t s)
{
    return launch_cell_keys_t(pts, n, g, keys, s);
}

cudaError_t launch_cell_keys(const float* pts, long long n, const GridConst& g, unsigned int* keys,
                             cudaStream_t s)
{
    return launch_cell_keys_t(pts, n, g, keys, s);
}

namespace {
template <class K>
cudaError_t launch_query_keys_t(const float* q, long long m, const GridConst& g, int shift,
                                K* keys, cudaStream_t s)
{
    const int b = grid_for(m, 256);
    count_launches(1);
    switch (g.d) {
    case 1: query_keys_kernel<1, K><<<b, 256, 0, s>>>(q, m, g, shift, keys); break;
    case 2: query_keys_kernel<2, K><<<b, 256, 0, s>>>(q, m, g, shift, keys); break;
    case 3: query_keys_kernel<3, K><<<b, 256, 0, s>>>(q, m, g, shift, keys); break;
    case 4: query_keys_kernel<4, K><<<b, 256, 0, s>>>(q, m, g, shift, keys); break;
    case 5: query_keys_kernel<5, K><<<b, 256, 0, s>>>(q, m, g, shift, keys); break;
    case 6: query_keys_kernel<6, K><<<b, 256, 0, s>>>(q, m, g, shift, keys); break;
    case 7: query_keys_kernel<7, K><<<b, 256, 0, s>>>(q, m, g, shift, keys); break;
    case 8: query_keys_kernel<8, K><<<b, 256, 0, s>>>(q, m, g, shift, keys); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_query_keys(const float* q, long long m, const GridConst& g, int shift,
                              unsigned int* keys, cudaStream_t s)
{
    return launch_query_keys_t(q, m, g, shift, keys, s);
}

size_t scan_temp_bytes(long long n)
{
    const long long nb = (n + kScanBlock - 1) / kScanBlock;
    return (size_t)(nb > 0 ? nb : 1) * sizeof(unsigned int);
}

cudaError_t scan_exclusive(const unsigned int* in, unsigned int* out, long long n, void* temp,
                           cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long nb = (n + kScanBlock - 1) / kScanBlock;
    unsigned int* sums = static_cast<unsigned int*>(temp);
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
    scan_spine_kernel<<<1, 1024, 0, s>>>(sums, nb);
    scan_down_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
    count_launches(3);
    return cudaGetLastError();
}

size_t radix_temp_bytes(long long n)
{
    const long long nb = (n + kSortTile - 1) / kSortTile;
    const long long entries = (nb > 0 ? nb : 1) * kRadixMax;
    size_t hist = (size_t)entries * sizeof(unsigned int);
    hist = (hist + 255) & ~(size_t)255;
    return hist + scan_temp_bytes(entries);
}

namespace {
template <class K>
cudaError_t radix_sort_pairs_t(K* keys_a, unsigned int* vals_a, K* keys_b, unsigned int* vals_b,
                               long long n, int bits, void* temp, K** result_keys,
                               unsigned int** result_vals, cudaStream_t s, bool identity_vals)
{
    const long long nb = (n + kSortTile - 1) / kSortTile;
    unsigned int* hist = static_cast<unsigned int*>(temp);
    const size_t hist_bytes =
        ((size_t)(nb * kRadixMax) * sizeof(unsigned int) + 255) & ~(size_t)255;
    void* scan_tmp = static_cast<char*>(temp) + hist_bytes;
    K *kin = keys_a, *kout = keys_b;
    unsigned int *vin = vals_a, *vout = vals_b;
    // passes: 8-bit digits, except that when 9-bit digits need fewer passes
    // (bits mod 8 small), the top `wide` passes take 9 bits
    const int p8 = (bits + 7) / 8, p9 = (bits + 8) / 9;
    const int passes = p9 < p8 ? p9 : p8;
    const int wide = p9 < p8 ? bits - 8 * passes : 0;
    int shift = 0;
    // with identity_vals the first pass makes the values (each element's
    // index) instead of reading them
    if (identity_vals && (passes == 0 || n <= 1)) {
        iota_kernel<<<grid_for(n, 256), 256, 0, s>>>(vals_a, n);
        count_launches(1);
    }
    for (int pass = 0; pass < passes && n > 1; ++pass) {
        const bool w9 = pass >= passes - wide;
        const long long entries = nb * (w9 ? 512 : 256);
        const unsigned int* src = pass == 0 && identity_vals ? nullptr : vin;
        if (w9)
            radix_hist_kernel<K, 512><<<(unsigned)nb, kSortThreads, 0, s>>>(kin, n, shift, hist,
                                                                          (unsigned)nb);
        else
            radix_hist_kernel<K, 256><<<(unsigned)nb, kSortThreads, 0, s>>>(kin, n, shift, hist,
                                                                          (unsigned)nb);
        cudaError_t e = scan_exclusive(hist, hist, entries, scan_tmp, s);
        if (e != cudaSuccess) return e;
        if (w9)
            radix_scatter_kernel<K, 512><<<(unsigned)nb, kSortThreads, 0, s>>>(
                kin, src, kout, vout, n, shift, hist, (unsigned)nb);
        else
            radix_scatter_kernel<K, 256><<<(unsigned)nb, kSortThreads, 0, s>>>(
                kin, src, kout, vout, n, shift, hist, (unsigned)nb);
        shift += w9 ? 9 : 8;
        count_launches(2);
        K* tk = kin;
        kin = kout;
        kout = tk;
        unsigned int* tv = vin;
        vin = vout;
        vout = tv;
    }
    *result_keys = kin;
    *result_vals = vin;
    return cudaGetLastError();
}
}  // namespace

cudaError_t radix_sort_pairs(unsigned long long* keys_a, unsigned int* vals_a,
                             unsigned long long* keys_b, unsigned int* vals_b, long long n,
                             int bits, void* temp, unsigned long long** result_keys,
                             unsigned int** result_vals, cudaStream_t s, bool identity_vals)
{
    return radix_sort_pairs_t(keys_a, vals_a, keys_b, vals_b, n, bits, temp, result_keys,
                              result_vals, s, identity_vals);
}

cudaError_t radix_sort_pairs(unsigned int* keys_a, unsigned int* vals_a, unsigned int* keys_b,
                             unsigned int* vals_b, long long n, int bits, void* temp,
                             unsigned int** result_keys, unsigned int** result_vals,
                             cudaStream_t s, bool identity_vals)
{
    return radix_sort_pairs_t(keys_a, vals_a, keys_b, vals_b, n, bits, temp, result_keys,
                              result_vals, s, identity_vals);
}

namespace {
template <class K>
cudaError_t launch_cells_t(const K* sorted_keys, long long n, void* scan_tmp,
                           unsigned long long* cell_key, unsigned int* cell_start, GridDev* gdev,
                           cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long nb = (n + kScanBlock - 1) / kScanBlock;
    unsigned int* sums = static_cast<unsigned int*>(scan_tmp);
    cells_count_kernel<K><<<(unsigned)nb, kScanThreads, 0, s>>>(sorted_keys, n, sums);
    scan_spine_kernel<<<1, 1024, 0, s>>>(sums, nb);
    cells_write_kernel<K><<<(unsigned)nb, kScanThreads, 0, s>>>(sorted_keys, n, sums, cell_key,
                                                                cell_start, gdev);
    count_launches(3);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_cells(const unsigned long long* sorted_keys, long long n, void* scan_tmp,
                         unsigned long long* cell_key, unsigned int* cell_start, GridDev* gdev,
                         cudaStream_t s)
{
    return launch_cells_t(sorted_keys, n, scan_tmp, cell_key, cell_start, gdev, s);
}

cudaError_t launch_cells(const unsigned int* sorted_keys, long long n, void* scan_tmp,
                         unsigned long long* cell_key, unsigned int* cell_start, GridDev* gdev,
                         cudaStream_t s)
{
    return launch_cells_t(sorted_keys, n, scan_tmp, cell_key, cell_start, gdev, s);
}

cudaError_t launch_dense_table(const unsigned long long* cell_key, const unsigned int* cell_start,
                               const GridDev* gdev, unsigned long long ncell_space,
                               unsigned int* dstart, void* scan_tmp, cudaStream_t s)
{
    // dstart has ncell_space + 1 entries; the last one ends up as n.
    cudaError_t e = cudaMemsetAsync(dstart, 0, (ncell_space + 1) * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    dense_counts_kernel<<<grid_for((long long)ncell_space, 256), 256, 0, s>>>(cell_key, cell_start,
                                                                             gdev, dstart);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return scan_exclusive(dstart, dstart, (long long)ncell_space + 1, scan_tmp, s);
}

cudaError_t launch_hash_table(const unsigned long long* cell_key, const unsigned int* cell_start,
                              const GridDev* gdev, HashSlot* slots, unsigned long long max_slots,
                              cudaStream_t s)
{
    hash_clear_kernel<<<grid_for((long long)max_slots, 256), 256, 0, s>>>(slots, gdev);
    hash_insert_kernel<<<grid_for((long long)(max_slots / 2), 256), 256, 0, s>>>(cell_key,
                                                                                cell_start, gdev,
                                                                                slots);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_bitmap(const unsigned long long* cell_key, const GridDev* gdev,
                          unsigned int* bitmap, unsigned long long words, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bitmap, 0, words * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    bitmap_kernel<<<grid_for((long long)words * 16, 256), 256, 0, s>>>(cell_key, gdev, bitmap);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_hash_clear(HashSlot* slots, const GridDev* gdev, unsigned long long max_slots,
                              cudaStream_t s)
{
    hash_clear_kernel<<<grid_for((long long)max_slots, 256), 256, 0, s>>>(slots, gdev);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather(const float* pts, long long n, int d, const unsigned int* order,
                          float* rows, cudaStream_t s)
{
    const int b = grid_for(n, 256);
    count_launches(1);
    switch (d) {
    case 1: gather_kernel<1><<<b, 256, 0, s>>>(pts, n, order, rows); break;
    case 2: gather_kernel<2><<<b, 256, 0, s>>>(pts, n, order, rows); break;
    case 3: gather_kernel<3><<<b, 256, 0, s>>>(pts, n, order, rows); break;
    case 4: gather_kernel<4><<<b, 256, 0, s>>>(pts, n, order, rows); break;
    case 5: gather_kernel<5><<<b, 256, 0, s>>>(pts, n, order, rows); break;
    case 6: gather_kernel<6><<<b, 256, 0, s>>>(pts, n, order, rows); break;
    case 7: gather_kernel<7><<<b, 256, 0, s>>>(pts, n, order, rows); break;
    case 8: gather_kernel<8><<<b, 256, 0, s>>>(pts, n, order, rows); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_small_build(const float* pts, long long n, int d, const GridConst& g,
                               unsigned long long space, unsigned int* rid, float* rows,
                               unsigned int* dstart, GridDev* gdev, cudaStream_t s)
{
    if (n < 1 || n > kSmallMaxN || space > kSmallMaxCells) return cudaErrorInvalidValue;
    const size_t bytes = small_build_smem_bytes();
    static bool ready[kMaxD + 1] = {false};
    cudaError_t e = cudaSuccess;
#define GHN_SMALL_CASE(DD)                                                                      \
    case DD:                                                                                   \
        if (!ready[DD]) {                                                                      \
            e = cudaFuncSetAttribute(small_build_kernel<DD>,                                   \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
            if (e != cudaSuccess) return e;                                                    \
            ready[DD] = true;                                                                  \
        }                                                                                      \
        small_build_kernel<DD><<<1, kSmallThreads, bytes, s>>>(pts, (int)n, g,                 \
                                                               (unsigned int)space, rid, rows, \
                                                               dstart, gdev);                  \
        break;
    switch (d) {
        GHN_SMALL_CASE(1)
        GHN_SMALL_CASE(2)
        GHN_SMALL_CASE(3)
        GHN_SMALL_CASE(4)
        GHN_SMALL_CASE(5)
        GHN_SMALL_CASE(6)
        GHN_SMALL_CASE(7)
        GHN_SMALL_CASE(8)
    default: return cudaErrorInvalidValue;
    }
#undef GHN_SMALL_CASE
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace ghn
