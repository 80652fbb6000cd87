// The paper's cell measurement (Sec. III.A) on the GPU: per dimension, the
// largest number s of equal splits of [min, max] such that every split holds a
// training point, and the width w = (max - min) / s.
//
// A value's split is its Eq. 1 coordinate with width w (single precision,
// round to nearest), clamped to s - 1 (the last split is closed).  With the
// values sorted, every split is occupied exactly when consecutive values never
// skip a split and the largest value lands in the last one (the split of a
// value is monotone in the value).  Two facts keep the search small:
//   - a gap G between consecutive values with G <= 0.49 w never skips a
//     split for s <= 2^21: the computed quotients carry a relative error of
//     at most 2^-23 each, so their difference stays below 0.49 + 0.5 < 1;
//   - for s > 4 r / G_max + 1 (G_max the largest gap, r = max - min) the
//     largest gap spans more than 3.5 splits and skips one, even after the
//     clamp of the last split: no such s is feasible.
// So each candidate s in [1, min(distinct values, 2^21, 4 r / G_max + 2)] only
// checks the gaps above 0.49 w, largest first, and the candidates are handed
// out in decreasing order: once one is feasible, smaller ones are skipped.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "../../include/ghn_knn.h"
#include "build_launch.cuh"
#include "ghn_internal.cuh"

using namespace ghn;

namespace {

constexpr long long kMaxSplits = 2097152;  // 2^21
constexpr int kThreads = 256;

__device__ __forceinline__ unsigned int float_key(float v)
{
    const unsigned int u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_float(unsigned long long k)
{
    const unsigned int u = (unsigned int)k;
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Split of value v among s splits of width w from lo.
__device__ __forceinline__ long long split_of(float v, float lo, float w, long long s)
{
    const float t = floorf(__fdiv_rn(__fsub_rn(v, lo), w));
    if (!(t < (float)s)) return s - 1;
    return (long long)t;
}

// Column j as 32-bit ordered keys (a non-finite value sets *bad).
__global__ void column_keys_kernel(const float* __restrict__ pts, long long n, int d, int j,
                                   unsigned long long* __restrict__ keys,
                                   unsigned int* __restrict__ vals, unsigned int* bad)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float v = __ldg(pts + i * d + j);
        if (!isfinite(v)) atomicOr(bad, 1u);
        keys[i] = float_key(v);
        vals[i] = (unsigned int)i;
    }
}

// Distinct values and the largest gap of the sorted column (gaps are >= 0, so
// their bit patterns order like their values).
__global__ void gap_stats_kernel(const unsigned long long* __restrict__ sk, long long n,
                                 unsigned long long* distinct, unsigned int* gmax)
{
    __shared__ unsigned int s_cnt, s_g;
    if (threadIdx.x == 0) {
        s_cnt = 0u;
        s_g = 0u;
    }
    __syncthreads();
    unsigned int cnt = 0u, g = 0u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float v = key_float(sk[i]);
        if (i == 0) {
            ++cnt;
        } else {
            const float p = key_float(sk[i - 1]);
            if (v != p) ++cnt;
            const unsigned int gb = __float_as_uint(__fsub_rn(v, p));
            g = gb > g ? gb : g;
        }
    }
    atomicAdd(&s_cnt, cnt);
    atomicMax(&s_g, g);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(distinct, (unsigned long long)s_cnt);
        atomicMax(gmax, s_g);
    }
}

// The gaps above thr, keyed so that an ascending sort puts the largest first.
__global__ void big_gaps_kernel(const unsigned long long* __restrict__ sk, long long n, float thr,
                                unsigned long long* __restrict__ gkeys,
                                unsigned int* __restrict__ gidx, unsigned int* count)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = 1 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float g = __fsub_rn(key_float(sk[i]), key_float(sk[i - 1]));
        if (g > thr) {
            const unsigned int at = atomicAdd(count, 1u);
            gkeys[at] = (unsigned long long)(0xffffffffu - __float_as_uint(g));
            gidx[at] = (unsigned int)i;
        }
    }
}

// Candidates s from *next down; each feasible one raises *best.  A thread stops
// when the candidates left cannot beat the best feasible one found.
__global__ void candidates_kernel(const unsigned long long* __restrict__ sk, float lo, float r,
                                  float vmax, const unsigned long long* __restrict__ gkeys,
                                  const unsigned int* __restrict__ gidx, long long ng,
                                  unsigned long long* next, unsigned long long* best)
{
    for (;;) {
        const long long s = (long long)atomicAdd(next, ~0ull);  // take s, leave s - 1
        if (s < 1) return;
        if ((unsigned long long)s <= *(volatile unsigned long long*)best) return;
        const float w = __fdiv_rn(r, (float)s);
        bool ok = w > 0.0f && split_of(vmax, lo, w, s) == s - 1;
        const float thr = 0.49f * w;
        for (long long t = 0; ok && t < ng; ++t) {
            const float g = __uint_as_float(0xffffffffu - (unsigned int)gkeys[t]);
            if (!(g > thr)) break;  // the rest are smaller
            const unsigned int i = gidx[t];
            if (split_of(key_float(sk[i]), lo, w, s) - split_of(key_float(sk[i - 1]), lo, w, s) > 1)
                ok = false;
        }
        if (ok) atomicMax(best, (unsigned long long)s);
    }
}

float host_key_float(unsigned long long k)
{
    const unsigned int u = (unsigned int)k;
    const unsigned int b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
}

struct Buffers {
    cudaStream_t s;
    void* p[12] = {};
    int n = 0;
    explicit Buffers(cudaStream_t st) : s(st) {}
    ~Buffers()
    {
        for (int i = 0; i < n; ++i) device_free(p[i], s);
    }
    template <class T>
    knn_status alloc(T** out, size_t count, const char* what)
    {
        void* v = nullptr;
        knn_status st = device_alloc(&v, count * sizeof(T) + 16, s, what);
        if (st == KNN_OK) p[n++] = v;
        *out = static_cast<T*>(v);
        return st;
    }
};

}  // namespace

extern "C" knn_status knn_measure_cells(const float* points, int64_t n, int32_t d, int64_t* splits,
                                        float* cell_widths, void* stream)
{
    if (!points || !splits || !cell_widths) {
        set_error("knn_measure_cells: NULL argument");
        return KNN_EINVAL;
    }
    if (n < 1 || n >= (1ll << 31) || d < 1 || d > kMaxD) {
        set_error("knn_measure_cells: n must be in [1, 2^31) and d in [1, 8]");
        return KNN_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = device_sms(dev);
    // the points on the device (staged when they are host memory)
    cudaPointerAttributes pa{};
    const bool on_dev = cudaPointerGetAttributes(&pa, points) == cudaSuccess &&
                        (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    Buffers buf(s);
    const float* pts = points;
    unsigned long long *ka, *kb, *gk, *gk2, *cnt;
    unsigned int *va, *vb, *gi, *gi2;
    char* rtmp;
    float* staged = nullptr;
    knn_status st = KNN_OK;
    if (!on_dev) {
        st = buf.alloc(&staged, (size_t)(n * d), "measure points");
        if (st != KNN_OK) return st;
        if (cudaMemcpyAsync(staged, points, (size_t)(n * d) * 4, cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
            set_error("knn_measure_cells: staging the points failed");
            return KNN_ECUDA;
        }
        pts = staged;
    }
    if ((st = buf.alloc(&ka, (size_t)n, "measure keys")) != KNN_OK ||
        (st = buf.alloc(&kb, (size_t)n, "measure keys")) != KNN_OK ||
        (st = buf.alloc(&va, (size_t)n, "measure values")) != KNN_OK ||
        (st = buf.alloc(&vb, (size_t)n, "measure values")) != KNN_OK ||
        (st = buf.alloc(&gk, (size_t)n, "measure gaps")) != KNN_OK ||
        (st = buf.alloc(&gk2, (size_t)n, "measure gaps")) != KNN_OK ||
        (st = buf.alloc(&gi, (size_t)n, "measure gaps")) != KNN_OK ||
        (st = buf.alloc(&gi2, (size_t)n, "measure gaps")) != KNN_OK ||
        (st = buf.alloc(&cnt, 8, "measure counters")) != KNN_OK ||
        (st = buf.alloc(&rtmp, radix_temp_bytes(n), "measure sort")) != KNN_OK)
        return st;
    const int blocks = (int)std::min<long long>((n + kThreads - 1) / kThreads, (long long)sms * 8);
    // counters: [0] bad, [1] distinct, [2] gmax bits, [3] big-gap count, [4] next, [5] best
    for (int j = 0; j < d; ++j) {
        cudaError_t e = cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s);
        unsigned int* bad = reinterpret_cast<unsigned int*>(cnt);
        if (e == cudaSuccess) {
            column_keys_kernel<<<blocks, kThreads, 0, s>>>(pts, n, d, j, ka, va, bad);
            e = cudaGetLastError();
        }
        unsigned long long* sk = nullptr;
        unsigned int* sv = nullptr;
        if (e == cudaSuccess) e = radix_sort_pairs(ka, va, kb, vb, n, 32, rtmp, &sk, &sv, s);
        if (e == cudaSuccess) {
            gap_stats_kernel<<<blocks, kThreads, 0, s>>>(sk, n, cnt + 1,
                                                          reinterpret_cast<unsigned int*>(cnt + 2));
            e = cudaGetLastError();
        }
        unsigned long long h[3] = {0, 0, 0}, ends[2] = {0, 0};
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[0], sk, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], sk + n - 1, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        count_launches(2);
        if (e != cudaSuccess) {
            set_error(cudaGetErrorString(e));
            return KNN_ECUDA;
        }
        if (h[0] & 0xffffffffull) {
            set_error("knn_measure_cells: a coordinate is not finite");
            return KNN_EINVAL;
        }
        const float lo = host_key_float(ends[0]), hi = host_key_float(ends[1]);
        const float r = hi - lo;
        splits[j] = 1;
        cell_widths[j] = 1.0f;
        if (!(r > 0.0f)) continue;  // one value: one split
        const unsigned int gbits = (unsigned int)h[2];
        float gmax;
        memcpy(&gmax, &gbits, sizeof gmax);
        long long s_hi = std::min<long long>((long long)h[1], kMaxSplits);
        if (gmax > 0.0f) {
            const double bound = 4.0 * (double)r / (double)gmax + 2.0;
            if (bound < (double)s_hi) s_hi = std::max<long long>(1, (long long)bound);
        }
        const float thr = 0.49f * (r / (float)s_hi);
        unsigned int* gcount = reinterpret_cast<unsigned int*>(cnt + 3);
        big_gaps_kernel<<<blocks, kThreads, 0, s>>>(sk, n, thr, gk, gi, gcount);
        e = cudaGetLastError();
        unsigned int ng = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ng, gcount, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        count_launches(1);
        unsigned long long* lk = gk;
        unsigned int* li = gi;
        if (e == cudaSuccess && ng > 1) e = radix_sort_pairs(gk, gi, gk2, gi2, ng, 32, rtmp, &lk, &li, s);
        const unsigned long long start[2] = {(unsigned long long)s_hi, 0ull};
        if (e == cudaSuccess) e = cudaMemcpyAsync(cnt + 4, start, sizeof start, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            candidates_kernel<<<sms * 8, kThreads, 0, s>>>(sk, lo, r, hi, lk, li, (long long)ng,
                                                           cnt + 4, cnt + 5);
            e = cudaGetLastError();
            count_launches(1);
        }
        unsigned long long best = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&best, cnt + 5, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error(cudaGetErrorString(e));
            return KNN_ECUDA;
        }
        if (best < 1) best = 1;  // one split always holds every value
        splits[j] = (int64_t)best;
        cell_widths[j] = r / (float)best;
    }
    return KNN_OK;
}
