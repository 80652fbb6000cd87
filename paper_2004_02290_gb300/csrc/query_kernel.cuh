// Query kernel: exploration (Sec. III.B, Algorithm 2) and prediction (Sec. I).
//
// One warp per query, persistent grid, queries taken from a global counter.
// For layer L = 0, 1, 2, ... the warp enumerates the rows of cube(L) clipped to
// the box of occupied cells.  A row is a run of cells along the last dimension
// with fixed outer coordinates; the cells of one row have consecutive linear
// ids, so their points are one contiguous range of the cell-ordered rows.
// Rows whose outer coordinates are at Chebyshev distance L from the central
// cell lie entirely on layer L; other rows touch layer L only in their two end
// cells.  Each lane resolves one row into at most two row ranges; the warp
// flattens the ranges of 32 rows and streams their points 32 at a time with
// coalesced 8/16/32-byte loads.
//
// The k-buffer ("a heap of size k", Sec. III.B) is a sorted list of 64-bit
// keys (squared-distance bits << 32 | training index) spread over the lanes
// (one key per lane for k <= 32, two for k <= 64).  Squared distances are
// non-negative floats, so unsigned comparison of the keys is the order
// (distance, index).  A candidate enters by a ballot-and-shift insertion.
// "Update" (the stop test of Sec. III.B) is: some point of the layer entered
// the buffer; it depends only on which points the layer holds, not on the
// order they are offered in, so the warp-parallel walk stops exactly where a
// sequential walk does.
//
// Geometric skipping (result-preserving): once the buffer is full, a row, or a
// whole layer, whose distance from the query provably exceeds the k-th
// distance cannot contribute an update and is not read.  The bound works in
// cell units with a relative margin far larger than the rounding of Eq. 1 and
// of the distance, so no point that could enter the buffer is ever skipped.
// knn_query_stats runs the same walk without skipping and counts the work.

#pragma once

#include "ghn_internal.cuh"

#include <math.h>

namespace ghn {
namespace qk {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

template <int P>
struct Row;
template <>
struct Row<2> {
    float v[2];
    __device__ __forceinline__ void load(const float* rows, unsigned pos)
    {
        const float2 a = __ldg(reinterpret_cast<const float2*>(rows) + pos);
        v[0] = a.x;
        v[1] = a.y;
    }
};
template <>
struct Row<4> {
    float v[4];
    __device__ __forceinline__ void load(const float* rows, unsigned pos)
    {
        const float4 a = __ldg(reinterpret_cast<const float4*>(rows) + pos);
        v[0] = a.x;
        v[1] = a.y;
        v[2] = a.z;
        v[3] = a.w;
    }
};
template <>
struct Row<8> {
    float v[8];
    __device__ __forceinline__ void load(const float* rows, unsigned pos)
    {
        const float4 a = __ldg(reinterpret_cast<const float4*>(rows) + 2 * (size_t)pos);
        const float4 b = __ldg(reinterpret_cast<const float4*>(rows) + 2 * (size_t)pos + 1);
        v[0] = a.x;
        v[1] = a.y;
        v[2] = a.z;
        v[3] = a.w;
        v[4] = b.x;
        v[5] = b.y;
        v[6] = b.z;
        v[7] = b.w;
    }
};

// Sorted warp-distributed k-buffer.  Entry e lives in lane e % 32, slot e / 32.
template <int NS>
struct TopK {
    unsigned long long s[NS];
    int k;
    int count;               // entries filled (warp-uniform)
    unsigned long long kth;  // largest kept key when full, else ~0

    __device__ __forceinline__ void init(int k_)
    {
#pragma unroll
        for (int i = 0; i < NS; ++i) s[i] = kEmptyKey;
        k = k_;
        count = 0;
        kth = kEmptyKey;
    }

    // Insert x (warp-uniform, x < kth).
    __device__ __forceinline__ void insert(unsigned long long x, int lane)
    {
        int pos = 0;
#pragma unroll
        for (int i = 0; i < NS; ++i) pos += __popc(__ballot_sync(FULL, s[i] < x));
        if constexpr (NS == 1) {
            const unsigned long long up = __shfl_up_sync(FULL, s[0], 1);
            if (lane > pos) s[0] = up;
            if (lane == pos) s[0] = x;
            if (lane >= k) s[0] = kEmptyKey;
        } else {
            const unsigned long long upa = __shfl_up_sync(FULL, s[0], 1);
            const unsigned long long upb = __shfl_up_sync(FULL, s[1], 1);
            const unsigned long long carry = __shfl_sync(FULL, s[0], 31);
            // slot 1 (entries 32..63)
            const int e1 = 32 + lane;
            if (e1 > pos) s[1] = lane == 0 ? carry : upb;
            if (e1 == pos) s[1] = x;
            if (e1 >= k) s[1] = kEmptyKey;
            // slot 0 (entries 0..31)
            if (lane > pos) s[0] = upa;
            if (lane == pos) s[0] = x;
            if (lane >= k) s[0] = kEmptyKey;
        }
        if (count < k) ++count;
        if (count == k) {
            const int e = k - 1;
            if constexpr (NS == 1) {
                kth = __shfl_sync(FULL, s[0], e & 31);
            } else {
                const unsigned long long a = __shfl_sync(FULL, s[0], e & 31);
                const unsigned long long b = __shfl_sync(FULL, s[1], e & 31);
                kth = e < 32 ? a : b;
            }
        }
    }
};

// Lower bound, in cell units, of |v - u| over v in the cells [a, b] of one
// dimension (v = (p - o) / w as Eq. 1 computes it for points of those cells).
__device__ __forceinline__ float axis_gap(long long a, long long b, float u)
{
    const float lo = (float)a, hi = (float)(b + 1);
    return fmaxf(0.0f, fmaxf(lo - u, u - hi));
}

// Margin for the rounding of Eq. 1 and of the float conversions (cell units).
__device__ __forceinline__ float axis_margin(long long c, float u)
{
    return 1e-6f * (fabsf((float)c) + fabsf(u) + 2.0f);
}

template <int D, int NS, bool DENSE>
__global__ void __launch_bounds__(kThreads, 2) query_kernel(const QueryArgs a)
{
    constexpr int P = row_floats(D);
    __shared__ unsigned int s_end[kWarps][32];   // inclusive end of each lane's ranges
    __shared__ unsigned int s_beg[kWarps][32];   // exclusive start of each lane's ranges
    __shared__ unsigned int s_a[kWarps][32];     // first range: start
    __shared__ unsigned int s_la[kWarps][32];    // first range: length
    __shared__ unsigned int s_b[kWarps][32];     // second range: start

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const bool counting = a.stats != nullptr;
    const float w = a.g.w;
    const float w2 = __fmul_rn(w, w);
    unsigned long long hmask = 0ull;
    if constexpr (!DENSE) hmask = a.gdev->hmask;

    for (;;) {
        unsigned long long qi = 0ull;
        if (lane == 0) qi = atomicAdd(a.counter, 1ull);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= (unsigned long long)a.m) break;
        const long long qid = a.order ? (long long)a.order[qi] : (long long)qi;

        float q[D], u[D];
        long long c0[D];
        bool finite = true;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            q[j] = __ldg(a.q + qid * D + j);
            finite &= isfinite(q[j]);
        }
        TopK<NS> tk;
        tk.init(a.k);
        long long L = 0, lmin = 0;
        long long cells = 0, cands = 0;
        bool limited = false;
        if (!finite) {
            if (lane == 0) atomicOr(a.status, kStatusNonFinite);
            limited = true;
        } else {
#pragma unroll
            for (int j = 0; j < D; ++j) {
                // Eq. 1 on the query, single precision, round to nearest
                u[j] = __fdiv_rn(__fsub_rn(q[j], a.g.lo[j]), w);
                float f = floorf(u[j]);
                f = fminf(fmaxf(f, -kQueryClamp), kQueryClamp);
                c0[j] = (long long)f;
                long long gap = 0;
                if (c0[j] < 0) gap = -c0[j];
                if (c0[j] > a.g.cmax[j]) gap = c0[j] - a.g.cmax[j];
                lmin = gap > lmin ? gap : lmin;
            }
            // layers nearer than the box of occupied cells are empty
            L = lmin;
        }

        while (!limited) {
            long long lo[D], hi[D];
            bool covers = true;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                lo[j] = c0[j] - L < 0 ? 0 : c0[j] - L;
                hi[j] = c0[j] + L > a.g.cmax[j] ? a.g.cmax[j] : c0[j] + L;
                covers &= (c0[j] - L <= 0) && (c0[j] + L >= a.g.cmax[j]);
            }
            const bool full = tk.count == tk.k;
            const float kth_d = __uint_as_float((unsigned)(tk.kth >> 32));
            const bool may_skip = !counting && full && kth_d < 1e30f;
            bool updated = false;

            bool skip_layer = false;
            if (may_skip && L > 0) {
                // every cell of layer L is outside cube(L-1): bound the distance
                // from the query to the sides of that cube that have cells
                float gmin = INFINITY;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    const float mj = axis_margin(c0[j] + L, u[j]);
                    if (c0[j] + L <= a.g.cmax[j])
                        gmin = fminf(gmin, fmaxf(0.0f, (float)(c0[j] + L) - u[j] - mj));
                    if (c0[j] - L >= 0)
                        gmin = fminf(gmin, fmaxf(0.0f, u[j] - (float)(c0[j] - L + 1) - mj));
                }
                const float lb = __fmul_rn(__fmul_rn(gmin, gmin), w2) * (1.0f - 1e-5f);
                skip_layer = lb > kth_d;
            }

            if (!skip_layer) {
                // rows of cube(L) clipped to the box: outer dimensions 0..D-2
                unsigned long long nrows = 1ull;
#pragma unroll
                for (int j = 0; j < D - 1; ++j) nrows *= (unsigned long long)(hi[j] - lo[j] + 1);
                if (nrows >= (1ull << 32)) {
                    limited = true;
                    if (lane == 0) atomicOr(a.status, kStatusLimit);
                    break;
                }
                for (unsigned int rbase = 0; rbase < (unsigned int)nrows; rbase += 32) {
                    const unsigned int r = rbase + lane;
                    unsigned int sa = 0, la = 0, sb = 0, lb_ = 0;
                    if (r < (unsigned int)nrows) {
                        // decode the row's outer coordinates (last outer dim fastest)
                        unsigned int rr = r;
                        long long oc[D > 1 ? D - 1 : 1];
                        long long ocheb = 0;
                        unsigned long long base = 0ull;
                        float og2 = 0.0f;  // squared outer gap (cell units)
#pragma unroll
                        for (int j = D - 2; j >= 0; --j) {
                            const unsigned int ext = (unsigned int)(hi[j] - lo[j] + 1);
                            oc[j] = lo[j] + (long long)(rr % ext);
                            rr /= ext;
                            const long long dd = oc[j] > c0[j] ? oc[j] - c0[j] : c0[j] - oc[j];
                            ocheb = dd > ocheb ? dd : ocheb;
                            base += (unsigned long long)oc[j] * a.g.stride[j];
                            const float gj = fmaxf(0.0f, axis_gap(oc[j], oc[j], u[j]) -
                                                             axis_margin(oc[j], u[j]));
                            og2 += gj * gj;
                        }
                        // the row's cells on layer L, as up to two runs [x0, x1]
                        const int dl = D - 1;
                        long long a0 = 0, a1 = -1, b0 = 0, b1 = -1;  // empty when x1 < x0
                        if (ocheb == L) {
                            a0 = lo[dl];
                            a1 = hi[dl];
                        } else {
                            if (c0[dl] - L >= 0) a0 = a1 = c0[dl] - L;
                            if (c0[dl] + L <= a.g.cmax[dl]) b0 = b1 = c0[dl] + L;
                        }
                        // a run's rows: [st, en) of the cell-ordered rows
                        auto resolve = [&](long long x0, long long x1, unsigned int& st,
                                           unsigned int& len) {
                            st = 0u;
                            len = 0u;
                            if (x1 < x0) return;
                            if (may_skip) {
                                const float gl = fmaxf(0.0f, axis_gap(x0, x1, u[dl]) -
                                                                 axis_margin(x1, u[dl]) -
                                                                 axis_margin(x0, u[dl]));
                                const float lbr = __fmul_rn(og2 + gl * gl, w2) * (1.0f - 1e-5f);
                                if (lbr > kth_d) return;
                            }
                            if constexpr (DENSE) {
                                const unsigned int s0 =
                                    __ldg(a.dstart + base + (unsigned long long)x0);
                                const unsigned int e0 =
                                    __ldg(a.dstart + base + (unsigned long long)x1 + 1ull);
                                if (counting) {
                                    unsigned int prev = s0;
                                    for (long long x = x0; x <= x1; ++x) {
                                        const unsigned int nx =
                                            __ldg(a.dstart + base + (unsigned long long)x + 1ull);
                                        cells += nx > prev;
                                        prev = nx;
                                    }
                                }
                                st = s0;
                                len = e0 - s0;
                            } else {
                                unsigned int s0 = 0xffffffffu, e0 = 0u;
                                for (long long x = x0; x <= x1; ++x) {
                                    const unsigned long long key = base + (unsigned long long)x;
                                    unsigned long long h = mix64(key) & hmask;
                                    for (unsigned long long probe = 0; probe <= hmask; ++probe) {
                                        const ulonglong2 e =
                                            __ldg(reinterpret_cast<const ulonglong2*>(a.slots) + h);
                                        if (e.x == key) {
                                            const unsigned int es = (unsigned int)e.y;
                                            const unsigned int ee = (unsigned int)(e.y >> 32);
                                            s0 = es < s0 ? es : s0;
                                            e0 = ee > e0 ? ee : e0;
                                            ++cells;
                                            break;
                                        }
                                        if (e.x == kEmptyKey) break;
                                        h = (h + 1ull) & hmask;
                                    }
                                }
                                if (e0 > 0u) {
                                    st = s0;
                                    len = e0 - s0;
                                }
                            }
                        };
                        resolve(a0, a1, sa, la);
                        resolve(b0, b1, sb, lb_);
                    }
                    if (la == 0u && lb_ != 0u) {
                        sa = sb;
                        la = lb_;
                        lb_ = 0u;
                    }
                    // flatten the 32 lanes' ranges
                    const unsigned int tot = la + lb_;
                    cands += tot;
                    unsigned int incl = tot;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned int y = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const unsigned int total = __shfl_sync(FULL, incl, 31);
                    __syncwarp();
                    s_end[wib][lane] = incl;
                    s_beg[wib][lane] = incl - tot;
                    s_a[wib][lane] = sa;
                    s_la[wib][lane] = la;
                    s_b[wib][lane] = sb;
                    __syncwarp();
                    for (unsigned int cb = 0; cb < total; cb += 32) {
                        const unsigned int t = cb + lane;
                        unsigned long long key = kEmptyKey;
                        const bool open = tk.kth == kEmptyKey;
                        const float cur_d = __uint_as_float((unsigned)(tk.kth >> 32));
                        if (t < total) {
                            int lo_l = 0, hi_l = 31;  // the lane whose ranges hold candidate t
                            while (lo_l < hi_l) {
                                const int mid = (lo_l + hi_l) >> 1;
                                if (s_end[wib][mid] > t)
                                    hi_l = mid;
                                else
                                    lo_l = mid + 1;
                            }
                            const int ow = lo_l;
                            const unsigned int ln = s_la[wib][ow];
                            const unsigned int off = t - s_beg[wib][ow];
                            const unsigned int pos =
                                off < ln ? s_a[wib][ow] + off : s_b[wib][ow] + (off - ln);
                            Row<P> row;
                            row.load(a.rows, pos);
                            float acc = 0.0f;
#pragma unroll
                            for (int j = 0; j < D; ++j) {
                                const float dj = __fsub_rn(q[j], row.v[j]);
                                acc = __fadd_rn(acc, __fmul_rn(dj, dj));
                            }
                            if (open || acc <= cur_d) {
                                const unsigned int id = __ldg(a.rid + pos);
                                key = ((unsigned long long)__float_as_uint(acc) << 32) | id;
                            }
                        }
                        unsigned int pass = __ballot_sync(FULL, key < tk.kth);
                        while (pass) {
                            const int src = __ffs(pass) - 1;
                            pass &= pass - 1u;
                            const unsigned long long x = __shfl_sync(FULL, key, src);
                            if (x < tk.kth) {
                                tk.insert(x, lane);
                                updated = true;
                            }
                        }
                    }
                    __syncwarp();
                }
            }

            if (tk.count == tk.k && !updated) break;  // the stop rule of Sec. III.B
            if (covers) break;                        // every occupied cell seen
            if (a.max_layers > 0 && L - lmin + 1 >= a.max_layers) {
                limited = true;
                if (lane == 0) atomicOr(a.status, kStatusLimit);
                break;
            }
            ++L;
        }

        // ---- outputs ----
        const long long obase = qid * (long long)a.k;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const int e = i * 32 + lane;
            if (e < a.k) {
                const unsigned long long key = limited ? kEmptyKey : tk.s[i];
                const bool ok = key != kEmptyKey;
                a.ids[obase + e] = ok ? (int)(unsigned int)key : -1;
                if (a.dist2) a.dist2[obase + e] = ok ? __uint_as_float((unsigned)(key >> 32)) : INFINITY;
            }
        }
        const int found = limited ? 0 : tk.count;
        if (a.mode == 0 && a.pred) {
            // majority label among the found neighbours, ties to the smallest label
            unsigned int lab[NS];
            bool val[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                val[i] = i * 32 + lane < found;
                lab[i] = val[i] ? __ldg(a.labels + (unsigned int)tk.s[i]) : 0u;
            }
            unsigned long long best = 0ull;
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                int cnt = 0;
                for (int e = 0; e < found; ++e) {
                    unsigned int other;
                    if constexpr (NS == 1) {
                        other = __shfl_sync(FULL, lab[0], e);
                    } else {
                        const unsigned int o0 = __shfl_sync(FULL, lab[0], e & 31);
                        const unsigned int o1 = __shfl_sync(FULL, lab[1], e & 31);
                        other = e < 32 ? o0 : o1;
                    }
                    cnt += other == lab[i];
                }
                if (val[i]) {
                    const unsigned long long sc = ((unsigned long long)cnt << 32) |
                                                  (0xffffffffu - (lab[i] ^ 0x80000000u));
                    best = sc > best ? sc : best;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(FULL, best, o);
                best = y > best ? y : best;
            }
            if (lane == 0)
                static_cast<int*>(a.pred)[qid] =
                    found ? (int)((0xffffffffu - (unsigned int)best) ^ 0x80000000u) : 0;
        } else if (a.mode == 1 && a.pred) {
            // mean of the found neighbours' outputs: double sum in neighbour order
            float y[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i)
                y[i] = i * 32 + lane < found
                           ? __uint_as_float(__ldg(a.labels + (unsigned int)tk.s[i]))
                           : 0.0f;
            double sum = 0.0;
            for (int e = 0; e < found; ++e) {
                float v;
                if constexpr (NS == 1) {
                    v = __shfl_sync(FULL, y[0], e);
                } else {
                    const float v0 = __shfl_sync(FULL, y[0], e & 31);
                    const float v1 = __shfl_sync(FULL, y[1], e & 31);
                    v = e < 32 ? v0 : v1;
                }
                sum = __dadd_rn(sum, (double)v);
            }
            if (lane == 0)
                static_cast<float*>(a.pred)[qid] =
                    found ? __double2float_rn(__ddiv_rn(sum, (double)found)) : __int_as_float(0x7fc00000);
        }
        if (counting) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                cells += __shfl_xor_sync(FULL, cells, o);
                cands += __shfl_xor_sync(FULL, cands, o);
            }
            if (lane == 0) {
                a.stats[3 * qid + 0] = L + 1;
                a.stats[3 * qid + 1] = cells;
                a.stats[3 * qid + 2] = cands;
            }
        }
    }
}

template <int D, int NS, bool DENSE>
cudaError_t launch_one(const QueryArgs& a, int blocks, cudaStream_t s)
{
    query_kernel<D, NS, DENSE><<<blocks, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_d(const QueryArgs& a, int blocks, cudaStream_t s)
{
    const bool two = a.k > 32;
    if (a.dense) return two ? launch_one<D, 2, true>(a, blocks, s) : launch_one<D, 1, true>(a, blocks, s);
    return two ? launch_one<D, 2, false>(a, blocks, s) : launch_one<D, 1, false>(a, blocks, s);
}

}  // namespace qk
}  // namespace ghn
