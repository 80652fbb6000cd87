// Query kernel: exploration (Sec. III.B, Algorithm 2) and prediction (Sec. I).
//
// One warp per query, persistent grid, queries taken from a global counter.
//
// Layers.  For L = 0, 1, 2, ... the warp enumerates the rows of cube(L)
// clipped to the box of occupied cells.  A row is the run of cells along the
// last dimension with fixed outer coordinates.  Cells of one row have
// consecutive linear ids, so the points of any run of occupied cells of a row
// are one contiguous range of the cell-ordered rows.  A row whose outer
// coordinates are at Chebyshev distance L from the central cell lies wholly on
// layer L; any other row meets layer L only in its two end cells.  So a lane
// turns one row into at most two ranges, with at most two table lookups per
// range: the dense table gives a range directly; with the hash table an
// occupancy bitmap (when the box is small enough to afford one) finds the
// first and last occupied cell of the run, and only those two are probed.
//
// Candidates.  The warp flattens the ranges of 32 rows and streams their
// points with coalesced 8/16/32-byte loads, several chunks of 32 in flight.
//
// k-buffer (the paper keeps the k best in a heap, Sec. III.B).  Sorted 64-bit
// keys (squared distance bits << 32 | training index) over the lanes, one key per lane for
// k <= 32 and two for k <= 64.  Squared distances are non-negative floats, so
// unsigned order of the keys is the order (distance, index).  Few entering
// candidates are inserted one by one (ballot and shift); many are sorted
// (bitonic) and merged.  "Update" (the stop test of Sec. III.B) is: some point
// of the layer entered the buffer.  That depends only on which points the
// layer holds, not on the order in which they are offered, so the parallel
// walk stops exactly where a sequential walk does.
//
// Skipping (result-preserving).  Once the buffer is full, the k-th distance r
// bounds the search: each axis of the cube is clipped to the cells within r of
// the query, rows whose outer coordinates are farther than r are dropped, and
// a layer with no cell left within r ends the walk (it cannot update).  The
// bounds work in cell units with a margin (1e-6 relative per axis, 1e-5 on the
// square) far above the rounding of Eq. 1 and of the distance, so no point
// that could enter the buffer is skipped.  knn_query_stats runs the same walk
// without skipping and counts the method's work.

#pragma once

#include "ghn_internal.cuh"

#include <limits.h>
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

    __device__ __forceinline__ void refresh_kth()
    {
        const int e = k - 1;
        if (count < k) {
            kth = kEmptyKey;
        } else if constexpr (NS == 1) {
            kth = __shfl_sync(FULL, s[0], e & 31);
        } else {
            const unsigned long long a = __shfl_sync(FULL, s[0], e & 31);
            const unsigned long long b = __shfl_sync(FULL, s[1], e & 31);
            kth = e < 32 ? a : b;
        }
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
            const int e1 = 32 + lane;  // slot 1 holds entries 32..63
            if (e1 > pos) s[1] = lane == 0 ? carry : upb;
            if (e1 == pos) s[1] = x;
            if (e1 >= k) s[1] = kEmptyKey;
            if (lane > pos) s[0] = upa;
            if (lane == pos) s[0] = x;
            if (lane >= k) s[0] = kEmptyKey;
        }
        if (count < k) ++count;
        refresh_kth();
    }

    // Merge a warp of candidate keys (one per lane, kEmptyKey for none), k <= 32.
    __device__ __forceinline__ void merge32(unsigned long long x, int lane)
    {
        // bitonic sort of the candidates, ascending with the lane
#pragma unroll
        for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                const unsigned long long y = __shfl_xor_sync(FULL, x, stride);
                const bool up = (lane & size) == 0 || size == 32;
                const bool lower = (lane & stride) == 0;
                x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
            }
        }
        // the lane-wise min of the buffer and the reversed candidates holds the
        // 32 smallest of both, as a bitonic sequence; one bitonic merge sorts it
        const unsigned long long rev = __shfl_sync(FULL, x, 31 - lane);
        unsigned long long c = s[0] < rev ? s[0] : rev;
#pragma unroll
        for (int stride = 16; stride > 0; stride >>= 1) {
            const unsigned long long y = __shfl_xor_sync(FULL, c, stride);
            c = ((lane & stride) == 0) ? (c < y ? c : y) : (c < y ? y : c);
        }
        s[0] = lane < k ? c : kEmptyKey;
        count = __popc(__ballot_sync(FULL, s[0] != kEmptyKey));
        refresh_kth();
    }
};

// An upper bound of the exact square of a distance whose rounded square is at
// most x, for the roots that turn a squared distance into a radius.  A normal
// square is rounded by at most half an ulp, far inside the margins taken with
// the roots; a subnormal one by up to half the subnormal step 2^-149, which
// can be half of x itself, so one step is added.  The bound is at least the
// smallest normal number: the approximate root never sees a subnormal.
__device__ __forceinline__ float square_bound(float x)
{
    return fmaxf(x + 1.4e-45f, 1.17549435e-38f);
}

// Margin for the rounding of Eq. 1 and of float conversions (cell units).
__device__ __forceinline__ float axis_margin(float c, float u)
{
    return 1e-6f * (fabsf(c) + fabsf(u) + 2.0f);
}

// Squared lower bound of the distance along one axis between a query at u and
// any point of the cells [c0, c1] of that axis (cell c spans [c, c + 1) in the
// quotient of Eq. 1): the gap in cell units less the margin, scaled by w
// before squaring so that the bound overflows only where every distance does.
__device__ __forceinline__ float axis_gap2(long long c0, long long c1, float u, float w)
{
    const float lo = (float)c0, hi = (float)(c1 + 1);
    const float g = fmaxf(0.0f, fmaxf(lo - u, u - hi) - axis_margin(fabsf(lo) + fabsf(hi), u));
    const float gw = g * w;
    return gw * gw;
}

// The same bound for cells inside the box (32-bit coordinates: extents stay
// below 2^31, so c1 + 1 fits), with single-word conversions.
__device__ __forceinline__ float axis_gap2(int c0, int c1, float u, float w)
{
    const float lo = (float)c0, hi = (float)(c1 + 1);
    const float g = fmaxf(0.0f, fmaxf(lo - u, u - hi) - axis_margin(fabsf(lo) + fabsf(hi), u));
    const float gw = g * w;
    return gw * gw;
}

// Bits [b0, b1] of the occupancy bitmap: first and last set bit (b1 + 1 if none).
__device__ __forceinline__ void bitmap_span(const unsigned int* bm, unsigned long long b0,
                                            unsigned long long b1, unsigned long long& first,
                                            unsigned long long& last, int& count, bool want_count)
{
    first = b1 + 1ull;
    last = b1 + 1ull;
    count = 0;
    // a bitmap exists only for boxes of at most 2^33 cells: word indices fit
    // 32 bits
    const unsigned int w0 = (unsigned int)(b0 >> 5), w1 = (unsigned int)(b1 >> 5);
    for (unsigned int wi = w0; wi <= w1; ++wi) {
        unsigned int word = __ldg(bm + wi);
        if (wi == w0) word &= 0xffffffffu << ((unsigned int)b0 & 31u);
        if (wi == w1) word &= 0xffffffffu >> (31u - ((unsigned int)b1 & 31u));
        if (word) {
            const unsigned long long at = (unsigned long long)wi << 5;
            if (first > b1) first = at + (unsigned long long)(__ffs(word) - 1);
            last = at + (unsigned long long)(31 - __clz(word));
            if (want_count) count += __popc(word);
        }
    }
}

// Continue probing the open-addressing table for cell id `key` from slot h,
// whose content e is already loaded: the cell's row range, or 0/0.
__device__ __forceinline__ void hash_probe(const HashSlot* slots, unsigned long long hmask,
                                           unsigned long long key, unsigned long long h,
                                           ulonglong2 e, unsigned int& st, unsigned int& en,
                                           bool& found)
{
    st = 0u;
    en = 0u;
    found = false;
    for (unsigned long long probe = 0; probe <= hmask; ++probe) {
        if (e.x == key) {
            st = (unsigned int)e.y;
            en = (unsigned int)(e.y >> 32);
            found = true;
            return;
        }
        if (e.x == kEmptyKey) return;
        h = (h + 1ull) & hmask;
        e = __ldg(reinterpret_cast<const ulonglong2*>(slots) + h);
    }
}

// Probe the table for cell id `key`: its row range, or 0/0.
__device__ __forceinline__ void hash_lookup(const HashSlot* slots, unsigned long long hmask,
                                            unsigned long long key, unsigned int& st,
                                            unsigned int& en, bool& found)
{
    const unsigned long long h = mix64(key) & hmask;
    hash_probe(slots, hmask, key, h, __ldg(reinterpret_cast<const ulonglong2*>(slots) + h), st,
               en, found);
}

// Row range of the occupied cells among the cells [base + x0, base + x1] of one
// row; `cells` counts the occupied cells (only when counting).
template <bool DENSE>
__device__ __forceinline__ void resolve_run(const QueryArgs& a, unsigned long long hmask,
                                            unsigned long long base, long long x0, long long x1,
                                            bool counting, unsigned int& st, unsigned int& len,
                                            long long& cells)
{
    st = 0u;
    len = 0u;
    const unsigned long long i0 = base + (unsigned long long)x0;
    const unsigned long long i1 = base + (unsigned long long)x1;
    if constexpr (DENSE) {
        const unsigned int s0 = __ldg(a.dstart + i0);
        const unsigned int e0 = __ldg(a.dstart + i1 + 1ull);
        if (counting) {
            unsigned int prev = s0;
            for (unsigned long long i = i0; i <= i1; ++i) {
                const unsigned int nx = __ldg(a.dstart + i + 1ull);
                cells += nx > prev;
                prev = nx;
            }
        }
        st = s0;
        len = e0 - s0;
    } else if (a.bitmap) {
        unsigned long long f, l;
        int cnt;
        bitmap_span(a.bitmap, i0, i1, f, l, cnt, counting);
        cells += cnt;
        if (f > i1) return;
        // the first slots of both cells are loaded together; a batch of
        // indexes shares one table, keyed by index and cell id
        f |= a.key_prefix;
        l |= a.key_prefix;
        const unsigned long long hf = mix64(f) & hmask, hl = mix64(l) & hmask;
        const ulonglong2 ef = __ldg(reinterpret_cast<const ulonglong2*>(a.slots) + hf);
        const ulonglong2 el = __ldg(reinterpret_cast<const ulonglong2*>(a.slots) + hl);
        unsigned int s0, e0, s1, e1;
        bool ok0, ok1;
        hash_probe(a.slots, hmask, f, hf, ef, s0, e0, ok0);
        hash_probe(a.slots, hmask, l, hl, el, s1, e1, ok1);
        if (ok0 && ok1) {
            st = s0;
            len = e1 - s0;
        }
    } else {
        unsigned int s0 = 0xffffffffu, e0 = 0u;
        for (unsigned long long i = i0; i <= i1; ++i) {
            unsigned int cs, ce;
            bool ok;
            hash_lookup(a.slots, hmask, i | a.key_prefix, cs, ce, ok);
            if (ok) {
                s0 = cs < s0 ? cs : s0;
                e0 = ce > e0 ? ce : e0;
                ++cells;
            }
        }
        if (e0 > 0u) {
            st = s0;
            len = e0 - s0;
        }
    }
}

// ---------------------------------------------------------------------------
// Per-query pieces shared by the warp kernel and the cooperative kernel
// ---------------------------------------------------------------------------

// Squared distance between a query and a stored row, in the order the
// oracle fixes: per dimension a rounded difference and a rounded square, then
// a rounded running sum over the dimensions in order (no fused multiply-add).
// The differences and squares of two dimensions are computed together by the
// packed single-precision instructions (sub/mul .rn.f32x2: each half rounded
// to nearest as the scalar instruction is, subnormals kept); the sum stays one
// scalar chain.  It starts from the first square itself: 0 + x is x for
// every square x (never -0).
template <int D, int P>
__device__ __forceinline__ float sq_dist(const float (&q)[D], const Row<P>& row)
{
    float sq[D];
#pragma unroll
    for (int j = 0; j + 1 < D; j += 2) {
        unsigned long long qq, xx, dd, ss;
        asm("mov.b64 %0, {%1, %2};" : "=l"(qq) : "f"(q[j]), "f"(q[j + 1]));
        asm("mov.b64 %0, {%1, %2};" : "=l"(xx) : "f"(row.v[j]), "f"(row.v[j + 1]));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dd) : "l"(qq), "l"(xx));
        asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(ss) : "l"(dd));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(sq[j]), "=f"(sq[j + 1]) : "l"(ss));
    }
    if constexpr (D % 2 == 1) {
        const float dl = __fsub_rn(q[D - 1], row.v[D - 1]);
        sq[D - 1] = __fmul_rn(dl, dl);
    }
    float acc = sq[0];
#pragma unroll
    for (int j = 1; j < D; ++j) acc = __fadd_rn(acc, sq[j]);
    return acc;
}

template <int D>
struct Query {
    float q[D];
    float u[D];       // Eq. 1 quotient (q - o) / w, single precision
    long long c0[D];  // central cell, clamped to [-2^40, 2^40]
    long long lmin;   // first layer that reaches the box of occupied cells
    bool finite;
};

template <int D>
__device__ __forceinline__ void query_setup(const QueryArgs& a, long long qid, Query<D>& s)
{
    s.finite = true;
    s.lmin = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        s.q[j] = __ldg(a.q + qid * D + j);
        s.finite &= isfinite(s.q[j]);
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
        // Eq. 1 on the query, single precision, round to nearest
        s.u[j] = __fdiv_rn(__fsub_rn(s.q[j], a.g.lo[j]), a.g.w[j]);
        float f = floorf(s.u[j]);
        f = fminf(fmaxf(f, -kQueryClamp), kQueryClamp);  // NaN becomes -2^40
        s.c0[j] = (long long)f;
        long long gap = 0;
        if (s.c0[j] < 0) gap = -s.c0[j];
        if (s.c0[j] > a.g.cmax[j]) gap = s.c0[j] - a.g.cmax[j];
        s.lmin = gap > s.lmin ? gap : s.lmin;
    }
}

// cube(L) clipped to the box; when skipping, also clipped to the cells within
// the k-th distance kd of the query.  `empty`: no cell of layer L is left.
template <int D>
struct Layer {
    int lo[D], hi[D];  // every clipped coordinate fits 32 bits
    bool covers;       // cube(L) covers the whole box
    bool empty;
};

template <int D>
__device__ __forceinline__ void layer_box(const QueryArgs& a, const Query<D>& s, long long L,
                                          bool skipping, float kd, Layer<D>& b)
{
    b.covers = true;
    b.empty = false;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        b.lo[j] = (int)(s.c0[j] - L < 0 ? 0 : s.c0[j] - L);
        b.hi[j] = (int)(s.c0[j] + L > a.g.cmax[j] ? a.g.cmax[j] : s.c0[j] + L);
        b.covers &= (s.c0[j] - L <= 0) && (s.c0[j] + L >= a.g.cmax[j]);
    }
    if (!skipping) return;
    // a cell farther than kd along one axis cannot hold a point that enters;
    // the radius r_j = sqrt(kd) / w_j in cell units is taken of square_bound(kd)
    // with fast approximate operations (errors near 1e-6) and widened by 1e-4
    const float kb = square_bound(kd);
    const float rk = kb * rsqrtf(kb) * (1.0f + 1e-4f);
    bool shell = false;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float r = rk * a.g.inv_w[j];
        const float m = 1e-5f * (fabsf(s.u[j]) + r) + 1e-3f;
        const float a0f = floorf(s.u[j] - r - m), a1f = floorf(s.u[j] + r + m);
        // beyond the int range the clip would not tighten the box anyway
        const int a0 = a0f <= -2147483520.0f ? INT_MIN
                       : a0f >= 2147483520.0f ? INT_MAX : (int)a0f;
        const int a1 = a1f >= 2147483520.0f ? INT_MAX
                       : a1f <= -2147483520.0f ? INT_MIN : (int)a1f;
        if (a0 > b.lo[j]) b.lo[j] = a0 > b.hi[j] ? b.hi[j] + 1 : a0;
        if (a1 < b.hi[j]) b.hi[j] = a1 < b.lo[j] ? b.lo[j] - 1 : a1;
        b.empty |= b.lo[j] > b.hi[j];
        shell |= (s.c0[j] - L >= b.lo[j] && s.c0[j] - L <= b.hi[j]) ||
                 (s.c0[j] + L >= b.lo[j] && s.c0[j] + L <= b.hi[j]);
    }
    b.empty |= !shell;
}

// The certified stop (a variant of the paper's rule whose result equals
// exhaustive KNN): after cube(L), every training point not yet seen lies in a
// cell beyond c0_j + L or below c0_j - L along some axis j where the box still
// holds cells.  The nearest such cell on each side bounds its distance from
// below (axis_gap2: the gap in cell units less the rounding margin of Eq. 1,
// scaled by w_j); the walk may stop when the smallest of these bounds, less
// the rounding of a single-precision squared distance, exceeds the k-th
// squared distance, which is the skipping test applied to every unseen cell.
template <int D>
__device__ __forceinline__ bool certified(const QueryArgs& a, const Query<D>& s, long long L,
                                          float kth_d)
{
    float g2 = INFINITY;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        if (s.c0[j] + L < a.g.cmax[j]) {
            const long long c = s.c0[j] + L + 1;
            g2 = fminf(g2, axis_gap2(c, c, s.u[j], a.g.w[j]));
        }
        if (s.c0[j] - L > 0) {
            const long long c = s.c0[j] - L - 1;
            g2 = fminf(g2, axis_gap2(c, c, s.u[j], a.g.w[j]));
        }
    }
    return g2 * (1.0f - 1e-5f) > kth_d;
}

template <int D>
__device__ __forceinline__ unsigned long long layer_rows(const Layer<D>& b)
{
    unsigned long long nrows = 1ull;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) nrows *= (unsigned long long)(b.hi[j] - b.lo[j] + 1);
    return nrows;
}

// x / e for x < 2^16 and 1 <= e < 2^31, from a single-precision reciprocal
// of e: the estimate is within 1/64 of x / e, so one step each way corrects
// it (no integer division on the walk's path).
__device__ __forceinline__ unsigned int udiv_small(unsigned int x, unsigned int e, float inv_e)
{
    unsigned int q = (unsigned int)((float)x * inv_e);
    if (q * e > x) --q;
    if ((q + 1u) * e <= x) ++q;
    return q;
}

// Row odometer over the outer axes 0..D-2 of the layer box, last outer axis
// fastest: digits of the starting row and of the stride between visits.
template <int D>
struct RowWalk {
    int dig[D > 1 ? D - 1 : 1];
    int inc[D > 1 ? D - 1 : 1];

    // first and step are below 2^16 (a lane or thread and the warp or block size)
    __device__ __forceinline__ void start(const Layer<D>& b, unsigned int first, unsigned int step)
    {
#pragma unroll
        for (int j = D - 2; j >= 0; --j) {
            const unsigned int e = (unsigned int)(b.hi[j] - b.lo[j] + 1);
            const float inv = __frcp_rn((float)e);
            const unsigned int qf = udiv_small(first, e, inv);
            const unsigned int qs = udiv_small(step, e, inv);
            dig[j] = (int)(first - qf * e);
            first = qf;
            inc[j] = (int)(step - qs * e);
            step = qs;
        }
    }
    __device__ __forceinline__ void advance(const Layer<D>& b)
    {
        int carry = 0;
#pragma unroll
        for (int j = D - 2; j >= 0; --j) {
            const int e = b.hi[j] - b.lo[j] + 1;
            const int v = dig[j] + inc[j] + carry;
            carry = v >= e;
            dig[j] = carry ? v - e : v;
        }
    }
};

// The ranges of one row of layer L: the whole clipped row when its outer
// coordinates are on the shell, else its two end cells.  A run that the
// k-th distance kth_d excludes is dropped when `prune` is set.
template <int D, bool DENSE>
__device__ __forceinline__ void row_ranges(const QueryArgs& a, unsigned long long hmask,
                                           const Query<D>& s, const Layer<D>& b,
                                           const RowWalk<D>& rw, long long L, bool prune,
                                           float kth_d, bool counting, unsigned int& sa,
                                           unsigned int& la, unsigned int& sb, unsigned int& lb,
                                           long long& cells)
{
    constexpr int dl = D - 1;
    long long ocheb = 0;
    unsigned long long base = 0ull;
    float og2 = 0.0f;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) {
        const long long c = (long long)(b.lo[j] + rw.dig[j]);
        const long long dd = c > s.c0[j] ? c - s.c0[j] : s.c0[j] - c;
        ocheb = dd > ocheb ? dd : ocheb;
        base += (unsigned long long)c * a.g.stride[j];
        og2 += axis_gap2((int)c, (int)c, s.u[j], a.g.w[j]);
    }
    long long x0a, x1a, x0b, x1b;
    if (ocheb == L) {
        x0a = b.lo[dl];
        x1a = b.hi[dl];
        x0b = 1;
        x1b = 0;
    } else {
        x0a = x1a = s.c0[dl] - L;
        x0b = x1b = s.c0[dl] + L;
        if (x0a < b.lo[dl] || x0a > b.hi[dl]) {
            x0a = 1;
            x1a = 0;
        }
        if (x0b < b.lo[dl] || x0b > b.hi[dl]) {
            x0b = 1;
            x1b = 0;
        }
    }
    sa = la = sb = lb = 0u;
    if (prune && kth_d <= 3.0e38f) {
        // along the row's own axis only the cells within the radius left over
        // by the outer axes, sqrt(kth_d - og2), can hold a point that enters:
        // clip both runs to them (the root of square_bound, approximate and
        // widened as in layer_box).
        // An infinite k-th distance (overflowed squares) clips nothing.
        const float rem = kth_d * (1.0f + 2e-5f) - og2;
        if (rem < 0.0f) return;
        const float rb = square_bound(rem);
        const float r = rb * rsqrtf(rb) * a.g.inv_w[dl] * (1.0f + 1e-4f);
        const float u = s.u[dl];
        const float m = 1e-5f * (fabsf(u) + r) + 1e-3f;
        const float c0f = floorf(u - r - m), c1f = floorf(u + r + m);
        // the clip only matters inside the row's 32-bit coordinate range
        const long long c0 = c0f <= -2147483520.0f ? (long long)INT_MIN : (long long)c0f;
        const long long c1 = c1f >= 2147483520.0f ? (long long)INT_MAX : (long long)c1f;
        x0a = x0a > c0 ? x0a : c0;
        x1a = x1a < c1 ? x1a : c1;
        x0b = x0b > c0 ? x0b : c0;
        x1b = x1b < c1 ? x1b : c1;
    }
    // the two runs by one copy of the lookup code (a smaller kernel: measured
    // 5% faster on large_cls than two inlined copies)
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
        const long long x0 = r ? x0b : x0a, x1 = r ? x1b : x1a;
        unsigned int st = 0u, ln = 0u;
        if (x0 <= x1 &&
            !(prune && (og2 + axis_gap2((int)x0, (int)x1, s.u[dl], a.g.w[dl])) * (1.0f - 1e-5f) >
                           kth_d))
            resolve_run<DENSE>(a, hmask, base, x0, x1, counting, st, ln, cells);
        if (r) {
            sb = st;
            lb = ln;
        } else {
            sa = st;
            la = ln;
        }
    }
    if (la == 0u) {
        sa = sb;
        la = lb;
        lb = 0u;
    }
}

// Above this many entering keys, one bitonic merge is cheaper than inserting
// the keys one by one (4 measured 1-2% slower on GB300).
constexpr int kMergeMin = 6;

// Offer one key per lane to the buffer; true when some key entered it.  Keys
// not below `cap` are refused (the cooperative kernel's block-wide k-th key).
template <int NS>
__device__ __forceinline__ bool offer(TopK<NS>& tk, unsigned long long key, int lane,
                                      unsigned long long cap = kEmptyKey)
{
    const bool pass = key < (tk.kth < cap ? tk.kth : cap);
    unsigned int pm = __ballot_sync(FULL, pass);
    if (pm == 0u) return false;
    if (NS == 1 && __popc(pm) > kMergeMin) {
        tk.merge32(pass ? key : kEmptyKey, lane);
    } else {
        while (pm) {
            const int src = __ffs(pm) - 1;
            pm &= pm - 1u;
            const unsigned long long x = __shfl_sync(FULL, key, src);
            if (x < tk.kth) tk.insert(x, lane);  // x < cap already
        }
    }
    return true;
}

// ids, squared distances and the prediction of one query, from its buffer.
template <int NS>
__device__ __forceinline__ void write_outputs(const QueryArgs& a, long long qid,
                                              const TopK<NS>& tk, bool limited, int lane)
{
    const long long obase = qid * (long long)a.k;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int e = i * 32 + lane;
        if (e < a.k) {
            const unsigned long long key = limited ? kEmptyKey : tk.s[i];
            const bool ok = key != kEmptyKey;
            a.ids[obase + e] = ok ? (int)(unsigned int)key : -1;
            if (a.dist2)
                a.dist2[obase + e] = ok ? __uint_as_float((unsigned)(key >> 32)) : INFINITY;
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
            y[i] = i * 32 + lane < found ? __uint_as_float(__ldg(a.labels + (unsigned int)tk.s[i]))
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
                found ? __double2float_rn(__ddiv_rn(sum, (double)found))
                      : __int_as_float(0x7fc00000);
    } else if (a.mode == 2 && a.pred) {
        // median of the found neighbours' outputs (Sec. I, Sec. III.D): each
        // value's rank under IEEE total order (ties by neighbour position),
        // then the one or two middle values; an even count averages them in
        // double
        unsigned int key[NS];
        float y[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const bool v = i * 32 + lane < found;
            const unsigned int u = v ? __ldg(a.labels + (unsigned int)tk.s[i]) : 0u;
            y[i] = __uint_as_float(u);
            key[i] = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
        }
        int rank[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) rank[i] = 0;
        for (int e = 0; e < found; ++e) {
            unsigned int other;
            if constexpr (NS == 1) {
                other = __shfl_sync(FULL, key[0], e);
            } else {
                const unsigned int o0 = __shfl_sync(FULL, key[0], e & 31);
                const unsigned int o1 = __shfl_sync(FULL, key[1], e & 31);
                other = e < 32 ? o0 : o1;
            }
#pragma unroll
            for (int i = 0; i < NS; ++i)
                rank[i] += other < key[i] || (other == key[i] && e < i * 32 + lane);
        }
        const int lo = (found - 1) >> 1, hi = found >> 1;
        float vlo = 0.0f, vhi = 0.0f;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const bool v = i * 32 + lane < found;
            const unsigned int blo = __ballot_sync(FULL, v && rank[i] == lo);
            const unsigned int bhi = __ballot_sync(FULL, v && rank[i] == hi);
            const float fl = __shfl_sync(FULL, y[i], blo ? __ffs(blo) - 1 : 0);
            const float fh = __shfl_sync(FULL, y[i], bhi ? __ffs(bhi) - 1 : 0);
            if (blo) vlo = fl;
            if (bhi) vhi = fh;
        }
        if (lane == 0) {
            float out = __int_as_float(0x7fc00000);
            if (found & 1)
                out = vlo;
            else if (found)
                out = __double2float_rn(__dmul_rn(__dadd_rn((double)vlo, (double)vhi), 0.5));
            static_cast<float*>(a.pred)[qid] = out;
        }
    }
}

// ---------------------------------------------------------------------------
// The warp kernel: one warp per query
// ---------------------------------------------------------------------------


// Resident blocks per SM the warp kernel is compiled for.  The walk is bound by
// memory latency and instruction issue, so more resident warps pay even when
// the register cap spills a little to L1 (measured: 8 blocks on the d=3 and
// d=4 workloads, where 6 was 3% slower; 6 for d=5 and 6, 3% faster than 4
// and 52% faster than 8 on the batched d=6 problems; 4 for the larger query
// state of d=7 and 8).
template <int D, int NS>
struct MinBlocks {
    static constexpr int value = NS == 1 ? (D <= 4 ? 8 : (D <= 6 ? 6 : 4)) : 2;
};

// Per-warp shared memory of the walk: the lanes' ranges of one row batch.
// Lane l's candidates are the flattened positions t in [end[l-1], end[l]):
// its first range for t < mid[l], its second one after, and the stored row
// of t is ao[l] + t or bo[l] + t (offsets taken modulo 2^32).
struct WarpSmem {
    unsigned int end[32];  // inclusive end of each lane's ranges, flattened
    unsigned int mid[32];  // where the lane's second range starts, flattened
    unsigned int ao[32];   // first range: row of t minus t
    unsigned int bo[32];   // second range: row of t minus t
};

// The lane whose ranges hold flattened candidate t (t < end[31]): binary
// search over the lanes' inclusive ends.
__device__ __forceinline__ unsigned int owner_of(const unsigned int* end, unsigned int t)
{
    int lo_l = 0, hi_l = 31;
#pragma unroll
    for (int it = 0; it < 5; ++it) {
        const int mid = (lo_l + hi_l) >> 1;
        if (end[mid] > t)
            hi_l = mid;
        else
            lo_l = mid + 1;
    }
    return (unsigned int)lo_l;
}

// One query by one warp.  Returns true when the query was deferred to the
// cooperative kernel (nothing written); otherwise its outputs are written.
template <int D, int NS, bool DENSE, bool EXACT, bool COUNT>
__device__ __forceinline__ bool walk_query(const QueryArgs& a, long long qid, WarpSmem& sm,
                                           int lane, bool may_defer)
{
    constexpr bool counting = COUNT;  // the exhaustive counting walk of knn_query_stats
    unsigned long long hmask = 0ull;
    if constexpr (!DENSE) hmask = a.gdev->hmask;
    Query<D> s;
    query_setup(a, qid, s);
    TopK<NS> tk;
    tk.init(a.k);
    long long L = s.lmin;
    long long cells = 0, cands = 0;
    unsigned long long rows_seen = 0ull;  // rows enumerated so far (the work bound)
    bool limited = !s.finite, deferred = false;
    if (!s.finite && lane == 0) atomicOr(a.status, kStatusNonFinite);

    while (!limited) {
        Layer<D> b;
        const float kd0 = __uint_as_float((unsigned)(tk.kth >> 32));
        layer_box(a, s, L, !counting && tk.count == tk.k && kd0 < 1e30f, kd0, b);
        bool updated = false;
        if (!b.empty) {
            const unsigned long long nrows = layer_rows(b);
            rows_seen += nrows;
            if (nrows >= (1ull << 32) ||
                (a.max_rows > 0 && rows_seen > (unsigned long long)a.max_rows)) {
                limited = true;
                if (lane == 0) atomicOr(a.status, kStatusLimit);
                break;
            }
            if (may_defer && nrows > a.heavy_rows) {
                deferred = true;
                break;
            }
            RowWalk<D> rw;
            rw.start(b, (unsigned int)lane, 32u);
            for (unsigned int rb = 0; rb < (unsigned int)nrows; rb += 32u) {
                unsigned int sa = 0u, la = 0u, sb = 0u, lb = 0u;
                const bool full = tk.count == tk.k;
                const float kth_d = __uint_as_float((unsigned)(tk.kth >> 32));
                if (rb + lane < (unsigned int)nrows)
                    row_ranges<D, DENSE>(a, hmask, s, b, rw, L, !counting && full, kth_d, counting,
                                         sa, la, sb, lb, cells);
                rw.advance(b);
                // flatten the lanes' ranges
                const unsigned int tot = la + lb;
                cands += tot;
                unsigned int incl = tot;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned int y = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += y;
                }
                const unsigned int total = __shfl_sync(FULL, incl, 31);
                if (total == 0u) continue;
                if (may_defer && total > a.heavy_cands) {
                    deferred = true;
                    break;
                }
                __syncwarp();
                sm.end[lane] = incl;
                sm.mid[lane] = incl - lb;
                sm.ao[lane] = sa - (incl - tot);
                sm.bo[lane] = sb - (incl - lb);
                __syncwarp();
                // chunks of 32 candidates, one per lane.  Each chunk loads its
                // own rows: with 6 to 8 resident blocks an SM, other warps
                // cover the load, and a row prefetched a chunk ahead cost a
                // copy per chunk and more spilled registers (measured 3%
                // slower on the d=6 batched group and on large_cls)
                constexpr int P = row_floats(D);
                // each lane's cursor: the lane `own` whose ranges hold its
                // next candidate (a binary search for the first chunk, then
                // forward moves only when a chunk step leaves own's ranges)
                // and a copy of own's range offsets
                unsigned int own = 0u, o_end = 0u, o_mid = 0u, o_ao = 0u, o_bo = 0u;
                if (lane < total) {
                    own = owner_of(sm.end, lane);
                    o_end = sm.end[own];
                    o_mid = sm.mid[own];
                    o_ao = sm.ao[own];
                    o_bo = sm.bo[own];
                }
                // the k-th squared distance (+inf while the buffer is short)
                float kf = tk.count == tk.k ? __uint_as_float((unsigned)(tk.kth >> 32)) : INFINITY;
                for (unsigned int cb = 0; cb < total; cb += 32u) {
                    const unsigned int t = cb + lane;
                    bool pass = false;
                    float acc = 0.0f;
                    unsigned int pos = 0u;
                    if (t < total) {
                        if (t >= o_end) {
                            do {
                                ++own;
                            } while (sm.end[own] <= t);  // ends at 31 at the latest
                            o_end = sm.end[own];
                            o_mid = sm.mid[own];
                            o_ao = sm.ao[own];
                            o_bo = sm.bo[own];
                        }
                        pos = (t < o_mid ? o_ao : o_bo) + t;
                        Row<P> row;
                        row.load(a.rows, pos);
                        acc = sq_dist<D, P>(s.q, row);
                        pass = acc <= kf;
                    }
                    // the training index is read only for the candidates that
                    // pass the distance test; the key's order then decides
                    if (__ballot_sync(FULL, pass)) {
                        const unsigned long long key =
                            pass ? ((unsigned long long)__float_as_uint(acc) << 32) |
                                       __ldg(a.rid + pos)
                                 : kEmptyKey;
                        if (offer(tk, key, lane)) {
                            updated = true;
                            kf = tk.count == tk.k ? __uint_as_float((unsigned)(tk.kth >> 32))
                                                  : INFINITY;
                        }
                    }
                }
                __syncwarp();
            }
            if (deferred) break;
        }
        // the stop rule of Sec. III.B, or the certified one (compiled apart)
        if constexpr (EXACT) {
            if (tk.count == tk.k && certified(a, s, L, __uint_as_float((unsigned)(tk.kth >> 32))))
                break;
        } else {
            if (tk.count == tk.k && !updated) break;
        }
        if (b.covers) break;                      // every occupied cell seen
        if (a.max_layers > 0 && L - s.lmin + 1 >= a.max_layers) {
            limited = true;
            if (lane == 0) atomicOr(a.status, kStatusLimit);
            break;
        }
        ++L;
    }
    if (deferred) return true;
    write_outputs(a, qid, tk, limited, lane);
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
    return false;
}

template <int D, int NS, bool DENSE, bool EXACT, bool COUNT>
__global__ void __launch_bounds__(kThreads, (MinBlocks<D, NS>::value))
    query_kernel(const QueryArgs a)
{
    __shared__ WarpSmem sm[kWarps];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const bool may_defer = !COUNT && a.heavy_list != nullptr;

    // the next query is claimed one query ahead, so the atomic's latency
    // overlaps the current query's work
    unsigned long long next = 0ull;
    if (lane == 0) next = atomicAdd(a.counter, 1ull);
    next = __shfl_sync(FULL, next, 0);
    while (next < (unsigned long long)a.m) {
        const unsigned long long qi = next;
        if (lane == 0) next = atomicAdd(a.counter, 1ull);
        const long long qid = a.order ? (long long)a.order[qi] : (long long)qi;
        if (walk_query<D, NS, DENSE, EXACT, COUNT>(a, qid, sm[wib], lane, may_defer) &&
            lane == 0) {
            // too much work for one warp: the cooperative kernel takes it
            a.heavy_list[atomicAdd(a.heavy_count, 1u)] = (unsigned int)qid;
        }
        next = __shfl_sync(FULL, next, 0);
    }
}

// ---------------------------------------------------------------------------
// The cooperative kernel: one block per deferred query.  Rows and candidates
// of each layer are spread over the block's warps.  Each warp collects the
// top k of its own share of the layer's candidates (refusing any key not below
// the block's k-th key), and at the end of the layer the warps' lists are
// merged into the block's buffer.  The merged buffer is the top k of the
// previous buffer and of every candidate of the layer, and the layer
// "updated" it exactly when it changed, so the stop rule is the one of the
// sequential walk.  A warp skips with min(its own k-th key, the block's),
// which is never below the merged k-th key.
//
// A deferred query is a latency chain: its layers, and the rounds of rows
// within a layer, run one after another, while few queries are deferred at
// a time.  The block is 512 threads, the widest that keeps the walk's
// registers (about 128 a thread) without spilling, so a round resolves 512
// rows.
// ---------------------------------------------------------------------------

constexpr int kCoopWarps = 16;
constexpr int kCoopThreads = kCoopWarps * 32;
constexpr int kRoundRows = kCoopThreads;  // rows resolved per round (one per thread)
constexpr int kRangeCap = 2 * kRoundRows;  // at most two ranges per row

// Shared memory of the cooperative walk.
struct CoopSmem {
    unsigned long long top[64];        // the block's buffer
    unsigned long long loc[kCoopWarps][64];  // each warp's list of the layer
    unsigned int r_start[kRangeCap];
    unsigned int r_len[kRangeCap];
    unsigned int r_end[kRangeCap];  // inclusive end of each range, flattened
    unsigned int wsum[kCoopWarps];
    unsigned int nr;
    int count;
    int updated;
};

// One query by the whole block (every thread calls it).
template <int D, int NS, bool DENSE, bool EXACT>
__device__ __forceinline__ void coop_query(const QueryArgs& a, long long qid, CoopSmem& sm)
{
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned long long hmask = 0ull;
    if constexpr (!DENSE) hmask = a.gdev->hmask;
    Query<D> s;
    query_setup(a, qid, s);
    if (threadIdx.x < 64) sm.top[threadIdx.x] = kEmptyKey;
    if (threadIdx.x == 0) sm.count = 0;
    __syncthreads();

    TopK<NS> tk;
    long long L = s.lmin;
    unsigned long long rows_seen = 0ull;  // rows enumerated so far (the work bound)
    bool limited = false;
    for (;;) {
        // the block's k-th key at the start of the layer, and an empty list
        // for this warp's share of the layer
        const unsigned long long gkth = sm.count == a.k ? sm.top[a.k - 1] : kEmptyKey;
        tk.init(a.k);
        Layer<D> b;
        const float kd0 = __uint_as_float((unsigned)(gkth >> 32));
        layer_box(a, s, L, gkth != kEmptyKey && kd0 < 1e30f, kd0, b);
        if (!b.empty) {
            const unsigned long long nrows = layer_rows(b);
            rows_seen += nrows;
            if (nrows >= (1ull << 32) ||
                (a.max_rows > 0 && rows_seen > (unsigned long long)a.max_rows)) {
                limited = true;
                if (threadIdx.x == 0) atomicOr(a.status, kStatusLimit);
                break;
            }
            RowWalk<D> rw;
            rw.start(b, (unsigned int)threadIdx.x, (unsigned int)kRoundRows);
            for (unsigned long long rb = 0; rb < nrows; rb += kRoundRows) {
                if (threadIdx.x == 0) sm.nr = 0u;
                __syncthreads();
                unsigned int sa = 0u, la = 0u, sb = 0u, lb = 0u;
                long long unused = 0;
                const unsigned long long ek = tk.kth < gkth ? tk.kth : gkth;
                if (rb + threadIdx.x < nrows)
                    row_ranges<D, DENSE>(a, hmask, s, b, rw, L, ek != kEmptyKey,
                                         __uint_as_float((unsigned)(ek >> 32)), false, sa, la, sb,
                                         lb, unused);
                rw.advance(b);
                // append the non-empty ranges to the block's list
                const unsigned int mine = (la > 0u) + (lb > 0u);
                unsigned int incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned int y = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += y;
                }
                unsigned int wbase = 0u;
                if (lane == 31 && incl) wbase = atomicAdd(&sm.nr, incl);
                wbase = __shfl_sync(FULL, wbase, 31);
                unsigned int at = wbase + incl - mine;
                if (la) {
                    sm.r_start[at] = sa;
                    sm.r_len[at] = la;
                    ++at;
                }
                if (lb) {
                    sm.r_start[at] = sb;
                    sm.r_len[at] = lb;
                }
                __syncthreads();
                // flatten the ranges: inclusive prefix of their lengths
                const unsigned int nr = sm.nr;
                const unsigned int i0 = 2u * threadIdx.x, i1 = i0 + 1u;
                const unsigned int v0 = i0 < nr ? sm.r_len[i0] : 0u;
                const unsigned int v1 = i1 < nr ? sm.r_len[i1] : 0u;
                unsigned int x = v0 + v1;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned int y = __shfl_up_sync(FULL, x, o);
                    if (lane >= o) x += y;
                }
                if (lane == 31) sm.wsum[wib] = x;
                __syncthreads();
                unsigned int pre = 0u;
                for (int w2 = 0; w2 < wib; ++w2) pre += sm.wsum[w2];
                x += pre;
                if (i0 < nr) sm.r_end[i0] = x - v1;
                if (i1 < nr) sm.r_end[i1] = x;
                unsigned int total = 0u;
                for (int w2 = 0; w2 < kCoopWarps; ++w2) total += sm.wsum[w2];
                __syncthreads();
                // the candidates, 32 per warp at a time; each thread keeps the
                // range of its last candidate and searches forward from it
                unsigned int r_own = 0u;
                for (unsigned int cb = 32u * wib; cb < total; cb += 32u * kCoopWarps) {
                    const unsigned int t = cb + lane;
                    bool pass = false;
                    float acc = 0.0f;
                    unsigned int pos = 0u;
                    if (t < total) {
                        if (sm.r_end[r_own] <= t) {
                            // first range ending past t, after r_own
                            unsigned int lo_r = r_own + 1u, hi_r = nr - 1u;
                            while (lo_r < hi_r) {
                                const unsigned int mid = (lo_r + hi_r) >> 1;
                                if (sm.r_end[mid] > t)
                                    hi_r = mid;
                                else
                                    lo_r = mid + 1u;
                            }
                            r_own = lo_r;
                        }
                        pos = sm.r_start[r_own] + (t - (sm.r_end[r_own] - sm.r_len[r_own]));
                        constexpr int P = row_floats(D);
                        Row<P> row;
                        row.load(a.rows, pos);
                        acc = sq_dist<D, P>(s.q, row);
                        const unsigned long long ek2 = tk.kth < gkth ? tk.kth : gkth;
                        pass = ek2 == kEmptyKey || acc <= __uint_as_float((unsigned)(ek2 >> 32));
                    }
                    if (__ballot_sync(FULL, pass)) {
                        const unsigned long long key =
                            pass ? ((unsigned long long)__float_as_uint(acc) << 32) |
                                       __ldg(a.rid + pos)
                                 : kEmptyKey;
                        offer(tk, key, lane, gkth);
                    }
                }
                __syncthreads();
            }
        }
        // merge the warps' lists into the block's buffer
#pragma unroll
        for (int i = 0; i < NS; ++i) sm.loc[wib][i * 32 + lane] = tk.s[i];
        __syncthreads();
        if (wib == 0) {
            // start from the block's buffer; the warps' lists hold only points
            // of this layer, so the merge has no duplicates
            TopK<NS> g;
            g.init(a.k);
#pragma unroll
            for (int i = 0; i < NS; ++i) g.s[i] = sm.top[i * 32 + lane];
            g.count = sm.count;
            g.refresh_kth();
            for (int w2 = 0; w2 < kCoopWarps; ++w2) {
                if (!(sm.loc[w2][0] < g.kth)) continue;  // sorted: nothing enters
                if constexpr (NS == 1) {
                    g.merge32(sm.loc[w2][lane], lane);
                } else {
                    for (int e = 0; e < 64; ++e) {
                        const unsigned long long xk = sm.loc[w2][e];
                        if (!(xk < g.kth)) break;  // the list is sorted
                        g.insert(xk, lane);
                    }
                }
            }
            bool changed = false;
#pragma unroll
            for (int i = 0; i < NS; ++i) changed |= g.s[i] != sm.top[i * 32 + lane];
            changed = __any_sync(FULL, changed);
            __syncwarp();
#pragma unroll
            for (int i = 0; i < NS; ++i) sm.top[i * 32 + lane] = g.s[i];
            if (lane == 0) {
                sm.count = g.count;
                sm.updated = changed ? 1 : 0;
            }
        }
        __syncthreads();
        const bool updated = sm.updated != 0;
        const bool full = sm.count == a.k;
        // the stop rule of Sec. III.B, or the certified one (compiled apart)
        if constexpr (EXACT) {
            if (full && certified(a, s, L, __uint_as_float((unsigned)(sm.top[a.k - 1] >> 32))))
                break;
        } else {
            if (full && !updated) break;
        }
        if (b.covers) break;
        if (a.max_layers > 0 && L - s.lmin + 1 >= a.max_layers) {
            limited = true;
            if (threadIdx.x == 0) atomicOr(a.status, kStatusLimit);
            break;
        }
        ++L;
    }
    if (wib == 0) {
        TopK<NS> g;
        g.init(a.k);
#pragma unroll
        for (int i = 0; i < NS; ++i) g.s[i] = sm.top[i * 32 + lane];
        g.count = sm.count;
        write_outputs(a, qid, g, limited, lane);
    }
    __syncthreads();
}

template <int D, int NS, bool DENSE, bool EXACT>
__global__ void __launch_bounds__(kCoopThreads, 1) heavy_kernel(const QueryArgs a)
{
    __shared__ CoopSmem sm;
    __shared__ unsigned int s_h;
    const unsigned int nheavy = *a.heavy_count;
    for (;;) {
        if (threadIdx.x == 0) s_h = atomicAdd(a.heavy_cursor, 1u);
        __syncthreads();
        const unsigned int h = s_h;
        __syncthreads();
        if (h >= nheavy) break;
        coop_query<D, NS, DENSE, EXACT>(a, (long long)a.heavy_list[h], sm);
    }
}

// ---------------------------------------------------------------------------
// Batched indexes: one persistent launch per dimension covers the queries of
// every index of that dimension.  Each query finds its index by binary search
// over the group's query offsets and runs the same walk with that index's
// arguments (read through L1 from the group's argument array).
// ---------------------------------------------------------------------------

__device__ __forceinline__ int group_index(const unsigned long long* qoff, int count,
                                           unsigned long long qi)
{
    int lo = 0, hi = count - 1;  // the last index whose first query is <= qi
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(qoff + mid) <= qi)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Every index of a group shares the dimension, the buffer width (k <= 32 or
// not), the table kind and the stop rule, so the walk is specialised as in
// the single-index kernel.
template <int D, int NS, bool DENSE, bool EXACT>
__global__ void __launch_bounds__(kThreads, (MinBlocks<D, NS>::value))
    batch_query_kernel(const BatchArgs g)
{
    __shared__ WarpSmem sm[kWarps];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const bool may_defer = g.heavy_list != nullptr;
    unsigned long long next = 0ull;
    if (lane == 0) next = atomicAdd(g.counter, 1ull);
    next = __shfl_sync(FULL, next, 0);
    while (next < g.total) {
        const unsigned long long qi = next;
        if (lane == 0) next = atomicAdd(g.counter, 1ull);
        const int i = group_index(g.qoff, g.count, qi);
        const QueryArgs& a = g.args[i];
        const long long qid = (long long)(qi - __ldg(g.qoff + i));
        const bool deferred =
            walk_query<D, NS, DENSE, EXACT, false>(a, qid, sm[wib], lane, may_defer);
        if (deferred && lane == 0) g.heavy_list[atomicAdd(g.heavy_count, 1u)] = (unsigned int)qi;
        next = __shfl_sync(FULL, next, 0);
    }
}

template <int D, int NS, bool DENSE, bool EXACT>
__global__ void __launch_bounds__(kCoopThreads, 1) batch_heavy_kernel(const BatchArgs g)
{
    __shared__ CoopSmem sm;
    __shared__ unsigned int s_h;
    const unsigned int nheavy = *g.heavy_count;
    for (;;) {
        if (threadIdx.x == 0) s_h = atomicAdd(g.heavy_cursor, 1u);
        __syncthreads();
        const unsigned int h = s_h;
        __syncthreads();
        if (h >= nheavy) break;
        const unsigned long long qi = g.heavy_list[h];
        const int i = group_index(g.qoff, g.count, qi);
        const QueryArgs& a = g.args[i];
        const long long qid = (long long)(qi - __ldg(g.qoff + i));
        coop_query<D, NS, DENSE, EXACT>(a, qid, sm);
    }
}

template <class Kernel>
int blocks_per_sm(Kernel k, int& cache, int threads = kThreads)
{
    if (cache == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k, threads, 0) != cudaSuccess ||
            v < 1)
            v = 1;
        cache = v;
    }
    return cache;
}

template <int D, int NS, bool DENSE, bool EXACT, bool COUNT>
cudaError_t launch_one(const QueryArgs& a, int sms, cudaStream_t s)
{
    static int per_sm = 0, per_sm_heavy = 0;
    long long blocks =
        (long long)sms * blocks_per_sm(query_kernel<D, NS, DENSE, EXACT, COUNT>, per_sm);
    const long long need = (a.m + kWarps - 1) / kWarps;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    query_kernel<D, NS, DENSE, EXACT, COUNT><<<(int)blocks, kThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    kernel_mark("search", s);
    if (e != cudaSuccess || a.heavy_list == nullptr || COUNT) return e;
    long long hb =
        (long long)sms *
        blocks_per_sm(heavy_kernel<D, NS, DENSE, EXACT>, per_sm_heavy, kCoopThreads);
    if (hb > a.m) hb = a.m;
    if (hb < 1) hb = 1;
    heavy_kernel<D, NS, DENSE, EXACT><<<(int)hb, kCoopThreads, 0, s>>>(a);
    count_launches(1);
    kernel_mark("coop", s);
    return cudaGetLastError();
}

template <int D, int NS, bool DENSE, bool EXACT>
cudaError_t launch_batch_one(const BatchArgs& g, int sms, cudaStream_t s)
{
    static int per_sm = 0, per_sm_heavy = 0;
    long long blocks =
        (long long)sms * blocks_per_sm(batch_query_kernel<D, NS, DENSE, EXACT>, per_sm);
    const long long need = (long long)((g.total + kWarps - 1) / kWarps);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    batch_query_kernel<D, NS, DENSE, EXACT><<<(int)blocks, kThreads, 0, s>>>(g);
    cudaError_t e = cudaGetLastError();
    kernel_mark(group_phase_name(D, NS, DENSE, EXACT, false), s);
    if (e != cudaSuccess || g.heavy_list == nullptr) return e;
    long long hb =
        (long long)sms *
        blocks_per_sm(batch_heavy_kernel<D, NS, DENSE, EXACT>, per_sm_heavy, kCoopThreads);
    if (hb > (long long)g.total) hb = (long long)g.total;
    if (hb < 1) hb = 1;
    batch_heavy_kernel<D, NS, DENSE, EXACT><<<(int)hb, kCoopThreads, 0, s>>>(g);
    count_launches(1);
    kernel_mark(group_phase_name(D, NS, DENSE, EXACT, true), s);
    return cudaGetLastError();
}

template <int D, bool EXACT, bool COUNT>
cudaError_t launch_rule(const QueryArgs& a, int sms, cudaStream_t s)
{
    const bool two = a.k > 32;
    if (a.dense)
        return two ? launch_one<D, 2, true, EXACT, COUNT>(a, sms, s)
                   : launch_one<D, 1, true, EXACT, COUNT>(a, sms, s);
    return two ? launch_one<D, 2, false, EXACT, COUNT>(a, sms, s)
               : launch_one<D, 1, false, EXACT, COUNT>(a, sms, s);
}

// The stop rule and the counting walk are compile-time choices: the kernels
// of the paper's rule carry no code of the certified rule or of the counting
// walk (whose registers would spill theirs).  The counting walk exists for
// the paper's rule only.
template <int D>
cudaError_t launch_d(const QueryArgs& a, int sms, cudaStream_t s)
{
    if (a.stats) return a.exact ? cudaErrorInvalidValue : launch_rule<D, false, true>(a, sms, s);
    return a.exact ? launch_rule<D, true, false>(a, sms, s) : launch_rule<D, false, false>(a, sms, s);
}

template <int D, bool EXACT>
cudaError_t launch_batch_rule(const BatchArgs& g, int sms, cudaStream_t s)
{
    if (g.dense)
        return g.ns == 2 ? launch_batch_one<D, 2, true, EXACT>(g, sms, s)
                         : launch_batch_one<D, 1, true, EXACT>(g, sms, s);
    return g.ns == 2 ? launch_batch_one<D, 2, false, EXACT>(g, sms, s)
                     : launch_batch_one<D, 1, false, EXACT>(g, sms, s);
}

template <int D>
cudaError_t launch_batch_d(const BatchArgs& g, int sms, cudaStream_t s)
{
    return g.exact ? launch_batch_rule<D, true>(g, sms, s) : launch_batch_rule<D, false>(g, sms, s);
}

}  // namespace qk
}  // namespace ghn
