/*
 * GHN oracle: a plain, slow, single-threaded CPU statement of the grid-hashing
 * nearest-neighbour method ("GHN: Grid Hashing Neighborhood") and of exhaustive
 * KNN, written to check the CUDA library against.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  The product path never does,
 * and this file shares no code, header or constant with the CUDA library.
 *
 * What it follows (paper section / equation / algorithm):
 *   - Eq. 1 (Sec. III.A): a point's cell id is the point divided by the cell
 *     measurement with integer ("floor") division, per dimension.
 *   - Algorithm 1 (Sec. III.A): cell sampling; every training point is appended,
 *     in input order, to the list of its cell; empty cells are never stored.
 *   - Sec. III.B and Algorithm 2: exploration from the central cell, layer by
 *     layer; every point of a visited cell goes through a k-bounded buffer that
 *     keeps the k nearest; the walk stops after a layer that changed nothing in
 *     the buffer.
 *   - Sec. I and Sec. III.D: prediction by majority vote (classification) or
 *     mean (regression) of the k neighbours' outputs.
 *   - Sec. I: original KNN, an exhaustive scan followed by a sort.
 *
 * Readings of points the paper leaves open (each is listed with its reason in
 * the design notes of the repository):
 *   origin    per-dimension minimum of the training points (splits cover the
 *             range of values, Sec. III.A).
 *   widths    one cell measurement w_j per dimension (Sec. III.A: all cells
 *             have one shape, which need not be a cube); a scalar width is
 *             the case w_j = w for every j.
 *   splits    when a grid comes from the paper's cell measurement (s_j equal
 *             splits of each range, the last one closed), training cells are
 *             clamped to s_j - 1 so that the maximum lies in the last split;
 *             queries are not clamped to the splits.
 *   measure   per dimension, the largest s (at most 2^21) for which every
 *             one of the s splits holds a training point, a point's split
 *             being its Eq. 1 coordinate with w = r / s (r = max - min, single
 *             precision) clamped to s - 1; a dimension with r = 0 gets s = 1
 *             and w = 1.
 *   key       t = (p_j - o_j) / w in IEEE single precision, round to nearest,
 *             c_j = floor(t); a query clamps floor(t) to [-2^40, 2^40].
 *   layer L   the cells whose Chebyshev distance to the central cell is L
 *             (8 then 16 cells in 2-D, Eq. 2); only cells inside the bounding
 *             box of occupied cells can hold points, so only those are looked
 *             up; layers that miss that box entirely are empty and are passed
 *             over without enumeration.
 *   update    some point of layer L entered the buffer.
 *   stop      after layer L, when the buffer holds k points and layer L made
 *             no update, or when cube(L) covers the whole box (every later
 *             layer is empty, so the result cannot change).
 *   exact     (a certified variant of the stop, not the paper's rule): after
 *             layer L, stop when the buffer holds k points and the k-th
 *             squared distance is below the squared distance from the query
 *             to every cell outside cube(L) that the box can hold, less
 *             rounding margins; the result then equals exhaustive KNN.
 *   order     (squared distance, training index) ascending; squared distance
 *             in single precision, dimension order, no fused multiply-add
 *             (compile with -ffp-contract=off).
 *   fewer     if fewer than k points exist, all of them are returned; ids are
 *             padded with -1 and distances with +inf.
 *   vote      largest count, ties to the smallest label.
 *   mean      double-precision sum in neighbour order divided by the count,
 *             rounded to single precision.
 *   median    (Sec. I and Sec. III.D name the median beside the average) the
 *             outputs sorted by IEEE total order (-0 before +0); an odd count
 *             takes the middle one, an even count the two middle ones a <= b
 *             as (double(a) + double(b)) / 2 rounded to single precision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GHN_ORACLE_MAXD 8
#define GHN_ORACLE_QCLAMP 1099511627776.0f /* 2^40 */

/* One occupied cell: its coordinate vector and its points in append order. */
typedef struct {
    int64_t c[GHN_ORACLE_MAXD];
    int32_t* members;
    int64_t count;
    int64_t cap;
    int64_t next; /* next cell in the same hash bucket, -1 at the end */
} oracle_cell;

typedef struct {
    int32_t d;
    float w[GHN_ORACLE_MAXD];       /* cell measurement per dimension */
    int64_t split[GHN_ORACLE_MAXD]; /* training cells clamped to split - 1 (0: no clamp) */
    int64_t n;
    float origin[GHN_ORACLE_MAXD];
    int64_t cmax[GHN_ORACLE_MAXD]; /* largest cell coordinate per dimension */
    float* points;                  /* copy of the training points, n*d */
    uint32_t* labels;               /* copy of the 32-bit outputs, n, or NULL */
    oracle_cell* cells;             /* occupied cells in creation order */
    int64_t ncells;
    int64_t cellcap;
    int64_t* bucket; /* head cell of each bucket, -1 if empty */
    int64_t nbucket; /* power of two */
} ghn_oracle;

/* ---- the hash table of Algorithm 1 (a dictionary keyed by the cell id) ---- */

static uint64_t hash_coords(const int64_t* c, int32_t d)
{
    uint64_t h = 1469598103934665603ull; /* FNV-1a over the coordinate bytes */
    for (int32_t j = 0; j < d; ++j) {
        uint64_t v = (uint64_t)c[j];
        for (int b = 0; b < 8; ++b) {
            h ^= (v >> (8 * b)) & 0xffu;
            h *= 1099511628211ull;
        }
    }
    return h;
}

static int same_coords(const int64_t* a, const int64_t* b, int32_t d)
{
    for (int32_t j = 0; j < d; ++j)
        if (a[j] != b[j]) return 0;
    return 1;
}

/* Index of the cell with coordinates c, or -1 when that cell is not stored. */
static int64_t find_cell(const ghn_oracle* g, const int64_t* c)
{
    uint64_t h = hash_coords(c, g->d) & (uint64_t)(g->nbucket - 1);
    for (int64_t e = g->bucket[h]; e >= 0; e = g->cells[e].next)
        if (same_coords(g->cells[e].c, c, g->d)) return e;
    return -1;
}

/* Eq. 1 for a training point: c_j = floor((p_j - o_j) / w_j), single
   precision; clamped into the last split when the grid has splits. */
static void training_cell(const ghn_oracle* g, const float* p, int64_t* c)
{
    for (int32_t j = 0; j < g->d; ++j) {
        float t = (p[j] - g->origin[j]) / g->w[j];
        c[j] = (int64_t)floorf(t);
        if (g->split[j] > 0 && c[j] > g->split[j] - 1) c[j] = g->split[j] - 1;
    }
}

/* Eq. 1 for a query; far queries are clamped so the coordinate fits int64. */
static void query_cell(const ghn_oracle* g, const float* q, int64_t* c)
{
    for (int32_t j = 0; j < g->d; ++j) {
        float t = floorf((q[j] - g->origin[j]) / g->w[j]);
        if (t < -GHN_ORACLE_QCLAMP) t = -GHN_ORACLE_QCLAMP;
        if (t > GHN_ORACLE_QCLAMP) t = GHN_ORACLE_QCLAMP;
        c[j] = (int64_t)t;
    }
}

/* Double the cell array and the bucket array; re-chain every stored cell. */
static int grow_cells(ghn_oracle* g)
{
    oracle_cell* cells =
        (oracle_cell*)realloc(g->cells, sizeof(oracle_cell) * (size_t)(2 * g->cellcap));
    if (!cells) return 1;
    g->cells = cells;
    memset(cells + g->cellcap, 0, sizeof(oracle_cell) * (size_t)g->cellcap);
    g->cellcap *= 2;
    int64_t* bucket = (int64_t*)realloc(g->bucket, sizeof(int64_t) * (size_t)(2 * g->cellcap));
    if (!bucket) return 1;
    g->bucket = bucket;
    g->nbucket = 2 * g->cellcap;
    for (int64_t b = 0; b < g->nbucket; ++b) g->bucket[b] = -1;
    for (int64_t e = 0; e < g->ncells; ++e) {
        uint64_t h = hash_coords(g->cells[e].c, g->d) & (uint64_t)(g->nbucket - 1);
        g->cells[e].next = g->bucket[h];
        g->bucket[h] = e;
    }
    return 0;
}

void oracle_free(ghn_oracle* g)
{
    if (!g) return;
    for (int64_t e = 0; e < g->ncells; ++e) free(g->cells[e].members);
    free(g->cells);
    free(g->bucket);
    free(g->points);
    free(g->labels);
    free(g);
}

/*
 * Cell sampling (Algorithm 1).  points: n*d row-major floats; labels: n
 * 32-bit outputs (int32 classes or float targets, kept as raw bits) or NULL;
 * widths: d cell measurements; splits: d split counts (training cells are
 * clamped to split - 1) or NULL.  Returns 0 on success, 1 on bad arguments
 * (n < 1, d outside 1..8, a width not a positive finite number, a split
 * below 1, a non-finite coordinate), 2 when out of memory.
 */
int oracle_build_grid(const float* points, const uint32_t* labels, int64_t n, int32_t d,
                      const float* widths, const int64_t* splits, ghn_oracle** out)
{
    *out = NULL;
    if (n < 1 || d < 1 || d > GHN_ORACLE_MAXD) return 1;
    for (int32_t j = 0; j < d; ++j) {
        if (!(widths[j] > 0.0f) || !isfinite(widths[j])) return 1;
        if (splits && splits[j] < 1) return 1;
    }
    for (int64_t i = 0; i < n * d; ++i)
        if (!isfinite(points[i])) return 1;

    ghn_oracle* g = (ghn_oracle*)calloc(1, sizeof(ghn_oracle));
    if (!g) return 2;
    g->d = d;
    for (int32_t j = 0; j < d; ++j) {
        g->w[j] = widths[j];
        g->split[j] = splits ? splits[j] : 0;
    }
    g->n = n;
    g->points = (float*)malloc(sizeof(float) * (size_t)(n * d));
    g->cellcap = 1024;
    g->cells = (oracle_cell*)calloc((size_t)g->cellcap, sizeof(oracle_cell));
    g->nbucket = 2048;
    g->bucket = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->nbucket);
    if (labels) g->labels = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    if (!g->points || !g->cells || !g->bucket || (labels && !g->labels)) {
        oracle_free(g);
        return 2;
    }
    memcpy(g->points, points, sizeof(float) * (size_t)(n * d));
    if (labels) memcpy(g->labels, labels, sizeof(uint32_t) * (size_t)n);
    for (int64_t b = 0; b < g->nbucket; ++b) g->bucket[b] = -1;

    /* the grid's origin: the smallest value of each feature */
    for (int32_t j = 0; j < d; ++j) {
        float lo = points[j], hi = points[j];
        for (int64_t i = 1; i < n; ++i) {
            if (points[i * d + j] < lo) lo = points[i * d + j];
            if (points[i * d + j] > hi) hi = points[i * d + j];
        }
        g->origin[j] = lo;
        g->cmax[j] = 0;
        /* refuse grids whose cell coordinates would not fit an int64 */
        if (!((hi - lo) / widths[j] < 4611686018427387904.0f)) {
            oracle_free(g);
            return 1;
        }
    }

    /* for each point: compute its cell id, create the cell if absent, append */
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[GHN_ORACLE_MAXD];
        training_cell(g, points + i * d, c);
        int64_t e = find_cell(g, c);
        if (e < 0) {
            if (g->ncells == g->cellcap && grow_cells(g)) {
                oracle_free(g);
                return 2;
            }
            e = g->ncells++;
            oracle_cell* cell = &g->cells[e];
            memcpy(cell->c, c, sizeof(int64_t) * (size_t)d);
            uint64_t h = hash_coords(c, d) & (uint64_t)(g->nbucket - 1);
            cell->next = g->bucket[h];
            g->bucket[h] = e;
        }
        oracle_cell* cell = &g->cells[e];
        if (cell->count == cell->cap) {
            int64_t cap = cell->cap ? 2 * cell->cap : 4;
            int32_t* m = (int32_t*)realloc(cell->members, sizeof(int32_t) * (size_t)cap);
            if (!m) {
                oracle_free(g);
                return 2;
            }
            cell->members = m;
            cell->cap = cap;
        }
        cell->members[cell->count++] = (int32_t)i;
        for (int32_t j = 0; j < d; ++j)
            if (c[j] > g->cmax[j]) g->cmax[j] = c[j];
    }
    *out = g;
    return 0;
}

/* ---- the cell measurement of Sec. III.A ---- */

static int cmp_float(const void* a, const void* b)
{
    float x = *(const float*)a, y = *(const float*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Split of value v among s splits of width w from lo (Eq. 1, the last split closed). */
static int64_t split_of(float v, float lo, float w, int64_t s)
{
    float t = floorf((v - lo) / w);
    if (!(t < (float)s)) return s - 1;
    return (int64_t)t;
}

#define GHN_ORACLE_MAX_SPLITS 2097152 /* 2^21 */

/*
 * Per dimension, the largest number of equal splits of the range of values
 * such that every split holds at least one training point (Sec. III.A, the
 * "cell measurements"); the width is range / splits.  Candidates go from
 * min(distinct values, 2^21) down; the first one whose splits are all
 * occupied wins (a split is occupied when some value lands in it; the values
 * are visited in increasing order, so it suffices that consecutive distinct
 * values never skip a split and that the largest lands in the last one).
 * splits, widths: d entries each.  Returns 0, 1 on bad arguments, 2 when out
 * of memory.
 */
int oracle_measure(const float* points, int64_t n, int32_t d, int64_t* splits, float* widths)
{
    if (n < 1 || d < 1 || d > GHN_ORACLE_MAXD) return 1;
    for (int64_t i = 0; i < n * d; ++i)
        if (!isfinite(points[i])) return 1;
    float* v = (float*)malloc(sizeof(float) * (size_t)n);
    if (!v) return 2;
    for (int32_t j = 0; j < d; ++j) {
        for (int64_t i = 0; i < n; ++i) v[i] = points[i * d + j];
        qsort(v, (size_t)n, sizeof(float), cmp_float);
        int64_t u = 0; /* distinct values, in place */
        for (int64_t i = 0; i < n; ++i)
            if (u == 0 || v[i] != v[u - 1]) v[u++] = v[i];
        float lo = v[0], r = v[u - 1] - v[0];
        splits[j] = 1;
        widths[j] = 1.0f;
        if (!(r > 0.0f)) continue; /* one value: one split */
        int64_t s = u < GHN_ORACLE_MAX_SPLITS ? u : GHN_ORACLE_MAX_SPLITS;
        for (; s >= 1; --s) {
            float w = r / (float)s;
            if (!(w > 0.0f)) continue;
            int ok = split_of(v[u - 1], lo, w, s) == s - 1;
            int64_t prev = split_of(v[0], lo, w, s);
            ok = ok && prev == 0;
            for (int64_t i = 1; ok && i < u; ++i) {
                int64_t c = split_of(v[i], lo, w, s);
                if (c - prev > 1) ok = 0;
                prev = c;
            }
            if (ok) {
                splits[j] = s;
                widths[j] = w;
                break;
            }
        }
    }
    free(v);
    return 0;
}

/* Cell sampling with one width w for every dimension and no splits. */
int oracle_build(const float* points, const uint32_t* labels, int64_t n, int32_t d, float w,
                 ghn_oracle** out)
{
    float widths[GHN_ORACLE_MAXD];
    *out = NULL;
    if (d < 1 || d > GHN_ORACLE_MAXD) return 1;
    for (int32_t j = 0; j < d; ++j) widths[j] = w;
    return oracle_build_grid(points, labels, n, d, widths, NULL, out);
}

/* ---- the k-bounded buffer (kept sorted by (distance, index)) ---- */

typedef struct {
    float dist;
    int32_t id;
} oracle_entry;

static int entry_less(float da, int32_t ia, float db, int32_t ib)
{
    return da < db || (da == db && ia < ib);
}

/* Offer one point; returns 1 when it entered the buffer. */
static int buffer_offer(oracle_entry* buf, int32_t* size, int32_t k, float dist, int32_t id)
{
    if (*size == k && !entry_less(dist, id, buf[k - 1].dist, buf[k - 1].id)) return 0;
    int32_t pos = (*size < k) ? *size : k - 1;
    while (pos > 0 && entry_less(dist, id, buf[pos - 1].dist, buf[pos - 1].id)) {
        buf[pos] = buf[pos - 1];
        --pos;
    }
    buf[pos].dist = dist;
    buf[pos].id = id;
    if (*size < k) ++*size;
    return 1;
}

/* Squared Euclidean distance, single precision, dimension order, no FMA. */
static float squared_distance(const float* q, const float* p, int32_t d)
{
    float acc = 0.0f;
    for (int32_t j = 0; j < d; ++j) {
        float t = q[j] - p[j];
        float s = t * t;
        acc = acc + s;
    }
    return acc;
}

/* ---- layer enumeration ---- */

/*
 * Visit every cell c with lo <= c <= hi (per dimension) whose Chebyshev
 * distance to centre is exactly L, odometer style, last dimension fastest.
 * visit() returns nonzero to abort.  Returns the number of cells visited.
 */
typedef int (*cell_visitor)(const int64_t* c, void* ctx);

static int64_t for_each_shell_cell(int32_t d, const int64_t* centre, int64_t L, const int64_t* lo,
                                   const int64_t* hi, cell_visitor visit, void* ctx)
{
    int64_t c[GHN_ORACLE_MAXD];
    int64_t visited = 0;
    for (int32_t j = 0; j < d; ++j) {
        if (lo[j] > hi[j]) return 0;
        c[j] = lo[j];
    }
    for (;;) {
        int64_t cheb = 0;
        for (int32_t j = 0; j < d; ++j) {
            int64_t a = c[j] - centre[j];
            if (a < 0) a = -a;
            if (a > cheb) cheb = a;
        }
        if (cheb == L) {
            ++visited;
            if (visit && visit(c, ctx)) return visited;
        }
        int32_t j = d - 1;
        while (j >= 0 && c[j] == hi[j]) {
            c[j] = lo[j];
            --j;
        }
        if (j < 0) break;
        ++c[j];
    }
    return visited;
}

/*
 * Number of cells on layer L of an unbounded d-dimensional grid, counted by
 * the same enumerator the exploration uses (Eq. 2 gives the closed form).
 */
int64_t oracle_shell_count(int32_t d, int64_t L)
{
    int64_t centre[GHN_ORACLE_MAXD], lo[GHN_ORACLE_MAXD], hi[GHN_ORACLE_MAXD];
    if (d < 1 || d > GHN_ORACLE_MAXD || L < 0) return -1;
    for (int32_t j = 0; j < d; ++j) {
        centre[j] = 0;
        lo[j] = -L;
        hi[j] = L;
    }
    return for_each_shell_cell(d, centre, L, lo, hi, NULL, NULL);
}

/* ---- exploration (Sec. III.B, Algorithm 2) ---- */

typedef struct {
    const ghn_oracle* g;
    const float* q;
    oracle_entry* buf;
    int32_t size;
    int32_t k;
    int updated;
    int64_t cells; /* occupied cells looked up */
    int64_t cands; /* points examined */
} explore_ctx;

static int visit_cell(const int64_t* c, void* vctx)
{
    explore_ctx* x = (explore_ctx*)vctx;
    int64_t e = find_cell(x->g, c);
    if (e < 0) return 0; /* empty cells are not stored (Sec. III.A) */
    const oracle_cell* cell = &x->g->cells[e];
    x->cells++;
    for (int64_t t = 0; t < cell->count; ++t) {
        int32_t i = cell->members[t];
        float dist = squared_distance(x->q, x->g->points + (int64_t)i * x->g->d, x->g->d);
        x->cands++;
        if (buffer_offer(x->buf, &x->size, x->k, dist, i)) x->updated = 1;
    }
    return 0;
}

/* IEEE total-order key of a float: unsigned comparison of keys orders
   -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN. */
static uint32_t total_order_key(float v)
{
    uint32_t u;
    memcpy(&u, &v, sizeof u);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

static int cmp_total_order(const void* a, const void* b)
{
    uint32_t x = total_order_key(*(const float*)a), y = total_order_key(*(const float*)b);
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Median of the outputs of the first `size` buffer entries (NaN when empty). */
static float median_of(const ghn_oracle* g, const oracle_entry* buf, int32_t size)
{
    if (size == 0) return NAN;
    float* v = (float*)malloc(sizeof(float) * (size_t)size);
    if (!v) return NAN;
    for (int32_t r = 0; r < size; ++r) memcpy(&v[r], &g->labels[buf[r].id], sizeof(float));
    qsort(v, (size_t)size, sizeof(float), cmp_total_order);
    float out;
    if (size % 2)
        out = v[size / 2];
    else
        out = (float)(((double)v[size / 2 - 1] + (double)v[size / 2]) / 2.0);
    free(v);
    return out;
}

/*
 * The certified stop: after cube(L) has been visited, can a point outside it
 * still enter a full buffer whose k-th squared distance is kth?  A training
 * point in a cell beyond c0_j + L along axis j lies at or above
 * o_j + (c0_j + L + 1) w_j, less the rounding of Eq. 1 (at most a relative
 * 2^-23 of the quotient, taken here as 2^-21); below c0_j - L it lies under
 * o_j + (c0_j - L) w_j plus that margin.  Sides where the box holds no cell
 * beyond cube(L) do not count.  The smallest such gap bounds the distance of
 * every point not yet seen; its single-precision squared distance is at least
 * gap^2 (1 - 2^-20) (d + 2 roundings of 2^-24 each).  Stop when kth is below
 * that.
 */
static int certified(const ghn_oracle* g, const float* q, const int64_t* c0, int64_t L, float kth)
{
    double gap = INFINITY;
    for (int32_t j = 0; j < g->d; ++j) {
        double w = (double)g->w[j], o = (double)g->origin[j], qj = (double)q[j];
        if (c0[j] + L < g->cmax[j]) {
            double cu = (double)(c0[j] + L + 1);
            double edge = o + cu * w - fabs(cu) * w * 0x1p-21;
            double up = edge - qj;
            if (up < gap) gap = up;
        }
        if (c0[j] - L > 0) {
            double cl = (double)(c0[j] - L);
            double edge = o + cl * w + fabs(cl) * w * 0x1p-21;
            double down = qj - edge;
            if (down < gap) gap = down;
        }
    }
    if (!(gap > 0.0)) return 0;
    return (double)kth < gap * gap * (1.0 - 0x1p-20);
}

/*
 * Predict one query.  ids[k] / dist2[k] receive the neighbours in
 * (distance, index) order, padded with -1 / +inf.  mode 0 = vote (labels read
 * as int32, pred is int32), mode 1 = mean and mode 2 = median (labels read as
 * float, pred is float), mode -1 = no prediction.  stats (may be NULL) receives
 * {layers visited (L* + 1), occupied cells looked up, points examined}.
 * stop_rule: 1 the paper's rule (Sec. III.B); 2 the certified stop (the
 * result equals exhaustive KNN); 0 no stop rule (the walk ends only when the
 * cube covers the box: exhaustive search).
 * Returns 0, or 1 on bad arguments.
 */
int oracle_query_ex(const ghn_oracle* g, const float* q, int32_t k, int32_t mode, int32_t stop_rule,
                    int32_t* ids, float* dist2, void* pred, int64_t* stats)
{
    if (!g || k < 1 || (mode >= 0 && !g->labels) || mode > 2) return 1;
    for (int32_t j = 0; j < g->d; ++j)
        if (!isfinite(q[j])) return 1;
    int32_t d = g->d;
    oracle_entry* buf = (oracle_entry*)malloc(sizeof(oracle_entry) * (size_t)k);
    if (!buf) return 1;

    int64_t c0[GHN_ORACLE_MAXD];
    query_cell(g, q, c0);

    /* layers nearer than the box of occupied cells hold no cell: start at the
       first layer that reaches it */
    int64_t L = 0;
    for (int32_t j = 0; j < d; ++j) {
        int64_t gap = 0;
        if (c0[j] < 0) gap = -c0[j];
        if (c0[j] > g->cmax[j]) gap = c0[j] - g->cmax[j];
        if (gap > L) L = gap;
    }

    explore_ctx x;
    x.g = g;
    x.q = q;
    x.buf = buf;
    x.size = 0;
    x.k = k;
    x.cells = 0;
    x.cands = 0;
    for (;; ++L) {
        int64_t lo[GHN_ORACLE_MAXD] = {0}, hi[GHN_ORACLE_MAXD] = {0};
        int covers = 1;
        for (int32_t j = 0; j < d; ++j) {
            lo[j] = c0[j] - L < 0 ? 0 : c0[j] - L;
            hi[j] = c0[j] + L > g->cmax[j] ? g->cmax[j] : c0[j] + L;
            if (c0[j] - L > 0 || c0[j] + L < g->cmax[j]) covers = 0;
        }
        x.updated = 0;
        for_each_shell_cell(d, c0, L, lo, hi, visit_cell, &x);
        if (stop_rule == 1 && x.size == k && !x.updated) break;
        if (stop_rule == 2 && x.size == k && certified(g, q, c0, L, buf[k - 1].dist)) break;
        if (covers) break;
    }

    for (int32_t r = 0; r < k; ++r) {
        ids[r] = r < x.size ? buf[r].id : -1;
        dist2[r] = r < x.size ? buf[r].dist : INFINITY;
    }
    if (mode == 0) {
        /* majority class, ties to the smallest label */
        int32_t best = 0, bestc = 0;
        for (int32_t r = 0; r < x.size; ++r) {
            int32_t lab = (int32_t)g->labels[buf[r].id], cnt = 0;
            for (int32_t s = 0; s < x.size; ++s)
                if ((int32_t)g->labels[buf[s].id] == lab) ++cnt;
            if (cnt > bestc || (cnt == bestc && lab < best)) {
                best = lab;
                bestc = cnt;
            }
        }
        *(int32_t*)pred = best;
    } else if (mode == 1) {
        /* average of the neighbours' outputs */
        double sum = 0.0;
        for (int32_t r = 0; r < x.size; ++r) {
            float y;
            memcpy(&y, &g->labels[buf[r].id], sizeof(float));
            sum += (double)y;
        }
        *(float*)pred = x.size ? (float)(sum / (double)x.size) : NAN;
    } else if (mode == 2) {
        *(float*)pred = median_of(g, buf, x.size);
    }
    if (stats) {
        stats[0] = L + 1;
        stats[1] = x.cells;
        stats[2] = x.cands;
    }
    free(buf);
    return 0;
}

/* A batch of m queries (q is m*d) under a stop rule (as oracle_query_ex);
   outputs m*k / m, stats m*3 (may be NULL). */
int oracle_query_rule(const ghn_oracle* g, const float* q, int64_t m, int32_t k, int32_t mode,
                      int32_t stop_rule, int32_t* ids, float* dist2, void* pred, int64_t* stats)
{
    for (int64_t i = 0; i < m; ++i) {
        void* p = pred ? (void*)((uint32_t*)pred + i) : NULL;
        int rc = oracle_query_ex(g, q + i * g->d, k, mode, stop_rule, ids + i * k, dist2 + i * k,
                                 mode >= 0 ? p : NULL, stats ? stats + 3 * i : NULL);
        if (rc) return rc;
    }
    return 0;
}

/* A batch of m queries under the paper's stop rule. */
int oracle_query(const ghn_oracle* g, const float* q, int64_t m, int32_t k, int32_t mode,
                 int32_t* ids, float* dist2, void* pred, int64_t* stats)
{
    return oracle_query_rule(g, q, m, k, mode, 1, ids, dist2, pred, stats);
}

/* ---- original KNN (Sec. I): scan everything, then sort ---- */

typedef struct {
    float dist;
    int32_t id;
} brute_entry;

static int brute_cmp(const void* a, const void* b)
{
    const brute_entry* x = (const brute_entry*)a;
    const brute_entry* y = (const brute_entry*)b;
    if (entry_less(x->dist, x->id, y->dist, y->id)) return -1;
    if (entry_less(y->dist, y->id, x->dist, x->id)) return 1;
    return 0;
}

int oracle_brute(const float* points, int64_t n, int32_t d, const float* q, int64_t m, int32_t k,
                 int32_t* ids, float* dist2)
{
    if (n < 1 || d < 1 || d > GHN_ORACLE_MAXD || k < 1) return 1;
    brute_entry* all = (brute_entry*)malloc(sizeof(brute_entry) * (size_t)n);
    if (!all) return 2;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t t = 0; t < n; ++t) {
            all[t].dist = squared_distance(q + i * d, points + t * d, d);
            all[t].id = (int32_t)t;
        }
        qsort(all, (size_t)n, sizeof(brute_entry), brute_cmp);
        for (int32_t r = 0; r < k; ++r) {
            ids[i * k + r] = r < n ? all[r].id : -1;
            dist2[i * k + r] = r < n ? all[r].dist : INFINITY;
        }
    }
    free(all);
    return 0;
}

/* ---- inspection, for the invariant tests ---- */

int64_t oracle_num_cells(const ghn_oracle* g) { return g->ncells; }

void oracle_origin(const ghn_oracle* g, float* origin, int64_t* cmax)
{
    for (int32_t j = 0; j < g->d; ++j) {
        origin[j] = g->origin[j];
        cmax[j] = g->cmax[j];
    }
}

/*
 * Copy out the cells: coords (ncells*d), counts (ncells) and members (n, the
 * member lists one after another in cell-creation order).
 */
void oracle_cells(const ghn_oracle* g, int64_t* coords, int64_t* counts, int32_t* members)
{
    int64_t off = 0;
    for (int64_t e = 0; e < g->ncells; ++e) {
        const oracle_cell* cell = &g->cells[e];
        for (int32_t j = 0; j < g->d; ++j) coords[e * g->d + j] = cell->c[j];
        counts[e] = cell->count;
        memcpy(members + off, cell->members, sizeof(int32_t) * (size_t)cell->count);
        off += cell->count;
    }
}

/* Cell coordinates of m points (training rule: no clamp) or queries (clamped). */
void oracle_cells_of(const ghn_oracle* g, const float* p, int64_t m, int32_t as_query, int64_t* c)
{
    for (int64_t i = 0; i < m; ++i) {
        if (as_query)
            query_cell(g, p + i * g->d, c + i * g->d);
        else
            training_cell(g, p + i * g->d, c + i * g->d);
    }
}

/* Number of occupied cells for width w, without keeping the grid (width search). */
int64_t oracle_count_cells(const float* points, int64_t n, int32_t d, float w)
{
    ghn_oracle* g = NULL;
    if (oracle_build(points, NULL, n, d, w, &g)) return -1;
    int64_t u = g->ncells;
    oracle_free(g);
    return u;
}
