// Grid kNN search and adaptive power (Sec. 3.2.4 / 4.1.4 and Eq. 2-6 of
// arXiv 1601.05904).
//
// One thread per query, as in the paper.  The thread locates the query's
// cell, then visits square rings of cells L = 0, 1, 2, ... around it.  Cells
// of one grid row are consecutive in the cell-ordered point array, so the
// top and bottom edges of a ring are each one contiguous range of points and
// the side columns are one cell each.  Candidates go through a register
// top-k on squared distances (no square roots until the end, Sec. 4.1.4),
// ordered by (d^2, original index).
//
// Stop rule.  The paper grows the ring until the block holds k points and
// then adds one more level (Sec. 3.2.4, remark on Fig. 4).  That is not
// exact: after the block first holds k points the k-th distance can reach
// (L+1)*sqrt(2)*cw while one more ring only guarantees (L+1)*cw.  Here the
// search stops after ring L only when the nearest point the block excludes
// (the distance from the query to the block's nearest outer edge) is
// farther than the current k-th distance, with a relative margin that covers
// the rounding of the float32 distances and of the cell assignment.  Sides
// of the block that reach the edge of the grid exclude nothing.  The
// paper's own rule is kept as an option (kStopPaperLevel, used by
// aidw_knn_paper_rule) to measure how often it misses a neighbour.
//
// After the search the thread computes r_obs (Eq. 3), R (Eq. 4), mu (Eq. 5)
// and alpha (Eq. 6) - in float64 on the float64 path; on the float32 path
// r_obs as a compensated float32 sum of float32 square roots and Eq. 4-6 in
// float32 - and writes one record for the weighting stage: alpha, the
// smallest squared distance and the mean z of data points at distance 0
// (the limit of Eq. 1 when the query coincides with data).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "aidw_device.cuh"
#include "aidw_internal.cuh"
#include "grid_device.cuh"

namespace aidw {

namespace {

constexpr int kKnnThreads = 128;      // single-job launches
constexpr int kKnnMaxThreads = 256;   // largest block of batched launches

template <bool F64>
struct DistT;
template <>
struct DistT<false> {
    using T = float;
    static __device__ __forceinline__ float d2(float qx, float qy, float px, float py)
    {
        return dist2_f32(qx, qy, px, py);
    }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};
template <>
struct DistT<true> {
    using T = double;
    static __device__ __forceinline__ double d2(float qx, float qy, float px, float py)
    {
        return dist2_f64(qx, qy, px, py);
    }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000LL); }
};

// Job whose flat query range [q_base, q_base + nq) contains gq.
__device__ __forceinline__ int knn_job_of(const KnnJob *__restrict__ jobs, int n_jobs,
                                          long long gq)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].q_base <= gq)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Sum of z over the points at distance 0 (the limit of Eq. 1 when a query
// coincides with data): float64 in the float64 path; a TwoSum-compensated
// float32 pair in the float32 path, so that the test on every candidate,
// which the compiler may predicate rather than branch around, issues no
// float64 instruction there.
template <bool F64>
struct HitSum;
template <>
struct HitSum<true> {
    double s = 0.0;
    __device__ __forceinline__ void add(float z) { s += (double)z; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct HitSum<false> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float z) { comp_add(hi, lo, z); }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Stop-rule bounds.  The distance from the query to the outer edge of the
// level-L block on one side is its distance to that edge of its own cell
// plus L cell widths.  The four own-cell distances are lower bounds taken
// once per query in float32 with directed rounding (edge positions rounded
// away from the query, cw rounded down), less a margin for the float64
// rounding of the points' cell assignment (a point of column c lies at
// least c * cw * 2^-52 short of its cell's edge); each ring then steps them
// with round-down arithmetic.  Every value is a lower bound of the true
// edge distance, so the stop test can only be late, never early.
struct EdgeBounds {
    float l, r, b, t, cw;
};

__device__ __forceinline__ EdgeBounds edge_bounds(float qx, float qy, const GridDev *g, int col,
                                                  int row)
{
    // The margin is at least the smallest normal float32 (results flushed to
    // zero are off by less than that); integer -> float conversions are
    // rounded in the safe direction too, so the bounds also hold for grids
    // of more than 2^24 cells per side.
    const float margin = fmaxf(
        __fmul_ru(__fmul_ru(__ll2float_ru(g->n_col + g->n_row + 2), g->cw_ru), 0x1p-50f),
        0x1p-126f);
    EdgeBounds e;
    e.l = __fsub_rd(__fsub_rd(qx, __fmaf_ru(__int2float_ru(col), g->cw_ru, g->min_x_f)), margin);
    e.r = __fsub_rd(__fsub_rd(__fmaf_rd(__int2float_rd(col + 1), g->cw_rd, g->min_x_f), qx),
                    margin);
    e.b = __fsub_rd(__fsub_rd(qy, __fmaf_ru(__int2float_ru(row), g->cw_ru, g->min_y_f)), margin);
    e.t = __fsub_rd(__fsub_rd(__fmaf_rd(__int2float_rd(row + 1), g->cw_rd, g->min_y_f), qy),
                    margin);
    e.cw = g->cw_rd;
    return e;
}

// True when no point outside the level-L block (sides that reach the grid's
// edge exclude nothing) can come before the current k-th entry: the block's
// nearest open edge, squared and shrunk by a relative 2^-20 that covers the
// rounding of the float32 squared distances, is beyond the k-th distance.
template <typename D>
__device__ __forceinline__ bool block_is_final(const EdgeBounds &e, float Lf, bool full_l,
                                               bool full_r, bool full_b, bool full_t, D kth)
{
    const float inf = __int_as_float(0x7f800000);
    const float step = __fmul_rd(Lf, e.cw);
    float dmin = inf;
    if (!full_l) dmin = fminf(dmin, __fadd_rd(e.l, step));
    if (!full_r) dmin = fminf(dmin, __fadd_rd(e.r, step));
    if (!full_b) dmin = fminf(dmin, __fadd_rd(e.b, step));
    if (!full_t) dmin = fminf(dmin, __fadd_rd(e.t, step));
    return dmin > 0.0f && (D)__fmul_rd(__fmul_rd(dmin, dmin), 0.99999904632568359375f) > kth;
}

// Eq. 3-6 for the float32 path, whose weights take alpha rounded to
// float32: r_obs as a TwoSum-compensated float32 sum of correctly rounded
// float32 square roots, R, the Eq. 5 cosine and Eq. 6 in float32 (alpha
// within a few float32 ulps; the float64 path evaluates Eq. 3-6 in float64,
// which on this GPU costs as much as the whole ring search).  Edge cases as
// nn_statistic / membership / decay_power.
template <int KMAX, typename D>
__device__ __forceinline__ float robs_f32(const D (&kd)[KMAX], int lo, int k)
{
    float hi = 0.0f, err = 0.0f;  // entries kd[lo .. lo + k), ascending
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        if (j >= lo && j < lo + k) comp_add(hi, err, sqrtf((float)kd[j]));
    return __fdiv_rn(add_rn(hi, err), (float)k);
}

__device__ __forceinline__ float membership_f32(float r_obs, const GridDev *g,
                                                const AlphaParams &ap)
{
    const float r_exp = ap.area_override_f > 0.0f
                            ? 0.5f / sqrtf((float)g->n_data / ap.area_override_f)
                            : (float)g->r_exp;
    const float R = r_obs == 0.0f ? 0.0f
                                  : (r_exp == 0.0f ? __int_as_float(0x7f800000) : r_obs / r_exp);
    if (R <= ap.r_min_f) return 0.0f;
    if (R >= ap.r_max_f) return 1.0f;
    return 0.5f - 0.5f * cosf(ap.pi_over_rmax_f * (R - ap.r_min_f));
}

__device__ __forceinline__ float decay_power_f32(float mu, const float (&a)[5])
{
    if (mu <= 0.1f) return a[0];
    if (mu <= 0.3f) return a[0] * (1.0f - 5.0f * (mu - 0.1f)) + 5.0f * a[1] * (mu - 0.1f);
    if (mu <= 0.5f) return 5.0f * a[2] * (mu - 0.3f) + a[1] * (1.0f - 5.0f * (mu - 0.3f));
    if (mu <= 0.7f) return a[2] * (1.0f - 5.0f * (mu - 0.5f)) + 5.0f * a[3] * (mu - 0.5f);
    if (mu <= 0.9f) return 5.0f * a[4] * (mu - 0.7f) + a[3] * (1.0f - 5.0f * (mu - 0.7f));
    return a[4];
}

// Register budget of the float32 kNN kernel per top-k width: a minimum of
// 2 resident blocks of 256 threads holds it to 128 registers.  Left free,
// the compiler gives the 32/24/16/8-slot forms 174/164/148/128 registers.
// Measured on GB300 at 1M (kNN ms incl. query order; free 32-slot form:
// uniform k = 32 2.83): caps on (32, 24, 16, 8) = (2, 1, 1, 1): uniform
// k = 10 0.666, clustered k = 8/10/24/32 0.939/1.189/2.279/2.671, uniform
// k = 32 1.690, 512-job build + kNN 29.15; (2, 2, 1, 1): 0.667, 0.939/1.199/
// 1.951/2.666, 1.690, 28.1; (2, 2, 2, 2): 0.546, 0.931/1.018/1.948/2.668,
// 1.689, 26.9.  Three blocks (80 registers) spill.  The float64 path is
// left free (capping its 32-slot form spills heavily).  With 64-bit keys
// and the exit test on every eighth step the 32-slot form spills 52 bytes
// (68 bytes of reloads, from L1) at 128 registers and is still the fastest
// measured form (clustered k = 32 at 1M: 2.04 ms, against 2.15 ms with the
// test on every fourth step and no spill).
constexpr int kKnnMinBlocks32 = 2, kKnnMinBlocks24 = 2, kKnnMinBlocks16 = 2,
              kKnnMinBlocks8 = 2;
constexpr int knn_min_blocks(bool f64, int kmax)
{
    return f64 ? 1
               : (kmax >= 32 ? kKnnMinBlocks32
                             : (kmax >= 24 ? kKnnMinBlocks24
                                           : (kmax >= 16 ? kKnnMinBlocks16 : kKnnMinBlocks8)));
}

template <bool F64, int KMAX>
__global__ void __launch_bounds__(kKnnMaxThreads, knn_min_blocks(F64, KMAX))
    k_knn(KnnJob job0, const KnnJob *__restrict__ jobs, int n_jobs, long long total_q,
          AlphaParams ap)
{
    using D = typename DistT<F64>::T;
    const long long gq = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gq >= total_q) return;
    // single-job launches pass the job by value and no table
    const KnnJob J = jobs ? jobs[knn_job_of(jobs, n_jobs, gq)] : job0;
    const GridDev *__restrict__ g = J.g;
    // a grid whose build failed (non-finite data) has no usable cells and no
    // query order: its queries get NaN results in input order
    const bool failed = (g->status & (kStatusNonfiniteData | kStatusCapacity)) != 0;
    const long long li = gq - J.q_base;
    const long long q = (J.order && !failed) ? (long long)J.order[li] : li;
    if (!AIDW_IN(q, J.nq, bounds::kKnnOrder)) return;
    const Point *__restrict__ pts = J.pts;
    const int *__restrict__ start = J.start;
    const int k = J.k;
    QRec *__restrict__ recs = J.recs;
    int *__restrict__ out_idx = J.out_idx;
    float *__restrict__ out_dist = J.out_dist;
    float *__restrict__ out_robs = J.out_robs;
    void *__restrict__ out_alpha = J.out_alpha;
    const float qx = J.qx[q], qy = J.qy[q];
    const double nanv = __longlong_as_double(0x7ff8000000000000LL);

    if (failed || !isfinite(qx) || !isfinite(qy)) {
        if (!failed) atomicOr(const_cast<int *>(&g->status), kStatusNonfiniteQuery);
        if (recs) {
            QRec r;
            r.alpha = nanv;
            r.hit_z = nanv;
            r.d1sq = __int_as_float(0x7fc00000);
            r.n_hit = 0;
            recs[q] = r;
        }
        for (int j = 0; j < k; ++j) {
            if (out_idx) out_idx[q * k + j] = -1;
            if (out_dist) out_dist[q * k + j] = __int_as_float(0x7fc00000);
        }
        if (out_robs) out_robs[q] = __int_as_float(0x7fc00000);
        if (out_alpha) {
            if (F64)
                static_cast<double *>(out_alpha)[q] = nanv;
            else
                static_cast<float *>(out_alpha)[q] = __int_as_float(0x7fc00000);
        }
        if (J.out_zlocal) {
            if (F64)
                static_cast<double *>(J.out_zlocal)[q] = nanv;
            else
                static_cast<float *>(J.out_zlocal)[q] = __int_as_float(0x7fc00000);
        }
        return;
    }

    const double minx = g->min_x, miny = g->min_y, cw = g->cw;
    const int nc = (int)g->n_col, nr = (int)g->n_row;
    long long colw = gridk::cell_floor(qx, g->min_x_f, g->inv_cw_f, minx, cw);
    long long roww = gridk::cell_floor(qy, g->min_y_f, g->inv_cw_f, miny, cw);
    const int col = (int)(colw < 0 ? 0 : (colw > nc - 1 ? nc - 1 : colw));
    const int row = (int)(roww < 0 ? 0 : (roww > nr - 1 ? nr - 1 : roww));
    const EdgeBounds eb = edge_bounds(qx, qy, g, col, row);

    // The k best (d^2, index) pairs, ascending, in the top k slots
    // [lo, KMAX): the k-th is always kd[KMAX - 1].  The slots below lo hold
    // -inf sentinels, which stop a candidate that bubbles down from the top.
    const int lo = KMAX - k;
    D kd[KMAX];
    int ki[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        kd[j] = j < lo ? -DistT<F64>::inf() : DistT<F64>::inf();
        ki[j] = j < lo ? -1 : 0x7fffffff;
    }
    D kth = DistT<F64>::inf();
    int kthi = 0x7fffffff;
    // float32 path: the list as 64-bit keys (bits of d^2 << 32 | index).  A
    // non-negative float32 orders like its bit pattern, so one unsigned
    // compare of two keys is the (d^2, index) order; sentinels are key 0
    // below lo and the key of (+inf, INT_MAX) above.
    constexpr unsigned long long kEmptyKey = (0x7f800000ull << 32) | 0x7fffffffull;
    unsigned long long kk[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) kk[j] = j < lo ? 0ull : kEmptyKey;
    unsigned long long kth_key = kEmptyKey;
    long long found = 0;
    int L0 = -1;  // paper rule: the first level whose block holds k points

    for (int L = 0;; ++L) {
        // Ring L as segments of one grid row each: the bottom and top edges
        // (contiguous runs of cells) and the two side cells of every row in
        // between.  Segment index sg enumerates them.
        const int c0 = max(col - L, 0), c1 = min(col + L, nc - 1);
        const bool left_in = col - L >= 0, right_in = col + L <= nc - 1;
        const int r0 = max(row - L + 1, 0), r1 = min(row + L - 1, nr - 1);
        const int nside = (L > 0 && (left_in || right_in) && r1 >= r0) ? r1 - r0 + 1 : 0;
        const int nsegs = L == 0 ? 1 : 2 + 2 * nside;
        for (int sg = 0; sg < nsegs; ++sg) {
            int r, ca, cb;
            if (L == 0) {
                r = row;
                ca = cb = col;
            } else if (sg < 2) {
                r = sg == 0 ? row - L : row + L;
                if (r < 0 || r > nr - 1) continue;
                ca = c0;
                cb = c1;
            } else {
                const int e = sg - 2;
                r = r0 + (e >> 1);
                const bool right = (e & 1) != 0;
                if (right ? !right_in : !left_in) continue;
                ca = cb = right ? col + L : col - L;
            }
            const long long base = (long long)r * nc;
            if (!AIDW_IN(base + ca, g->n_cells + 1, bounds::kKnnHead) ||
                !AIDW_IN(base + cb + 1, g->n_cells + 1, bounds::kKnnHead))
                continue;
            const int a = start[base + ca], b = start[base + cb + 1];
            if (!AIDW_IN(b, g->n_data + 1, bounds::kKnnPoints)) continue;
            found += b - a;
            // the next point's load is issued before the current one is
            // tested, so its L2 latency overlaps the top-k update (kNN ms at
            // 1M, uniform k = 10 / clustered k = 10, 24, 32: 0.545 / 1.011,
            // 1.948, 2.668 -> 0.528 / 0.958, 1.818, 2.556)
            const float4 *P4 = reinterpret_cast<const float4 *>(pts);
            float4 nxt = a < b ? P4[a] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            for (int s = a; s < b; ++s) {
                const float4 p = nxt;
                if (s + 1 < b) nxt = P4[s + 1];
                const int pidx = __float_as_int(p.w);
                const D d2 = DistT<F64>::d2(qx, qy, p.x, p.y);
                // A candidate that beats the k-th replaces it and bubbles
                // down to its place.  Once it stops, no later step swaps, so
                // the exit test may be skipped on some steps.  The float32
                // path compares and moves one 64-bit key per slot instead of
                // a (d^2, index) pair (kNN ms at 1M, uniform k = 10 /
                // clustered k = 24, 32 / uniform k = 32: 0.525 / 1.81, 2.57 /
                // 1.67 -> 0.470 / 1.55, 2.15 / 1.35 with the exit test on
                // every second step up to 16 slots and every fourth for 24
                // and 32) and takes the test on every fourth step up to 16
                // slots and every eighth for 24 and 32: 0.437 / 1.47, 2.04 /
                // 1.27 (every fourth for all: 0.438 / 1.55, 2.15 / 1.35;
                // every eighth for all: 0.461 / 1.48, 2.04 / 1.27; every
                // sixteenth for 24 and 32: 1.56, 2.12 / 1.35; every second
                // for 24 and 32: 1.98, 2.91 / 1.89).  The float64 path keeps
                // the pair, with the test on every second step up to 16
                // slots and every fourth for 32 (with pairs, measured at 1M:
                // on every step, k = 10 0.70 vs 0.57 ms; for 32 slots on
                // every step, 2x slower; never, 1.2-1.5x slower at k =
                // 20..32).  While the list fills, the candidate passes
                // every empty slot above its place; a separate fill branch
                // that starts it at the first empty slot was slower (uniform
                // / clustered k = 10: 0.526 / 0.955 -> 0.685 / 1.087 ms:
                // divergence) and made the 24- and 32-slot forms spill.  An
                // insertion without a chain (rank from independent compares,
                // then every slot above it shifted by independent selects)
                // was slower for 24 and 32 slots (clustered k = 24 / 32,
                // uniform k = 32: 1.81 / 2.56 / 1.67 -> 2.59 / 3.91 / 2.49
                // ms): the bubble's early exit saves more.
                if (!F64) {
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint((float)d2) << 32) | (unsigned)pidx;
                    if (key < kth_key) {
                        kk[KMAX - 1] = key;
#pragma unroll
                        for (int j = KMAX - 1; j > 0; --j) {
                            const bool sw = kk[j] < kk[j - 1];
                            if ((j & (KMAX <= 16 ? 3 : 7)) == 0 && !sw) break;
                            const unsigned long long t = kk[j], u = kk[j - 1];
                            kk[j] = sw ? u : t;
                            kk[j - 1] = sw ? t : u;
                        }
                        kth_key = kk[KMAX - 1];
                        kth = (D)__uint_as_float((unsigned)(kth_key >> 32));
                    }
                } else if (d2 < kth || (d2 == kth && pidx < kthi)) {
                    kd[KMAX - 1] = d2;
                    ki[KMAX - 1] = pidx;
#pragma unroll
                    for (int j = KMAX - 1; j > 0; --j) {
                        const bool sw =
                            kd[j] < kd[j - 1] || (kd[j] == kd[j - 1] && ki[j] < ki[j - 1]);
                        if ((j & (KMAX <= 16 ? 1 : 3)) == 0 && !sw) break;
                        const D td = kd[j], tl = kd[j - 1];
                        const int ti = ki[j], tj = ki[j - 1];
                        kd[j] = sw ? tl : td;
                        ki[j] = sw ? tj : ti;
                        kd[j - 1] = sw ? td : tl;
                        ki[j - 1] = sw ? ti : tj;
                    }
                    kth = kd[KMAX - 1];
                    kthi = ki[KMAX - 1];
                }
            }
        }
        const bool full_l = col - L <= 0, full_r = col + L >= nc - 1;
        const bool full_b = row - L <= 0, full_t = row + L >= nr - 1;
        if (full_l && full_r && full_b && full_t) break;  // whole grid visited
        if (J.stop_rule == kStopPaperLevel) {
            if (L0 < 0 && found >= k) L0 = L;
            if (L0 >= 0 && L == L0 + 1) break;
            continue;
        }
        if (found >= k &&
            block_is_final(eb, __int2float_rd(L), full_l, full_r, full_b, full_t, kth))
            break;
    }

    if (!F64) {
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            kd[j] = j < lo ? -DistT<F64>::inf() : (D)__uint_as_float((unsigned)(kk[j] >> 32));
            ki[j] = j < lo ? -1 : (int)(unsigned)(kk[j] & 0xffffffffull);
        }
    }

    // Eq. 3 (r_obs), Eq. 2 (r_exp, possibly with an explicit area), Eq. 4-6.
    double r_obs, alpha;
    if (F64) {
        r_obs = 0.0;
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
            if (j >= lo) r_obs += sqrt((double)kd[j]);
        r_obs /= (double)k;
        const double r_exp = ap.area_override > 0.0
                                 ? 1.0 / (2.0 * sqrt((double)g->n_data / ap.area_override))
                                 : g->r_exp;
        const double mu = membership(nn_statistic(r_obs, r_exp), ap.r_min, ap.r_max);
        alpha = decay_power(mu, ap.level[0], ap.level[1], ap.level[2], ap.level[3], ap.level[4]);
    } else {
        const float rf = robs_f32<KMAX>(kd, lo, k);
        r_obs = rf;
        alpha = decay_power_f32(membership_f32(rf, g, ap), ap.level_f);
    }
    D d1 = kd[KMAX - 1];  // the nearest, kd[lo]
#pragma unroll
    for (int j = 0; j < KMAX - 1; ++j)
        if (j == lo) d1 = kd[j];

    // Data points at distance 0 (the limit of Eq. 1 for a query on data):
    // counted and their z summed by a second scan, only for a query whose
    // nearest neighbour is at distance 0, instead of a test on every
    // candidate of the search.  Such a point is within the underflow range
    // of the squared distance of the query (|dx|, |dy| < 2^-63), so its cell
    // index differs from the query's by at most ceil(2^-63 / cw) + 1 per
    // axis (1 on any grid whose cells are wider than 2^-63).
    int n_hit = 0;
    double hit_z = 0.0;
    if (d1 == (D)0) {
        const double reach = 0x1p-63 / cw;
        const int R = reach < 1.0 ? 1 : (int)fmin(ceil(reach) + 1.0, (double)max(nc, nr));
        HitSum<F64> hits;
        for (int r = max(row - R, 0); r <= min(row + R, nr - 1); ++r) {
            const long long base = (long long)r * nc;
            if (!AIDW_IN(base + min(col + R, nc - 1) + 1, g->n_cells + 1, bounds::kKnnHead))
                continue;
            const int a = start[base + max(col - R, 0)], b = start[base + min(col + R, nc - 1) + 1];
            for (int s = a; s < b; ++s) {
                const float4 p = reinterpret_cast<const float4 *>(pts)[s];
                if (DistT<F64>::d2(qx, qy, p.x, p.y) == (D)0) {
                    ++n_hit;
                    hits.add(p.z);
                }
            }
        }
        hit_z = hits.value() / (double)n_hit;
    }
    if (recs) {
        QRec r;
        r.alpha = alpha;
        r.hit_z = hit_z;
        r.d1sq = (float)d1;
        r.n_hit = n_hit;
        recs[q] = r;
    }
    if (out_idx || out_dist) {
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j >= lo) {
                if (out_idx) out_idx[q * k + j - lo] = ki[j];
                if (out_dist) out_dist[q * k + j - lo] = (float)sqrt(kd[j]);
            }
        }
    }
    if (out_robs) out_robs[q] = (float)r_obs;
    if (out_alpha) {
        if (F64)
            static_cast<double *>(out_alpha)[q] = alpha;
        else
            static_cast<float *>(out_alpha)[q] = (float)alpha;
    }
    if (J.out_zlocal) {
        // Eq. 1 over the k neighbours; coincident neighbours give their mean
        // z.  Float64 path: pow(d^2, -alpha/2) and float64 sums.  Float32
        // path: weights (d^2 / d1^2)^(-alpha/2) on the SFU (largest weight 1)
        // and TwoSum-compensated float32 sums of at most 32 terms (float64
        // adds would cost more than the whole search on this GPU), one
        // float64 division at the end.
        double zl;
        if (F64) {
            double sw = 0.0, swz = 0.0, hz = 0.0;
            int nh = 0;
#pragma unroll
            for (int j = 0; j < KMAX; ++j) {
                if (j >= lo) {
                    const double zj = (double)J.zorig[ki[j]];
                    if (kd[j] == (D)0) {
                        ++nh;
                        hz += zj;
                    } else {
                        const double w = pow((double)kd[j], -0.5 * alpha);
                        sw += w;
                        swz += w * zj;
                    }
                }
            }
            zl = nh ? hz / (double)nh : swz / sw;
        } else {
            const float c = (float)(-0.5 * alpha);
            const float b = -c * lg2_sfu((float)d1);
            float swh = 0.0f, swl = 0.0f, szh = 0.0f, szl = 0.0f, hzh = 0.0f, hzl = 0.0f;
            int nh = 0;
#pragma unroll
            for (int j = 0; j < KMAX; ++j) {
                if (j >= lo) {
                    const float zj = J.zorig[ki[j]];
                    if (kd[j] == (D)0) {
                        ++nh;
                        comp_add(hzh, hzl, zj);
                    } else {
                        const float w = ex2_sfu(fma_rn(lg2_sfu((float)kd[j]), c, b));
                        comp_add(swh, swl, w);
                        comp_add(szh, szl, mul_rn(w, zj));
                    }
                }
            }
            zl = nh ? ((double)hzh + (double)hzl) / (double)nh
                    : ((double)szh + (double)szl) / ((double)swh + (double)swl);
        }
        if (F64)
            static_cast<double *>(J.out_zlocal)[q] = zl;
        else
            static_cast<float *>(J.out_zlocal)[q] = (float)zl;
    }
}

// Warp-per-query variant: the 32 lanes of a warp search one query together.
// Each ring segment is read 32 consecutive points at a time (coalesced), and
// the k best (d^2, index) pairs are held one per lane, sorted by lane.  A
// ballot picks the candidates that beat the current k-th; each is inserted
// by counting the entries below it (ballot + popc) and shifting the larger
// entries up one lane (shfl_up).  Same ring order and stop rule as k_knn.
template <bool F64>
__global__ void __launch_bounds__(kKnnMaxThreads)
    k_knn_warp(KnnJob job0, const KnnJob *__restrict__ jobs, int n_jobs, long long total_q,
               AlphaParams ap)
{
    using D = typename DistT<F64>::T;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long gq = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gq >= total_q) return;  // uniform across the warp
    const KnnJob J = jobs ? jobs[knn_job_of(jobs, n_jobs, gq)] : job0;
    const GridDev *__restrict__ g = J.g;
    const bool failed = (g->status & (kStatusNonfiniteData | kStatusCapacity)) != 0;
    const long long li = gq - J.q_base;
    const long long q = (J.order && !failed) ? (long long)J.order[li] : li;
    if (!AIDW_IN(q, J.nq, bounds::kKnnOrder)) return;
    const Point *__restrict__ pts = J.pts;
    const int *__restrict__ start = J.start;
    const int k = J.k;
    const float qx = J.qx[q], qy = J.qy[q];
    const double nanv = __longlong_as_double(0x7ff8000000000000LL);

    if (failed || !isfinite(qx) || !isfinite(qy)) {
        if (lane == 0) {
            if (!failed) atomicOr(const_cast<int *>(&g->status), kStatusNonfiniteQuery);
            if (J.recs) {
                QRec r;
                r.alpha = nanv;
                r.hit_z = nanv;
                r.d1sq = __int_as_float(0x7fc00000);
                r.n_hit = 0;
                J.recs[q] = r;
            }
            if (J.out_robs) J.out_robs[q] = __int_as_float(0x7fc00000);
            if (J.out_alpha) {
                if (F64)
                    static_cast<double *>(J.out_alpha)[q] = nanv;
                else
                    static_cast<float *>(J.out_alpha)[q] = __int_as_float(0x7fc00000);
            }
        }
        if (lane < k) {
            if (J.out_idx) J.out_idx[q * k + lane] = -1;
            if (J.out_dist) J.out_dist[q * k + lane] = __int_as_float(0x7fc00000);
        }
        return;
    }

    const double minx = g->min_x, miny = g->min_y, cw = g->cw;
    const int nc = (int)g->n_col, nr = (int)g->n_row;
    long long colw = gridk::cell_floor(qx, g->min_x_f, g->inv_cw_f, minx, cw);
    long long roww = gridk::cell_floor(qy, g->min_y_f, g->inv_cw_f, miny, cw);
    const int col = (int)(colw < 0 ? 0 : (colw > nc - 1 ? nc - 1 : colw));
    const int row = (int)(roww < 0 ? 0 : (roww > nr - 1 ? nr - 1 : roww));
    const EdgeBounds eb = edge_bounds(qx, qy, g, col, row);

    D md = DistT<F64>::inf();  // this lane's entry of the sorted top-k list
    int mi = 0x7fffffff;
    D kth = DistT<F64>::inf();
    int kthi = 0x7fffffff;
    long long found = 0;
    int n_hit = 0;
    HitSum<F64> hits;
    int L0 = -1;  // paper rule: the first level whose block holds k points

    for (int L = 0;; ++L) {
        const int c0 = max(col - L, 0), c1 = min(col + L, nc - 1);
        const bool left_in = col - L >= 0, right_in = col + L <= nc - 1;
        const int r0 = max(row - L + 1, 0), r1 = min(row + L - 1, nr - 1);
        const int nside = (L > 0 && (left_in || right_in) && r1 >= r0) ? r1 - r0 + 1 : 0;
        const int nsegs = L == 0 ? 1 : 2 + 2 * nside;
        for (int sg = 0; sg < nsegs; ++sg) {
            int r, ca, cb;
            if (L == 0) {
                r = row;
                ca = cb = col;
            } else if (sg < 2) {
                r = sg == 0 ? row - L : row + L;
                if (r < 0 || r > nr - 1) continue;
                ca = c0;
                cb = c1;
            } else {
                const int e = sg - 2;
                r = r0 + (e >> 1);
                const bool right = (e & 1) != 0;
                if (right ? !right_in : !left_in) continue;
                ca = cb = right ? col + L : col - L;
            }
            const long long base = (long long)r * nc;
            if (!AIDW_IN(base + ca, g->n_cells + 1, bounds::kKnnHead) ||
                !AIDW_IN(base + cb + 1, g->n_cells + 1, bounds::kKnnHead))
                continue;
            const int a = start[base + ca], b = start[base + cb + 1];
            if (!AIDW_IN(b, g->n_data + 1, bounds::kKnnPoints)) continue;
            found += b - a;
            for (int s0 = a; s0 < b; s0 += 32) {
                const int s = s0 + lane;
                D d2 = DistT<F64>::inf();
                int pidx = 0x7fffffff;
                if (s < b) {
                    const float4 p = reinterpret_cast<const float4 *>(pts)[s];
                    pidx = __float_as_int(p.w);
                    d2 = DistT<F64>::d2(qx, qy, p.x, p.y);
                    if (d2 == (D)0) {
                        ++n_hit;
                        hits.add(p.z);
                    }
                }
                unsigned m = __ballot_sync(full, d2 < kth || (d2 == kth && pidx < kthi));
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    const D cd = __shfl_sync(full, d2, src);
                    const int ci = __shfl_sync(full, pidx, src);
                    if (!(cd < kth || (cd == kth && ci < kthi))) continue;
                    const bool lt = lane < k && (md < cd || (md == cd && mi < ci));
                    const int pos = __popc(__ballot_sync(full, lt));
                    const D up_d = __shfl_up_sync(full, md, 1);
                    const int up_i = __shfl_up_sync(full, mi, 1);
                    if (lane < k && lane >= pos) {
                        md = lane == pos ? cd : up_d;
                        mi = lane == pos ? ci : up_i;
                    }
                    kth = __shfl_sync(full, md, k - 1);
                    kthi = __shfl_sync(full, mi, k - 1);
                }
            }
        }
        const bool full_l = col - L <= 0, full_r = col + L >= nc - 1;
        const bool full_b = row - L <= 0, full_t = row + L >= nr - 1;
        if (full_l && full_r && full_b && full_t) break;
        if (J.stop_rule == kStopPaperLevel) {
            if (L0 < 0 && found >= k) L0 = L;
            if (L0 >= 0 && L == L0 + 1) break;
            continue;
        }
        if (found >= k &&
            block_is_final(eb, __int2float_rd(L), full_l, full_r, full_b, full_t, kth))
            break;
    }

    // Eq. 3-6 (the order of the r_obs sum differs from k_knn only in rounding)
    double rs = lane < k ? (F64 ? sqrt((double)md) : (double)sqrtf((float)md)) : 0.0;
    double hit_sum = hits.value();
    for (int o = 16; o > 0; o >>= 1) {
        rs += __shfl_xor_sync(full, rs, o);
        n_hit += __shfl_xor_sync(full, n_hit, o);
        hit_sum += __shfl_xor_sync(full, hit_sum, o);
    }
    double r_obs, alpha;
    if (F64) {
        r_obs = rs / (double)k;
        const double r_exp = ap.area_override > 0.0
                                 ? 1.0 / (2.0 * sqrt((double)g->n_data / ap.area_override))
                                 : g->r_exp;
        const double mu = membership(nn_statistic(r_obs, r_exp), ap.r_min, ap.r_max);
        alpha = decay_power(mu, ap.level[0], ap.level[1], ap.level[2], ap.level[3], ap.level[4]);
    } else {
        const float rf = (float)rs / (float)k;
        r_obs = rf;
        alpha = decay_power_f32(membership_f32(rf, g, ap), ap.level_f);
    }
    const D d1 = __shfl_sync(full, md, 0);
    if (lane == 0) {
        if (J.recs) {
            QRec r;
            r.alpha = alpha;
            r.hit_z = n_hit > 0 ? hit_sum / (double)n_hit : 0.0;
            r.d1sq = (float)d1;
            r.n_hit = n_hit;
            J.recs[q] = r;
        }
        if (J.out_robs) J.out_robs[q] = (float)r_obs;
        if (J.out_alpha) {
            if (F64)
                static_cast<double *>(J.out_alpha)[q] = alpha;
            else
                static_cast<float *>(J.out_alpha)[q] = (float)alpha;
        }
    }
    if (lane < k) {
        if (J.out_idx) J.out_idx[q * k + lane] = mi;
        if (J.out_dist) J.out_dist[q * k + lane] = (float)sqrt(md);
    }
}

// The kNN of the authors' earlier GPU AIDW (Sec. 3.1, the "original"
// algorithm the paper improves on): every query thread scans ALL data points
// and keeps its k best in a sorted register list.  Data points are staged
// through shared memory in tiles of kBruteTile (the "tiled" form).  Same
// float32 distance and (d^2, index) order as k_knn, so the result is the
// same; kept as the baseline of the grid search.
constexpr int kBruteTile = 1024;
constexpr int kBruteThreads = 256;

template <int KMAX>
__global__ void __launch_bounds__(kBruteThreads)
    k_knn_brute(const Point *__restrict__ pts, long long n, const float *__restrict__ qxa,
                const float *__restrict__ qya, long long nq, int k, int *__restrict__ out_idx,
                float *__restrict__ out_dist, float *__restrict__ out_robs)
{
    __shared__ float4 tile[kBruteTile];
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = q < nq;
    const float qx = active ? qxa[q] : 0.0f, qy = active ? qya[q] : 0.0f;
    float kd[KMAX];
    int ki[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        kd[j] = __int_as_float(0x7f800000);
        ki[j] = 0x7fffffff;
    }
    float kth = __int_as_float(0x7f800000);
    int kthi = 0x7fffffff;
    for (long long base = 0; base < n; base += kBruteTile) {
        const int cnt = (int)min((long long)kBruteTile, n - base);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x)
            tile[i] = reinterpret_cast<const float4 *>(pts)[base + i];
        __syncthreads();
        if (!active) continue;
        for (int j = 0; j < cnt; ++j) {
            const float4 p = tile[j];
            const int pidx = __float_as_int(p.w);
            const float d2 = dist2_f32(qx, qy, p.x, p.y);
            if (d2 < kth || (d2 == kth && pidx < kthi)) {
                float cd = d2;
                int ci = pidx;
#pragma unroll
                for (int t = 0; t < KMAX; ++t) {
                    const bool lt = (t < k) && (cd < kd[t] || (cd == kd[t] && ci < ki[t]));
                    const float td = kd[t];
                    const int ti = ki[t];
                    kd[t] = lt ? cd : td;
                    ki[t] = lt ? ci : ti;
                    cd = lt ? td : cd;
                    ci = lt ? ti : ci;
                }
                kth = kd[0];
                kthi = ki[0];
#pragma unroll
                for (int t = 1; t < KMAX; ++t) {
                    if (t == k - 1) {
                        kth = kd[t];
                        kthi = ki[t];
                    }
                }
            }
        }
    }
    if (!active) return;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        if (j < k) {
            if (out_idx) out_idx[q * k + j] = ki[j];
            if (out_dist) out_dist[q * k + j] = sqrtf(kd[j]);
        }
    }
    if (out_robs) out_robs[q] = robs_f32<KMAX>(kd, 0, k);  // as the grid kNN's float32 path
}

template <bool F64, int KMAX>
void launch_knn(const KnnJob &job0, const KnnJob *jobs, int n_jobs, long long total_q,
                const AlphaParams &ap, int threads, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((total_q + threads - 1) / threads);
    k_knn<F64, KMAX><<<blocks, threads, 0, s>>>(job0, jobs, n_jobs, total_q, ap);
}

// threads == 0 selects the warp-per-query kernel (128-thread blocks).
template <bool F64>
void launch_knn_k(const KnnJob &job0, const KnnJob *jobs, int n_jobs, long long total_q,
                  int kmax, const AlphaParams &ap, int threads, cudaStream_t s)
{
    if (threads == 0) {
        const unsigned blocks = (unsigned)((total_q * 32 + 127) / 128);
        k_knn_warp<F64><<<blocks, 128, 0, s>>>(job0, jobs, n_jobs, total_q, ap);
        return;
    }
    if (kmax <= 8)
        launch_knn<F64, 8>(job0, jobs, n_jobs, total_q, ap, threads, s);
    else if (kmax <= 16)
        launch_knn<F64, 16>(job0, jobs, n_jobs, total_q, ap, threads, s);
    else if (kmax <= 24)
        launch_knn<F64, 24>(job0, jobs, n_jobs, total_q, ap, threads, s);
    else
        launch_knn<F64, 32>(job0, jobs, n_jobs, total_q, ap, threads, s);
}

// ---- queries in grid-cell order ----------------------------------------------
// Random query order mixes queries from dense clusters and sparse background
// in one warp, which then runs as long as its slowest query.  Visiting the
// queries by grid cell (a counting sort over the data grid's cells) gives
// each warp neighbouring queries with similar ring counts and shared cells.
// The order changes no result: every query is computed independently.
__global__ void __launch_bounds__(gridk::kThreads)
    k_qkeys(const float *__restrict__ qx, const float *__restrict__ qy, long long nq,
            const GridDev *__restrict__ g, int *__restrict__ count, int *__restrict__ key,
            int *__restrict__ rank)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    float x = qx[i], y = qy[i];
    if (!isfinite(x) || !isfinite(y)) x = y = 0.0f;  // flagged by the kNN kernel
    gridk::key_one_xy(i, x, y, g, count, key, rank);
}

__global__ void __launch_bounds__(gridk::kThreads) k_qscan(int *a, long long len,
                                                           unsigned long long *flags,
                                                           int *ticket, GridDev *g)
{
    gridk::scan_lookback_block(a, len, flags, ticket, &g->status);
}
__global__ void __launch_bounds__(gridk::kThreads)
    k_qscatter(long long nq, const int *__restrict__ start, const int *__restrict__ key,
               const int *__restrict__ rank, int *__restrict__ order)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nq) gridk::scatter_one(i, start, key, rank, order, nq);
}

// Whether the single-grid kNN sorts its queries by cell (AIDW_KNN_SORT=0|1
// overrides; default on from 4096 queries).
bool knn_sort_queries(long long nq)
{
    static const int v = [] {
        const char *e = getenv("AIDW_KNN_SORT");
        return e ? (atoi(e) != 0 ? 1 : 0) : -1;
    }();
    return v >= 0 ? v == 1 : nq >= 4096;
}

// Fills *order (pool memory, freed by the caller with lib_free) with the
// queries in cell order; the temporaries are returned to the pool.
aidw_status query_order(const aidw_grid *g, const float *qx, const float *qy, long long nq,
                        int **order, cudaStream_t s, int *launches)
{
    using namespace gridk;
    const long long len = g->cap_cells + 1;
    const long long nb = (len + kScanChunk - 1) / kScanChunk;
    const long long n_ints = grid_cell_start_ints(g->cap_cells);  // counts, scan records, tickets
    const long long rec_off = (len + 1) / 2 * 2;
    int *count = nullptr, *key = nullptr, *rank = nullptr;
    *order = nullptr;
    cudaError_t e = lib_alloc((void **)&count, sizeof(int) * n_ints, s);
    if (e == cudaSuccess) e = lib_alloc((void **)&key, sizeof(int) * nq, s);
    if (e == cudaSuccess) e = lib_alloc((void **)&rank, sizeof(int) * nq, s);
    if (e == cudaSuccess) e = lib_alloc((void **)order, sizeof(int) * nq, s);
    if (e == cudaSuccess) {
        const unsigned qb = (unsigned)((nq + kThreads - 1) / kThreads);
        unsigned long long *flags = reinterpret_cast<unsigned long long *>(count + rec_off);
        int *ticket = count + rec_off + 2 * nb;
        cudaMemsetAsync(count, 0, sizeof(int) * n_ints, s);
        k_qkeys<<<qb, kThreads, 0, s>>>(qx, qy, nq, g->dev, count, key, rank);
        k_qscan<<<(unsigned)nb, kThreads, 0, s>>>(count, len, flags, ticket, g->dev);
        k_qscatter<<<qb, kThreads, 0, s>>>(nq, count, key, rank, *order);
        *launches += 3;
        e = cudaGetLastError();
    }
    lib_free(count, s);
    lib_free(key, s);
    lib_free(rank, s);
    if (e != cudaSuccess) {
        lib_free(*order, s);
        *order = nullptr;
        return e == cudaErrorMemoryAllocation ? AIDW_ERR_OOM : cuda_status(e);
    }
    return AIDW_OK;
}

}  // namespace

// Launch shape of the single-grid kNN: thread per query (block size) or warp
// per query (0).  Thread per query was faster for every k measured on GB300
// (clustered 1M points: 4.3 vs 15.0 ms at k = 10, 23.9 vs 40.7 ms at k = 32:
// most ring segments are single cells, which leave most lanes of a warp
// idle).  AIDW_KNN_MODE=warp selects the warp kernel.
int knn_default_threads(int k)
{
    static const bool warp = [] {
        const char *e = getenv("AIDW_KNN_MODE");
        return e && strcmp(e, "warp") == 0;
    }();
    (void)k;
    return warp ? 0 : kKnnThreads;
}

aidw_status knn_launch(const aidw_grid *g, const float *qx, const float *qy, long long n_query,
                       int k, bool fp64, const AlphaParams &ap, QRec *recs, int *out_idx,
                       float *out_dist, float *out_robs, void *out_alpha, cudaStream_t s,
                       void *out_zlocal, bool sort, int stop_rule)
{
    NvtxRange nvtx_("knn");
    if (n_query <= 0) return AIDW_OK;
    KnnJob j;
    j.g = g->dev;
    j.pts = g->pts;
    j.start = g->cell_start;
    j.qx = qx;
    j.qy = qy;
    j.recs = recs;
    j.out_idx = out_idx;
    j.out_dist = out_dist;
    j.out_robs = out_robs;
    j.out_alpha = out_alpha;
    j.zorig = g->zorig;
    j.out_zlocal = out_zlocal;
    j.order = nullptr;
    j.nq = n_query;
    j.q_base = 0;
    j.k = k;
    j.stop_rule = stop_rule;
    const int threads = out_zlocal ? kKnnThreads : knn_default_threads(k);
    const int prof = profile_begin(s);
    int launches = 1;
    int *order = nullptr;
    if (sort && knn_sort_queries(n_query)) {
        const aidw_status st = query_order(g, qx, qy, n_query, &order, s, &launches);
        if (st != AIDW_OK) return st;
        j.order = order;
    }
    if (fp64)
        launch_knn_k<true>(j, nullptr, 1, n_query, k, ap, threads, s);
    else
        launch_knn_k<false>(j, nullptr, 1, n_query, k, ap, threads, s);
    profile_end(prof, s, AIDW_STAGE_KNN, launches);
    lib_free(order, s);
    return cuda_status(cudaGetLastError());
}

aidw_status knn_launch_brute(const aidw_grid *g, const float *qx, const float *qy,
                             long long n_query, int k, int *out_idx, float *out_dist,
                             float *out_robs, cudaStream_t s)
{
    if (n_query <= 0) return AIDW_OK;
    const unsigned blocks = (unsigned)((n_query + kBruteThreads - 1) / kBruteThreads);
    const int prof = profile_begin(s);
    if (k <= 8)
        k_knn_brute<8><<<blocks, kBruteThreads, 0, s>>>(g->pts, g->n_data, qx, qy, n_query, k,
                                                        out_idx, out_dist, out_robs);
    else if (k <= 16)
        k_knn_brute<16><<<blocks, kBruteThreads, 0, s>>>(g->pts, g->n_data, qx, qy, n_query, k,
                                                         out_idx, out_dist, out_robs);
    else
        k_knn_brute<32><<<blocks, kBruteThreads, 0, s>>>(g->pts, g->n_data, qx, qy, n_query, k,
                                                         out_idx, out_dist, out_robs);
    profile_end(prof, s, AIDW_STAGE_KNN, 1);
    return cuda_status(cudaGetLastError());
}

aidw_status knn_launch_batch(const KnnJob *jobs, int n_jobs, long long total_q, int kmax,
                             bool fp64, const AlphaParams &ap, int threads, cudaStream_t s)
{
    if (total_q <= 0 || n_jobs <= 0) return AIDW_OK;
    if (threads != 0 && (threads < 32 || threads > kKnnMaxThreads)) threads = kKnnThreads;
    KnnJob none;
    memset(&none, 0, sizeof(none));
    if (fp64)
        launch_knn_k<true>(none, jobs, n_jobs, total_q, kmax, ap, threads, s);
    else
        launch_knn_k<false>(none, jobs, n_jobs, total_q, kmax, ap, threads, s);
    return cuda_status(cudaGetLastError());
}

}  // namespace aidw
