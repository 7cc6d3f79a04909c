// Per-element and per-block bodies of the even-grid build (Sec. 3.2.1-3.2.3,
// 4.1.1-4.1.3 of arXiv 1601.05904), shared by the single-grid kernels
// (grid_build.cu) and the batched kernels that build many grids in one
// launch per step (batch.cu).
#pragma once

#include <float.h>
#include <math.h>

#include "aidw_internal.cuh"

namespace aidw {
namespace gridk {

constexpr int kThreads = 256;
constexpr int kScanItems = 16;                     // per thread
constexpr int kScanChunk = kThreads * kScanItems;  // per block

// Order-preserving integer encoding of float32 (the form in which the
// grid record keeps its bounding box).
__device__ __forceinline__ int enc_float(float f)
{
    const int b = __float_as_int(f);
    return b >= 0 ? b : (b ^ 0x7FFFFFFF);
}
__device__ __forceinline__ float dec_float(int e)
{
    return __int_as_float(e >= 0 ? e : (e ^ 0x7FFFFFFF));
}

__device__ __forceinline__ void grid_dims(GridDev *g, double cell_scale, double area_param,
                                          long long cap);

// ---- bounding box and dimensions in one launch --------------------------------
// The grid's points are reduced by nblocks blocks of kThreads threads; this is
// block lb of them.  Each block reduces its points to (min x, max x, min y,
// max y, non-finite flag) and stores them in part[5 * lb]; the last block to
// finish (an atomic ticket, which it resets for the next launch) reduces the
// blocks' records, writes the whole grid record (status included, so the
// record needs no initialisation) and computes the dimensions.
__device__ __forceinline__ void bbox_dims_block(const float *__restrict__ x,
                                                const float *__restrict__ y,
                                                const float *__restrict__ z, long long n,
                                                float *__restrict__ part, int *ticket, GridDev *g,
                                                double cell_scale, double area_param,
                                                long long cap, long long lb, long long nblocks)
{
    float mnx = FLT_MAX, mny = FLT_MAX, mxx = -FLT_MAX, mxy = -FLT_MAX;
    int bad = 0;
    const long long stride = nblocks * kThreads;
    for (long long i = lb * kThreads + threadIdx.x; i < n; i += stride) {
        const float xi = __ldg(x + i), yi = __ldg(y + i), zi = __ldg(z + i);
        if (!isfinite(xi) || !isfinite(yi) || !isfinite(zi)) {
            bad = 1;
            continue;
        }
        mnx = fminf(mnx, xi);
        mxx = fmaxf(mxx, xi);
        mny = fminf(mny, yi);
        mxy = fmaxf(mxy, yi);
    }
    __shared__ float s[5][kThreads / 32];
    __shared__ bool last;
    for (int round = 0; round < 2; ++round) {
        for (int o = 16; o > 0; o >>= 1) {
            mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
            mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
            mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
            mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
        }
        bad = __any_sync(0xffffffffu, bad);
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) {
            s[0][w] = mnx;
            s[1][w] = mxx;
            s[2][w] = mny;
            s[3][w] = mxy;
            s[4][w] = bad ? 1.0f : 0.0f;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 1; i < kThreads / 32; ++i) {
                mnx = fminf(mnx, s[0][i]);
                mxx = fmaxf(mxx, s[1][i]);
                mny = fminf(mny, s[2][i]);
                mxy = fmaxf(mxy, s[3][i]);
                bad |= s[4][i] != 0.0f;
            }
        }
        if (round == 1) break;
        if (threadIdx.x == 0) {
            float *p = part + 5 * lb;
            p[0] = mnx;
            p[1] = mxx;
            p[2] = mny;
            p[3] = mxy;
            p[4] = bad ? 1.0f : 0.0f;
            __threadfence();
            last = atomicAdd(ticket, 1) == (int)nblocks - 1;
        }
        __syncthreads();
        if (!last) return;
        // the last block: every block's record is visible (each fenced
        // before taking its ticket); reduce them with the same code
        __threadfence();
        mnx = mny = FLT_MAX;
        mxx = mxy = -FLT_MAX;
        bad = 0;
        for (long long b = threadIdx.x; b < nblocks; b += kThreads) {
            const float *p = part + 5 * (long long)b;
            mnx = fminf(mnx, __ldcg(p + 0));
            mxx = fmaxf(mxx, __ldcg(p + 1));
            mny = fminf(mny, __ldcg(p + 2));
            mxy = fmaxf(mxy, __ldcg(p + 3));
            bad |= __ldcg(p + 4) != 0.0f;
        }
        __syncthreads();  // s[] is reused
    }
    if (threadIdx.x == 0) {
        *ticket = 0;
        g->enc_min_x = enc_float(mnx);
        g->enc_max_x = enc_float(mxx);
        g->enc_min_y = enc_float(mny);
        g->enc_max_y = enc_float(mxy);
        g->n_data = n;
        g->status = bad ? kStatusNonfiniteData : 0;
        grid_dims(g, cell_scale, area_param, cap);
    }
}

// Grid dimensions.  cap is the capacity of the cell arrays: if the box's
// aspect ratio or an explicit area would need more cells, the width is
// doubled until it fits (the kNN result does not depend on it).
__device__ __forceinline__ void grid_dims(GridDev *g, double cell_scale, double area_param,
                                          long long cap)
{
    if (g->status & kStatusNonfiniteData) {
        // a failed grid still gets in-range dimensions (one empty cell), so
        // no later kernel can index outside its arrays
        g->min_x = g->min_y = g->max_x = g->max_y = 0.0;
        g->area = 0.0;
        g->r_exp = 0.0;
        g->cw = 1.0;
        g->min_x_f = g->min_y_f = 0.0f;
        g->inv_cw_f = g->cw_rd = g->cw_ru = 1.0f;
        g->n_col = g->n_row = g->n_cells = 1;
        return;
    }
    const double minx = (double)dec_float(g->enc_min_x), maxx = (double)dec_float(g->enc_max_x);
    const double miny = (double)dec_float(g->enc_min_y), maxy = (double)dec_float(g->enc_max_y);
    const double W = maxx - minx, H = maxy - miny;
    const double n = (double)g->n_data;
    const double area = area_param > 0.0 ? area_param : W * H;
    const double r_exp = (area > 0.0) ? 1.0 / (2.0 * sqrt(n / area)) : 0.0;  // Eq. 2
    double cw = cell_scale * r_exp;
    if (!(cw > 0.0)) {
        const double side = W > H ? W : H;
        cw = side > 0.0 ? cell_scale * side / (2.0 * n) : 1.0;
    }
    for (int it = 0; it < 2100; ++it) {
        const double nc = floor((W + cw) / cw), nr = floor((H + cw) / cw);
        if (nc * nr <= (double)cap) break;
        cw = cw * 2.0;
    }
    g->min_x = minx;
    g->min_y = miny;
    g->max_x = maxx;
    g->max_y = maxy;
    g->area = area;
    g->r_exp = r_exp;
    g->cw = cw;
    g->min_x_f = (float)minx;
    g->min_y_f = (float)miny;
    g->inv_cw_f = (float)(1.0 / cw);
    g->cw_rd = __double2float_rd(cw);
    g->cw_ru = __double2float_ru(cw);
    g->n_col = (long long)((W + cw) / cw);
    g->n_row = (long long)((H + cw) / cw);
    g->n_cells = g->n_col * g->n_row;
    if (g->n_cells > cap) atomicOr(&g->status, kStatusCapacity);
}

__device__ __forceinline__ bool grid_failed(const GridDev *g)
{
    return (g->status & (kStatusNonfiniteData | kStatusCapacity)) != 0;
}

// floor((x - min) / cw) of the cell formula, equal to the floor of the
// correctly rounded float64 quotient of the float64 difference (the
// definition).  Fast path in float32: x and min are float32 values, and
// q = fl32(fl32(x - min) * fl32(1/cw)) is within 3 * 2^-24 (+ tiny) of the
// exact quotient, relatively, as is the float64 quotient; so where q is
// farther than 2^-21 |q| from every integer the two have the same floor
// (q - floor(q) and floor(q) + 1 - q are exact for |q| < 2^23; beyond that
// the margin exceeds 1 and the test always fails).  Otherwise - about one
// coordinate in 10^3 at a thousand cells per side - the float64 division
// is used.  Float64 runs at a small fraction of float32 on this GPU.
// Negative and huge quotients (queries outside the grid) are clamped by
// the caller, so an inexact floor there changes nothing.
__device__ __forceinline__ long long cell_floor(float x, float min_f, float inv_f, double min_d,
                                                double cw)
{
    const float q = __fmul_rn(__fsub_rn(x, min_f), inv_f);
    const float f = floorf(q);
    const float tol = fabsf(q) * 0x1p-21f;
    // (a float32 -> int32 conversion saturates out of range; the caller
    // clamps, and the int64 conversion would run on the float64 pipe)
    if (q - f > tol && (f + 1.0f) - q > tol) return (long long)__float2int_rz(f);
    return (long long)floor(((double)x - min_d) / cw);
}

// Row-major cell of the point (x, y), clamped to the grid.
__device__ __forceinline__ int cell_index(float x, float y, const GridDev *g)
{
    const long long nc = g->n_col, nr = g->n_row;
    long long col = cell_floor(x, g->min_x_f, g->inv_cw_f, g->min_x, g->cw);
    long long row = cell_floor(y, g->min_y_f, g->inv_cw_f, g->min_y, g->cw);
    col = col < 0 ? 0 : (col > nc - 1 ? nc - 1 : col);
    row = row < 0 ? 0 : (row > nr - 1 ? nr - 1 : row);
    return (int)(row * nc + col);
}

// Cell of the point (x, y) stored as item i, and its (unstable) rank among
// the items of that cell.
__device__ __forceinline__ void key_one_xy(long long i, float x, float y, const GridDev *g,
                                           int *__restrict__ count, int *__restrict__ key,
                                           int *__restrict__ rank)
{
    const int c = cell_index(x, y, g);
    key[i] = c;
    rank[i] = AIDW_IN(c, g->n_cells, bounds::kKeyCell) ? atomicAdd(count + c, 1) : 0;
}

// Cell of data point i and its (unstable) rank among the points of that cell.
__device__ __forceinline__ void key_one(long long i, const float *__restrict__ x,
                                        const float *__restrict__ y, const GridDev *g,
                                        int *__restrict__ count, int *__restrict__ key,
                                        int *__restrict__ rank)
{
    key_one_xy(i, x[i], y[i], g, count, key, rank);
}

// Block-wide exclusive scan of one value per thread; total gets the sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int &total)
{
    __shared__ int warp_tot[kThreads / 32];
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (l >= o) incl += t;
    }
    if (l == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int t = l < kThreads / 32 ? warp_tot[l] : 0;
        int ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, ti, o);
            if (l >= o) ti += u;
        }
        if (l < kThreads / 32) warp_tot[l] = ti - t;  // exclusive warp offsets
        if (l == kThreads / 32 - 1) total = ti;
    }
    __syncthreads();
    const int r = warp_tot[w] + incl - v;
    __syncthreads();
    return r;
}

// ---- single-pass exclusive scan (decoupled look-back) --------------------------
// In-place exclusive scan of a[0, len) in chunks of kScanChunk, one chunk per
// block, in one launch.  Blocks take their chunk from an atomic ticket, so
// every chunk before a block's own belongs to a block that has already
// started.  A block publishes its chunk sum (flag 1), then its first warp
// looks back over the preceding chunks' records 32 at a time (lane i reads
// the i-th nearest), adding sums up to the nearest inclusive prefix (flag
// 2); the block publishes its own inclusive prefix and scans its chunk from
// there.  Records are 64-bit (flag << 32 | value), written with release and
// read with acquire semantics.  Waiting for a record that is not yet
// published is bounded: after kLookbackTries rounds the block sets
// kStatusTimeout in *status and carries on (the result is then wrong and the
// caller reports the error).  flags[] (one per chunk) and *ticket must be
// zero before the launch; values are int32 (sums up to 2^31 - 1).
constexpr int kLookbackTries = 1 << 22;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void scan_lookback_block(int *__restrict__ a, long long len,
                                                    unsigned long long *flags, int *ticket,
                                                    int *status)
{
    __shared__ long long chunk_s;
    __shared__ int prefix_s;
    __shared__ int tot;
    if (threadIdx.x == 0) chunk_s = atomicAdd(ticket, 1);
    __syncthreads();
    const long long chunk = chunk_s;
    const long long base = chunk * kScanChunk + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < len) ? a[base + j] : 0;
        sum += v[j];
    }
    const int ex = block_exclusive_scan(sum, tot);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int prefix = 0;
        if (chunk == 0) {
            if (lane == 0) st_release_u64(flags, (2ull << 32) | (unsigned)tot);
        } else {
            if (lane == 0) st_release_u64(flags + chunk, (1ull << 32) | (unsigned)tot);
            long long j = chunk - 1;  // nearest predecessor not yet added
            int tries = 0;
            for (;;) {
                const long long at = j - lane;
                // chunk 0 always publishes an inclusive prefix, so a window
                // reaching below it never needs those lanes
                const unsigned long long r = at >= 0 ? ld_acquire_u64(flags + at) : (2ull << 32);
                const unsigned f = (unsigned)(r >> 32);
                const unsigned inc = __ballot_sync(0xffffffffu, f == 2);
                const unsigned pending = __ballot_sync(0xffffffffu, f == 0);
                const int first = inc ? __ffs(inc) - 1 : 31;           // lanes 0..first are needed
                const unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
                if (pending & need) {
                    if (++tries > kLookbackTries) {
                        if (lane == 0) atomicOr(status, kStatusTimeout);
                        break;
                    }
                    continue;
                }
                int add = lane <= first ? (int)(unsigned)r : 0;
                for (int o = 16; o > 0; o >>= 1) add += __shfl_xor_sync(0xffffffffu, add, o);
                prefix += add;
                if (inc) break;
                j -= 32;
            }
            if (lane == 0) st_release_u64(flags + chunk, (2ull << 32) | (unsigned)(prefix + tot));
        }
        if (lane == 0) prefix_s = prefix;
    }
    __syncthreads();
    int run = prefix_s + ex;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < len) a[base + j] = run;
        run += v[j];
    }
}

__device__ __forceinline__ void scatter_one(long long i, const int *__restrict__ start,
                                            const int *__restrict__ key,
                                            const int *__restrict__ rank, int *__restrict__ tmp,
                                            long long n_out)
{
    const int dest = start[key[i]] + rank[i];
    if (!AIDW_IN(dest, n_out, bounds::kScatterDest)) return;
    tmp[dest] = (int)i;
}

// Data point i goes to its cell's segment (in arrival order) as a whole
// record, read here in input order: the fix-up then reads the records back
// in cell order instead of gathering x, y, z and the key of each point from
// arrays that, past a few million points, no longer fit in L2.
__device__ __forceinline__ void scatter_point(long long i, const float *__restrict__ x,
                                              const float *__restrict__ y,
                                              const float *__restrict__ z,
                                              const int *__restrict__ start,
                                              const int *__restrict__ key,
                                              const int *__restrict__ rank,
                                              Point *__restrict__ tmp,
                                              const GridDev *__restrict__ g, long long n)
{
    const int c = key[i];
    if (!AIDW_IN(c, g->n_cells, bounds::kScatterHead)) return;
    const int dest = start[c] + rank[i];
    if (!AIDW_IN(dest, n, bounds::kScatterDest)) return;
    Point p;
    p.x = x[i];
    p.y = y[i];
    p.z = z[i];
    p.idx = (int)i;
    tmp[dest] = p;
}

// Position s holds some point i of cell c (recomputed from its coordinates
// by the arithmetic that keyed it); its stable place is the head of c plus
// the number of indices smaller than i in c's segment.  The point is
// written there in both layouts.
__device__ __forceinline__ void fixup_one(long long s, const GridDev *__restrict__ g,
                                          const int *__restrict__ start,
                                          const Point *__restrict__ tmp, Point *__restrict__ pts,
                                          int *__restrict__ perm, float *__restrict__ wt,
                                          long long n)
{
    const Point p = tmp[s];
    const int i = p.idx;
    const int c = cell_index(p.x, p.y, g);
    if (!AIDW_IN(c, g->n_cells, bounds::kFixupHead)) return;
    const int a = start[c], b = start[c + 1];
    if (!AIDW_IN(b - 1, n, bounds::kFixupSegment)) return;
    int r = 0;
    for (int t = a; t < b; ++t) r += (tmp[t].idx < i);
    const long long pos = (long long)a + r;
    if (!AIDW_IN(pos, n, bounds::kFixupDest)) return;
    pts[pos] = p;
    perm[pos] = i;
    float *tile = wt + (pos / kWeightTile) * (3 * kWeightTile) + pos % kWeightTile;
    tile[0] = -p.x;
    tile[kWeightTile] = -p.y;
    tile[2 * kWeightTile] = p.z;
}

// Padding position i >= n: +inf coordinates, whose weight is exactly 0
// (d^2 = inf, log2 = inf, exp2(-inf) = 0), in both layouts.
__device__ __forceinline__ void pad_one(long long i, long long n_pad, long long n_wpad,
                                        Point *__restrict__ pts, float *__restrict__ wt)
{
    const float inf = __int_as_float(0x7f800000);
    if (i < n_pad) {
        Point p;
        p.x = inf;
        p.y = inf;
        p.z = 0.0f;
        p.idx = -1;
        pts[i] = p;
    }
    if (i < n_wpad) {
        float *tile = wt + (i / kWeightTile) * (3 * kWeightTile) + i % kWeightTile;
        tile[0] = -inf;
        tile[kWeightTile] = -inf;
        tile[2 * kWeightTile] = 0.0f;
    }
}

}  // namespace gridk
}  // namespace aidw
