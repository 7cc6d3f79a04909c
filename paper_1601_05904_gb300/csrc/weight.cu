// Weighting stage: Eq. 1 of arXiv 1601.05904 summed over ALL data points.
//
// Work decomposition (stream-K).  The pair space is cut into units of one
// query tile (kQPT queries per thread x kThreads threads) by one piece of a
// data tile (kDTile cell-ordered points, or 1/2 .. 1/16 of them when the
// point set is too small to give every CTA several whole tiles).  Units are
// numbered tile-major (u = t * D + d) and every resident CTA of a persistent
// grid takes one contiguous, equal share of them, so all SMs finish together
// whatever the query count.  A CTA's share covers the tail of one query tile, whole tiles
// and the head of another; for each query tile it touches it writes one
// partial (sum w, sum w z) per query to slot (tile + cta) of a scratch array,
// and a finalize kernel adds the pieces of each query in CTA order
// (deterministic, no atomics).  Many independent jobs (each its own data and
// queries) run in the same launch by numbering their units, query tiles and
// queries one job after the other; a CTA finds the job of a unit by binary
// search in the job table, so one launch balances jobs of any sizes.
//
// Data staging.  One elected thread streams each data tile into shared
// memory with bulk (TMA) copies that complete on an mbarrier, kStages tiles
// ahead.  The float32 path stages a tile as three cell-ordered arrays
// (-x, -y, z); every thread reads four consecutive values of each with one
// broadcast 16-byte shared load and applies them, two points per packed
// f32x2 instruction, to its kQPT queries held in registers.  The float64
// path stages the tile as one run of 16-byte points.
//
// Float32 path (AIDW_FP32_COMP).  With d1^2 the smallest squared distance of
// the query (from the kNN stage, computed by the same float32 code):
//     w = (d^2 / d1^2)^(-alpha/2) = exp2(c * log2(d^2) + b),
//     c = -alpha/2, b = -c * log2(d1^2)
// which is Eq. 1's weight d^-alpha multiplied by d1^alpha (cancels in the
// ratio) and is at most 1, so nothing overflows.  log2 and exp2 are the SFU
// approximations, except for a fixed share of the exp2s (and, as an option,
// log2s) evaluated by polynomials on the FMA pipe to balance the two pipes.
// Sums over kChunk points per lane are plain float32; the chunk sums are
// added into a (hi, lo) pair with TwoSum, and the final ratio is formed in
// float64.
//
// Float64 path (AIDW_FP64_PLAIN): w = pow(d^2, -alpha/2) in float64, plain
// float64 sums, same decomposition.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <type_traits>

#include "aidw_device.cuh"
#include "aidw_internal.cuh"
#include "weight_loop.cuh"

namespace aidw {

namespace {

constexpr int kDTile = 2048;   // points per shared-memory stage
static_assert(kDTile == kWeightTile, "weighting tiles are staged whole");
constexpr int kStages = 3;
constexpr int kWaitTries = 2000;  // tries of up to ~1 ms: a data-tile wait gives up after ~2 s

template <bool F64>
struct WCfg;
// float32: 256 threads x 4 queries at 128 registers (2 CTAs per SM).  512 x 2
// at 64 registers (twice the warps) measured 360 vs 353 ms at n = m = 1M.
template <>
struct WCfg<false> {
    static constexpr int kThreads = 256;
    static constexpr int kQPT = 4;
    static constexpr int kQTile = kThreads * kQPT;
    static constexpr int kMinBlocks = 2;
    using Part = float4;
};
template <>
struct WCfg<true> {
    static constexpr int kThreads = 256;
    static constexpr int kQPT = 2;
    static constexpr int kQTile = kThreads * kQPT;
    static constexpr int kMinBlocks = 1;
    using Part = double2;
};

// First unit of CTA j when U units are split over G CTAs.
__host__ __device__ __forceinline__ long long sk_begin(long long j, long long U, long long G)
{
    return (j * U) / G;
}
// CTA whose share contains unit u.
__host__ __device__ __forceinline__ long long sk_owner(long long u, long long U, long long G)
{
    return ((u + 1) * G - 1) / U;
}

struct SKArgs {
    WJob job0;          // the job of a single-job launch (jobs == nullptr)
    const WJob *jobs;   // job table of a batched launch
    int n_jobs;
    long long U;        // units of all jobs
    long long G;        // CTAs
    const long long *bounds;  // [G + 1] first unit of each CTA's share, strictly
                              // increasing (cost-balanced, batched launches); or
                              // null for equal unit counts
    long long total_q;  // queries of all jobs
    long long n_slots;  // partial-sum slots of the scratch array (query tiles + CTAs)
    int *status;
    int *fail;          // this launch's failure flag: zeroed before the launch, set by a
                        // CTA whose wait expired; the finalize then writes NaN
    int wait_tries;     // bound of every mbarrier wait (tries; hook launches only)
    long long skip_unit;  // test hook: the data tile of this unit is never
                          // copied, so its wait expires (-1: none)
};

// Share of CTA j and the owner of unit u, from the launch's boundaries.
__device__ __forceinline__ long long share_begin(const SKArgs &a, long long j)
{
    return a.bounds ? a.bounds[j] : sk_begin(j, a.U, a.G);
}
__device__ __forceinline__ long long share_owner(const SKArgs &a, long long u)
{
    if (!a.bounds) return sk_owner(u, a.U, a.G);
    long long lo = 0, hi = a.G - 1;  // the last CTA whose share starts at or before u
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (a.bounds[mid] <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ WJob job_of_unit(const SKArgs &a, long long u)
{
    if (!a.jobs) return a.job0;
    int lo = 0, hi = a.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.jobs[mid].unit_base <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return a.jobs[lo];
}

__device__ __forceinline__ WJob job_of_query(const SKArgs &a, long long gq)
{
    if (!a.jobs) return a.job0;
    int lo = 0, hi = a.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.jobs[mid].q_base <= gq)
            lo = mid;
        else
            hi = mid - 1;
    }
    return a.jobs[lo];
}

// Points of data unit d (pieces of kDTile >> shift points) that the float32
// kernel processes: the valid ones rounded up to kChunk2 (the tile's padding
// has weight 0).
constexpr int kMaxPieceShift = 4;
static_assert((kDTile >> kMaxPieceShift) % kChunk2 == 0, "pieces are whole chunks");
__host__ __device__ __forceinline__ int soa_count(long long n_data, long long d, int shift)
{
    const long long piece = kDTile >> shift;
    const long long rem = n_data - d * piece;
    const long long c = (rem + kChunk2 - 1) / kChunk2 * kChunk2;
    return (int)(c < piece ? c : piece);
}

// Points of data tile d in the float64 kernel's AoS layout.
__device__ __forceinline__ int aos_count(long long n_pad, long long d)
{
    return (int)min((long long)kDTile, n_pad - d * kDTile);
}

template <bool HOOK, bool PIECES>
__device__ __forceinline__ void issue_tile_soa(const SKArgs &a, float *buf, uint64_t *bar,
                                               long long u)
{
    if (HOOK && u == a.skip_unit) return;
    const WJob J = job_of_unit(a, u);
    const int sh = PIECES ? J.piece_shift : 0;
    const long long d = (u - J.unit_base) % J.D;
    const uint32_t bytes = (uint32_t)soa_count(J.n_data, d, sh) * 4u;
    // piece d is piece (d mod 2^sh) of weighting tile (d >> sh); pieces are
    // multiples of kChunk2 points, so every copy starts 512-byte aligned
    const long long piece = kDTile >> sh;
    if (!AIDW_IN(d >> sh, (J.n_data + kDTile - 1) / kDTile, bounds::kWeightTile) ||
        !AIDW_IN((d & ((1LL << sh) - 1)) * piece + bytes / 4 - 1, kDTile, bounds::kWeightPiece))
        return;  // (checked build) the copy is skipped; the consumer's bounded wait expires
    const float *src = J.wt + (d >> sh) * (3 * kDTile) + (d & ((1LL << sh) - 1)) * piece;
    mbar_expect_tx(bar, 3u * bytes);
    bulk_g2s(buf, src, bytes, bar);
    bulk_g2s(buf + kDTile, src + kDTile, bytes, bar);
    bulk_g2s(buf + 2 * kDTile, src + 2 * kDTile, bytes, bar);
}

template <bool HOOK>
__device__ __forceinline__ void issue_tile_aos(const SKArgs &a, Point *buf, uint64_t *bar,
                                               long long u)
{
    if (HOOK && u == a.skip_unit) return;
    const WJob J = job_of_unit(a, u);
    const long long d = (u - J.unit_base) % J.D;
    const uint32_t bytes = (uint32_t)aos_count(J.n_pad, d) * (uint32_t)sizeof(Point);
    if (!AIDW_IN(d * kDTile + bytes / sizeof(Point) - 1, J.n_pad, bounds::kWeightPiece)) return;
    mbar_expect_tx(bar, bytes);
    bulk_g2s(buf, J.pts + d * kDTile, bytes, bar);
}

// ---------------------------------------------------------------------------
// float32 compensated weighting
// ---------------------------------------------------------------------------
// Each thread holds kQPT queries; every packed instruction applies one query
// to two consecutive data points (lanes), so a 16-byte shared load of the
// tile's x (or y, z) array feeds two packed operands.
// PE, PL: how many of the 2 x kQPT (point pair, query) products of one inner
// step take exp2 (PE, counted from the first product) and lg2 (PL, counted
// from the last) from FMA-pipe polynomials instead of the SFU.  The SFU
// evaluates lg2 at half the rate of ex2, so with one of each per pair the SFU
// is the bound; moving part of the work to the FMA pipe balances the two.
// HOOK: the instantiation launched only while the timeout test hook is armed
// (aidw_test_expire_next_wait); the normal kernel has no trace of it.
// PIECES: units may be pieces of a data tile (WJob::piece_shift); the
// whole-tile instantiation keeps the shift out of the kernel, which measured
// 1.5 % faster at n = m = 1M (334.1 against 339.2 ms).
template <int PE, int PL, bool HOOK = false, int PE2 = PE, int THREADS = WCfg<false>::kThreads,
          int Q = WCfg<false>::kQPT, int MINB = WCfg<false>::kMinBlocks, bool PIECES = false>
__global__ void __launch_bounds__(THREADS, MINB)
    k_weight_f32(SKArgs a, float4 *__restrict__ part)
{
    const int wait_tries = HOOK ? a.wait_tries : kWaitTries;
    using C = WCfg<false>;
    static_assert(THREADS * Q == C::kQTile, "a query tile is THREADS x Q queries");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *buf = reinterpret_cast<float *>(smem_raw);
    __shared__ __align__(8) uint64_t full[kStages];

    const long long cta = blockIdx.x;
    const long long u0 = share_begin(a, cta), u1 = share_begin(a, cta + 1);
    if (u0 >= u1) return;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < kStages; ++s)
            if (u0 + s < u1)
                issue_tile_soa<HOOK, PIECES>(a, buf + s * 3 * kDTile, &full[s], u0 + s);

    const F2 zero2 = f2_pack(0.0f, 0.0f);
    long long u = u0;
    while (u < u1) {
        const WJob J = job_of_unit(a, u);
        const long long t = (u - J.unit_base) / J.D;
        const long long seg_end = min(u1, J.unit_base + (t + 1) * J.D);

        F2 qx2[Q], qy2[Q], c2[Q], b2[Q], hw[Q], lw[Q], hz[Q], lz[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const long long q = t * C::kQTile + (long long)i * THREADS + threadIdx.x;
            float qx = 0.0f, qy = 0.0f, c = -1.0f, b = 0.0f;
            if (q < J.nq) {
                qx = J.qx[q];
                qy = J.qy[q];
                const QRec r = J.recs[q];
                if (r.n_hit > 0 || !(r.alpha == r.alpha)) {
                    c = 0.0f;  // result replaced in the finalize step
                } else {
                    c = (float)(-0.5 * r.alpha);
                    b = -c * lg2_sfu(r.d1sq);
                }
            }
            qx2[i] = f2_pack(qx, qx);
            qy2[i] = f2_pack(qy, qy);
            c2[i] = f2_pack(c, c);
            b2[i] = f2_pack(b, b);
            hw[i] = lw[i] = hz[i] = lz[i] = zero2;
        }

        for (; u < seg_end; ++u) {
            const int s = (int)((u - u0) % kStages);
            const uint32_t par = (uint32_t)(((u - u0) / kStages) & 1);
            const bool ok = mbar_wait_bounded(&full[s], par, wait_tries);
            const float *X = buf + s * 3 * kDTile;
            const float *Y = X + kDTile;
            const float *Z = Y + kDTile;
            const int cnt =
                soa_count(J.n_data, (u - J.unit_base) % J.D, PIECES ? J.piece_shift : 0);
            if (ok) {
                for (int c0 = 0; c0 < cnt; c0 += kChunk2) {
                    F2 ps[Q], pz[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) ps[i] = pz[i] = zero2;
                    weight_chunk_f32<Q, PE, PL, PE2>(X, Y, Z, c0, qx2, qy2, c2, b2, ps, pz);
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        f2_comp_add(hw[i], lw[i], ps[i]);
                        f2_comp_add(hz[i], lz[i], pz[i]);
                    }
                }
            }
            // every thread is done with stage s before it is refilled
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) {
                    atomicOr(a.status, kStatusTimeout);
                    atomicOr(a.fail, 1);
                }
                // drain the copies this CTA still has in flight, then leave
                if (threadIdx.x == 0)
                    for (long long v = u; v < min(u1, u + kStages); ++v)
                        mbar_wait_bounded(&full[(v - u0) % kStages],
                                          (uint32_t)(((v - u0) / kStages) & 1), wait_tries);
                __syncthreads();
                return;
            }
            if (threadIdx.x == 0 && u + kStages < u1)
                issue_tile_soa<HOOK, PIECES>(a, buf + s * 3 * kDTile, &full[s], u + kStages);
        }

        const long long slot = J.tile_base + t + cta;
        if (!AIDW_IN(slot, a.n_slots, bounds::kWeightSlot)) continue;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float w0, w1, wl0, wl1, z0, z1, zl0, zl1;
            f2_unpack(hw[i], w0, w1);
            f2_unpack(lw[i], wl0, wl1);
            f2_unpack(hz[i], z0, z1);
            f2_unpack(lz[i], zl0, zl1);
            comp_add(w0, wl0, w1);
            comp_add(z0, zl0, z1);
            part[slot * C::kQTile + (long long)i * THREADS + threadIdx.x] =
                make_float4(w0, add_rn(wl0, wl1), z0, add_rn(zl0, zl1));
        }
    }
}

// Adds the pieces of each query's partial sums in CTA order and divides.
__global__ void k_finalize_f32(SKArgs a, const float4 *__restrict__ part)
{
    using C = WCfg<false>;
    const long long gq = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gq >= a.total_q) return;
    const WJob J = job_of_query(a, gq);
    const long long q = gq - J.q_base;
    float *out_z = static_cast<float *>(J.out_z);
    const QRec r = J.recs[q];
    if (!(r.alpha == r.alpha) || *a.fail) {  // non-finite query, or a sum cut short
        out_z[q] = __int_as_float(0x7fc00000);
        return;
    }
    if (r.n_hit > 0) {
        out_z[q] = (float)r.hit_z;
        return;
    }
    const long long t = q / C::kQTile, l = q % C::kQTile;
    const long long ub = J.unit_base + t * J.D;
    const long long j0 = share_owner(a, ub), j1 = share_owner(a, ub + J.D - 1);
    float hw = 0.0f, lw = 0.0f, hz = 0.0f, lz = 0.0f;
    for (long long j = j0; j <= j1; ++j) {
        if (!AIDW_IN(J.tile_base + t + j, a.n_slots, bounds::kWeightSlot)) break;
        const float4 v = part[(J.tile_base + t + j) * C::kQTile + l];
        comp_add(hw, lw, v.x);
        lw = add_rn(lw, v.y);
        comp_add(hz, lz, v.z);
        lz = add_rn(lz, v.w);
    }
    out_z[q] = (float)(((double)hz + (double)lz) / ((double)hw + (double)lw));
}

// ---------------------------------------------------------------------------
// float64 plain weighting
// ---------------------------------------------------------------------------
template <bool HOOK = false>
__global__ void __launch_bounds__(WCfg<true>::kThreads, WCfg<true>::kMinBlocks)
    k_weight_f64(SKArgs a, double2 *__restrict__ part)
{
    const int wait_tries = HOOK ? a.wait_tries : kWaitTries;
    using C = WCfg<true>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Point *buf = reinterpret_cast<Point *>(smem_raw);
    __shared__ __align__(8) uint64_t full[kStages];

    const long long cta = blockIdx.x;
    const long long u0 = share_begin(a, cta), u1 = share_begin(a, cta + 1);
    if (u0 >= u1) return;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < kStages; ++s)
            if (u0 + s < u1) issue_tile_aos<HOOK>(a, buf + s * kDTile, &full[s], u0 + s);

    long long u = u0;
    while (u < u1) {
        const WJob J = job_of_unit(a, u);
        const long long t = (u - J.unit_base) / J.D;
        const long long seg_end = min(u1, J.unit_base + (t + 1) * J.D);
        float qx[C::kQPT], qy[C::kQPT];
        double e[C::kQPT], sw[C::kQPT], swz[C::kQPT];
#pragma unroll
        for (int i = 0; i < C::kQPT; ++i) {
            const long long q = t * C::kQTile + (long long)i * C::kThreads + threadIdx.x;
            qx[i] = 0.0f;
            qy[i] = 0.0f;
            e[i] = -1.0;
            if (q < J.nq) {
                qx[i] = J.qx[q];
                qy[i] = J.qy[q];
                const double al = J.recs[q].alpha;
                if (al == al) e[i] = -0.5 * al;
            }
            sw[i] = swz[i] = 0.0;
        }
        for (; u < seg_end; ++u) {
            const int s = (int)((u - u0) % kStages);
            const uint32_t par = (uint32_t)(((u - u0) / kStages) & 1);
            const bool ok = mbar_wait_bounded(&full[s], par, wait_tries);
            const Point *tile = buf + s * kDTile;
            const int cnt = aos_count(J.n_pad, (u - J.unit_base) % J.D);
            if (ok) {
                for (int jj = 0; jj < cnt; ++jj) {
                    const float4 p = reinterpret_cast<const float4 *>(tile)[jj];
#pragma unroll
                    for (int i = 0; i < C::kQPT; ++i) {
                        const double w = pow(dist2_f64(qx[i], qy[i], p.x, p.y), e[i]);
                        sw[i] += w;
                        swz[i] = fma(w, (double)p.z, swz[i]);
                    }
                }
            }
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) {
                    atomicOr(a.status, kStatusTimeout);
                    atomicOr(a.fail, 1);
                }
                if (threadIdx.x == 0)
                    for (long long v = u; v < min(u1, u + kStages); ++v)
                        mbar_wait_bounded(&full[(v - u0) % kStages],
                                          (uint32_t)(((v - u0) / kStages) & 1), wait_tries);
                __syncthreads();
                return;
            }
            if (threadIdx.x == 0 && u + kStages < u1)
                issue_tile_aos<HOOK>(a, buf + s * kDTile, &full[s], u + kStages);
        }
        const long long slot = J.tile_base + t + cta;
        if (!AIDW_IN(slot, a.n_slots, bounds::kWeightSlot)) continue;
#pragma unroll
        for (int i = 0; i < C::kQPT; ++i)
            part[slot * C::kQTile + (long long)i * C::kThreads + threadIdx.x] =
                make_double2(sw[i], swz[i]);
    }
}

__global__ void k_finalize_f64(SKArgs a, const double2 *__restrict__ part)
{
    using C = WCfg<true>;
    const long long gq = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gq >= a.total_q) return;
    const WJob J = job_of_query(a, gq);
    const long long q = gq - J.q_base;
    double *out_z = static_cast<double *>(J.out_z);
    const QRec r = J.recs[q];
    if (!(r.alpha == r.alpha) || *a.fail) {  // non-finite query, or a sum cut short
        out_z[q] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    if (r.n_hit > 0) {
        out_z[q] = r.hit_z;
        return;
    }
    const long long t = q / C::kQTile, l = q % C::kQTile;
    const long long ub = J.unit_base + t * J.D;
    const long long j0 = share_owner(a, ub), j1 = share_owner(a, ub + J.D - 1);
    double sw = 0.0, swz = 0.0;
    for (long long j = j0; j <= j1; ++j) {
        if (!AIDW_IN(J.tile_base + t + j, a.n_slots, bounds::kWeightSlot)) break;
        const double2 v = part[(J.tile_base + t + j) * C::kQTile + l];
        sw += v.x;
        swz += v.y;
    }
    out_z[q] = swz / sw;
}

// Polynomial split of the float32 kernel: products per inner step whose exp2
// (first number) and lg2 (second) run on the FMA pipe, and (third) the exp2
// products of every second step where steps alternate.  Measured on GB300 at
// n = m = 1M (weighting ms, 64-point chunks, point loop unrolled 16x):
// {2,0} 334.8, {0,0} 352.4, {3,0} 354.8, {4,0} 382.1, {0,1} 345.3,
// {1,1} 348.3, {0,2} 369.2, so {2,0} is the default.  AIDW_WEIGHT_POLY
// ("E,L" or "E,L,E2") selects another entry of the table, for measuring the
// balance on a given GPU.
// Each entry holds the whole-tile kernel and, for the default split, the
// kernel that also takes pieces of tiles (other splits run whole tiles).
using F32Kernel = void (*)(SKArgs, float4 *);
struct PolySplit {
    int e, l, e2;
    F32Kernel kernel;
    F32Kernel pieces;
};
using WCf = WCfg<false>;
const PolySplit kPolySplits[] = {
    {2, 0, 2, k_weight_f32<2, 0>,
     k_weight_f32<2, 0, false, 2, WCf::kThreads, WCf::kQPT, WCf::kMinBlocks, true>},
    {0, 0, 0, k_weight_f32<0, 0>, nullptr}, {3, 0, 3, k_weight_f32<3, 0>, nullptr},
    {4, 0, 4, k_weight_f32<4, 0>, nullptr}, {0, 1, 0, k_weight_f32<0, 1>, nullptr},
    {1, 1, 1, k_weight_f32<1, 1>, nullptr}, {0, 2, 0, k_weight_f32<0, 2>, nullptr},
    {2, 0, 3, k_weight_f32<2, 0, false, 3>, nullptr},
    {1, 0, 2, k_weight_f32<1, 0, false, 2>, nullptr}};
// The kernel of the timeout test hook takes pieces too (any launch may arm it).
constexpr F32Kernel kHookKernel =
    k_weight_f32<2, 0, true, 2, WCf::kThreads, WCf::kQPT, WCf::kMinBlocks, true>;
constexpr int kNumPolySplits = (int)(sizeof(kPolySplits) / sizeof(kPolySplits[0]));
const PolySplit &f32_split()
{
    static const int idx = [] {
        const char *e = getenv("AIDW_WEIGHT_POLY");
        int pe = -1, pl = -1, pe2 = -1;
        const int got = e ? sscanf(e, "%d,%d,%d", &pe, &pl, &pe2) : 0;
        if (got == 2) pe2 = pe;
        if (got >= 2)
            for (int i = 0; i < kNumPolySplits; ++i)
                if (kPolySplits[i].e == pe && kPolySplits[i].l == pl && kPolySplits[i].e2 == pe2)
                    return i;
        return 0;
    }();
    return kPolySplits[idx];
}
F32Kernel f32_kernel() { return f32_split().kernel; }

// Work of the float32 loop per (query, data point) pair, counted from the
// source above and from f2_exp2_poly / f2_log2_poly (aidw_device.cuh), for
// roofline accounting.  FMA-pipe lane operations: the base loop takes 7 (two
// differences, the squared distance as a multiply and an fma, the exponent
// fma, the two sums); an exp2 polynomial 8 (three for the reduction, five
// fmas); a log2 polynomial 10 (two for the reduction, eight fmas).
// Instructions other than the SFU's own (a packed f32x2 instruction covers
// two pairs): base 3.5; exp2 polynomial 7 (four packed, one fmax and two
// integer exponent operations per lane); log2 polynomial 12 (five packed,
// five integer operations and a compare-select per lane).  Loads, loop
// control and the chunk folds (about 0.2 per pair) are not included.
constexpr double kFmaLanes[3] = {7.0, 8.0, 10.0};
constexpr double kInstr[3] = {3.5, 7.0, 12.0};

// Dynamic shared memory of the weighting kernels: kStages data tiles.
template <bool F64>
constexpr size_t stage_smem()
{
    return F64 ? (size_t)kStages * kDTile * sizeof(Point)
               : (size_t)kStages * 3 * kDTile * sizeof(float);
}

template <bool F64>
int resident_ctas(int device)
{
    static std::mutex mu;
    static int cached[2][64] = {};
    if (device < 0 || device >= 64) return 1;
    std::lock_guard<std::mutex> lk(mu);
    int &c = cached[F64 ? 1 : 0][device];
    if (c) return c;
    const size_t smem = stage_smem<F64>();
    int sms = 1, per_sm = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (F64) {
        cudaFuncSetAttribute(k_weight_f64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        cudaFuncSetAttribute(k_weight_f64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_weight_f64<false>,
                                                      WCfg<true>::kThreads, smem);
    } else {
        for (int i = 0; i < kNumPolySplits; ++i) {
            cudaFuncSetAttribute(kPolySplits[i].kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (kPolySplits[i].pieces)
                cudaFuncSetAttribute(kPolySplits[i].pieces,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        }
        cudaFuncSetAttribute(kHookKernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f32_kernel(),
                                                      WCfg<false>::kThreads, smem);
    }
    c = std::max(1, sms * std::max(1, per_sm));
    return c;
}

// Test hook (aidw_test_expire_next_wait): the next weighting launch skips
// the copy of its first unit's data tile and bounds its waits at the given
// number of tries, so the wait expires and the timeout path runs.
std::mutex g_hook_mu;
int g_hook_tries = 0;

// Launches the weighting kernel and the finalize kernel for the jobs in a.
template <bool F64>
aidw_status launch(SKArgs a, void *part, cudaStream_t s)
{
    NvtxRange nvtx_("weighting");
    a.wait_tries = kWaitTries;
    a.skip_unit = -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cudaGetLastError();
    if (cs == cudaStreamCaptureStatusNone) {  // never bake the hook into a graph
        std::lock_guard<std::mutex> lk(g_hook_mu);
        if (g_hook_tries > 0) {
            a.wait_tries = g_hook_tries;
            a.skip_unit = 0;
            g_hook_tries = 0;
        }
    }
    using C = WCfg<F64>;
    using Part = typename C::Part;
    const size_t smem = stage_smem<F64>();
    int prof = profile_begin(s);
    cudaMemsetAsync(a.fail, 0, sizeof(int), s);
    if (F64) {
        if (a.skip_unit >= 0)
            k_weight_f64<true><<<(unsigned)a.G, C::kThreads, smem, s>>>(a, static_cast<double2 *>(part));
        else
            k_weight_f64<<<(unsigned)a.G, C::kThreads, smem, s>>>(a, static_cast<double2 *>(part));
    } else if (a.skip_unit >= 0) {
        kHookKernel<<<(unsigned)a.G, C::kThreads, smem, s>>>(a, static_cast<float4 *>(part));
    } else {
        // only single-job launches cut tiles into pieces
        const F32Kernel k = (!a.jobs && a.job0.piece_shift > 0) ? f32_split().pieces
                                                                  : f32_split().kernel;
        k<<<(unsigned)a.G, C::kThreads, smem, s>>>(a, static_cast<float4 *>(part));
    }
    profile_end(prof, s, AIDW_STAGE_WEIGHT, 1);
    prof = profile_begin(s);
    const unsigned fb = (unsigned)((a.total_q + 255) / 256);
    if (F64)
        k_finalize_f64<<<fb, 256, 0, s>>>(a, static_cast<const double2 *>(part));
    else
        k_finalize_f32<<<fb, 256, 0, s>>>(a, static_cast<const float4 *>(part));
    profile_end(prof, s, AIDW_STAGE_FINALIZE, 1);
    (void)sizeof(Part);
    return cuda_status(cudaGetLastError());
}

// Pieces per weighting tile (as a shift) for one job of n_data points and T
// query tiles on at most G_max CTAs: the shift whose largest CTA share, in
// points, is smallest, each unit charged kUnitCost points more for its
// barrier wait, copy issue and chunk folds (8: the fit of the measured
// 51,200-point step, 0.853 ms with 512-point pieces against 0.838 with
// 256, is about 6).  Whole tiles unless the point
// set is too small to give every CTA several of them (at n = m = 10,240:
// 50 whole-tile units for 304 CTAs, against 800 units of 128 points).
// AIDW_WEIGHT_PIECES=s (0..4) fixes the shift, for measurement.
int piece_shift_for(long long n_data, long long T, long long G_max)
{
    static const int forced = [] {
        const char *e = getenv("AIDW_WEIGHT_PIECES");
        int v = -1;
        if (e && sscanf(e, "%d", &v) == 1 && v >= 0 && v <= kMaxPieceShift) return v;
        return -1;
    }();
    if (!f32_split().pieces) return 0;  // this split runs whole tiles only
    if (forced >= 0) return forced;
    constexpr double kUnitCost = 8.0;
    int best = 0;
    double best_cost = 0.0;
    for (int sh = 0; sh <= kMaxPieceShift; ++sh) {
        const long long piece = kDTile >> sh;
        const long long U = T * ((n_data + piece - 1) / piece);
        const long long G = std::max(1LL, std::min(G_max, U));
        const double cost =
            (double)((U + G - 1) / G) * ((double)soa_count(n_data, 0, sh) + kUnitCost);
        if (sh == 0 || cost < best_cost) {
            best = sh;
            best_cost = cost;
        }
    }
    return best;
}

// The single job of a grid and one query set, on at most G_max CTAs.
template <bool F64>
SKArgs single_job(const aidw_grid *g, const float *qx, const float *qy, long long nq,
                  const QRec *recs, void *out_z, long long G_max)
{
    using C = WCfg<F64>;
    SKArgs a;
    memset(&a, 0, sizeof(a));
    WJob &J = a.job0;
    J.wt = g->wt;
    J.pts = g->pts;
    J.qx = qx;
    J.qy = qy;
    J.recs = recs;
    J.out_z = out_z;
    J.n_data = g->n_data;
    J.n_pad = g->n_pad;
    J.T = (nq + C::kQTile - 1) / C::kQTile;
    J.piece_shift = F64 ? 0 : piece_shift_for(g->n_data, J.T, G_max);
    const long long piece = kDTile >> J.piece_shift;
    J.D = F64 ? weight_data_tiles(g->n_data, g->n_pad, true) : (g->n_data + piece - 1) / piece;
    J.nq = nq;
    a.jobs = nullptr;
    a.n_jobs = 1;
    a.U = J.T * J.D;
    a.G = std::max(1LL, std::min(G_max, a.U));
    a.n_slots = J.T + a.G;
    a.total_q = nq;
    a.status = &g->dev->status;
    return a;
}

template <bool F64>
aidw_status run(const aidw_grid *g, const float *qx, const float *qy, long long nq,
                const QRec *recs, void *out_z, cudaStream_t s)
{
    using C = WCfg<F64>;
    SKArgs a = single_job<F64>(g, qx, qy, nq, recs, out_z, resident_ctas<F64>(g->device));
    void *part = nullptr;
    const size_t part_bytes = sizeof(typename C::Part) * (size_t)C::kQTile * (size_t)(a.job0.T + a.G);
    if (lib_alloc(&part, part_bytes + 256, s) != cudaSuccess) return AIDW_ERR_OOM;
    a.fail = reinterpret_cast<int *>(static_cast<unsigned char *>(part) + part_bytes);
    const aidw_status st = launch<F64>(a, part, s);
    lib_free(part, s);
    return st;
}

template <bool F64>
aidw_status run_scratch(const aidw_grid *g, const float *qx, const float *qy, long long nq,
                        const QRec *recs, void *out_z, void *scratch, size_t scratch_bytes,
                        cudaStream_t s)
{
    using C = WCfg<F64>;
    const long long slot_bytes = (long long)sizeof(typename C::Part) * C::kQTile;
    if (scratch_bytes < 512) return AIDW_ERR_INVALID_ARG;
    const size_t part_room = scratch_bytes - 256;  // the last 256 bytes hold the flag
    const long long T = (nq + C::kQTile - 1) / C::kQTile;
    const long long g_fit = (long long)(part_room / (size_t)slot_bytes) - T;
    if (g_fit < 1) return AIDW_ERR_INVALID_ARG;
    SKArgs a = single_job<F64>(g, qx, qy, nq, recs, out_z,
                               std::min<long long>(resident_ctas<F64>(g->device), g_fit));
    a.fail = reinterpret_cast<int *>(static_cast<unsigned char *>(scratch) + part_room);
    return launch<F64>(a, scratch, s);
}

}  // namespace

void weight_mix(int *products, int *poly_exp2, int *poly_lg2, double *fma_lanes, double *instr)
{
    // counted over two inner steps (the period of an alternating split)
    const PolySplit &sp = f32_split();
    if (products) *products = 2 * 2 * WCfg<false>::kQPT;
    if (poly_exp2) *poly_exp2 = sp.e + sp.e2;
    if (poly_lg2) *poly_lg2 = 2 * sp.l;
    for (int i = 0; i < 3; ++i) {
        if (fma_lanes) fma_lanes[i] = kFmaLanes[i];
        if (instr) instr[i] = kInstr[i];
    }
}

void weight_expire_next_wait(int tries)
{
    std::lock_guard<std::mutex> lk(g_hook_mu);
    g_hook_tries = tries;
}

long long weight_unit_points(long long n_data, long long n_pad, long long d, bool fp64)
{
    if (fp64) return std::min<long long>(kDTile, n_pad - d * kDTile);
    const long long rem = n_data - d * kDTile;
    return std::min<long long>(kDTile, (rem + kChunk2 - 1) / kChunk2 * kChunk2);
}

long long weight_data_tiles(long long n_data, long long n_pad, bool fp64)
{
    return fp64 ? (n_pad + kDTile - 1) / kDTile : (n_data + kDTile - 1) / kDTile;
}

long long weight_query_tile(bool fp64)
{
    return fp64 ? WCfg<true>::kQTile : WCfg<false>::kQTile;
}

int weight_resident_ctas(int device, bool fp64)
{
    return fp64 ? resident_ctas<true>(device) : resident_ctas<false>(device);
}

size_t weight_partial_bytes(bool fp64)
{
    return fp64 ? sizeof(WCfg<true>::Part) * WCfg<true>::kQTile
                : sizeof(WCfg<false>::Part) * WCfg<false>::kQTile;
}

aidw_status weight_launch_scratch(const aidw_grid *g, const float *qx, const float *qy,
                                  long long n_query, bool fp64, const QRec *recs, void *out_z,
                                  void *scratch, size_t scratch_bytes, cudaStream_t s)
{
    if (n_query <= 0) return AIDW_OK;
    return fp64 ? run_scratch<true>(g, qx, qy, n_query, recs, out_z, scratch, scratch_bytes, s)
                : run_scratch<false>(g, qx, qy, n_query, recs, out_z, scratch, scratch_bytes, s);
}

aidw_status weight_launch(const aidw_grid *g, const float *qx, const float *qy,
                          long long n_query, bool fp64, const QRec *recs, void *out_z,
                          cudaStream_t s)
{
    if (n_query <= 0) return AIDW_OK;
    return fp64 ? run<true>(g, qx, qy, n_query, recs, out_z, s)
                : run<false>(g, qx, qy, n_query, recs, out_z, s);
}

aidw_status weight_launch_batch(const WJob *jobs, int n_jobs, long long total_u,
                                long long total_q, bool fp64, void *part, long long G,
                                const long long *bounds, int *status, int *fail, int device,
                                cudaStream_t s, long long n_slots)
{
    if (total_u <= 0 || total_q <= 0) return AIDW_OK;
    SKArgs a;
    memset(&a, 0, sizeof(a));
    a.jobs = jobs;
    a.n_jobs = n_jobs;
    a.U = total_u;
    a.G = std::max<long long>(1, std::min<long long>(G, total_u));
    a.bounds = a.G == G ? bounds : nullptr;
    a.total_q = total_q;
    a.n_slots = n_slots;
    a.status = status;
    a.fail = fail;
    (void)device;
    return fp64 ? launch<true>(a, part, s) : launch<false>(a, part, s);
}

}  // namespace aidw
