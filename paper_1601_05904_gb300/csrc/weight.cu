// Weighting stage: Eq. 1 of arXiv 1601.05904 summed over ALL data points.
//
// Work decomposition (stream-K).  The pair space is cut into units of one
// query tile (kQPT queries per thread x kThreads threads) by one data tile
// (kDTile cell-ordered points).  Units are numbered tile-major
// (u = t * D + d) and every resident CTA of a persistent grid takes one
// contiguous, equal share of them, so all SMs finish together whatever the
// query count.  A CTA's share covers the tail of one query tile, whole tiles
// and the head of another; for each query tile it touches it writes one
// partial (sum w, sum w z) per query to slot (t + cta) of a scratch array,
// and a finalize kernel adds the pieces of each query in CTA order
// (deterministic, no atomics).
//
// Data staging.  Each data tile is one contiguous run of 16-byte points; one
// elected thread streams it into shared memory with a bulk (TMA) copy that
// completes on an mbarrier, kStages tiles ahead.  Every thread then reads
// each point as a broadcast 16-byte shared load and applies it to its kQPT
// queries held in registers.
//
// Float32 path (AIDW_FP32_COMP).  With d1^2 the smallest squared distance of
// the query (from the kNN stage, computed by the same float32 code):
//     w = (d^2 / d1^2)^(-alpha/2) = exp2(c * log2(d^2) + b),
//     c = -alpha/2, b = -c * log2(d1^2)
// which is Eq. 1's weight d^-alpha multiplied by d1^alpha (cancels in the
// ratio) and is at most 1, so nothing overflows.  log2 and exp2 are the SFU
// approximations.  Sums over kChunk points are plain float32; the chunk sums
// are added into a (hi, lo) pair with TwoSum, and the final ratio is formed
// in float64.
//
// Float64 path (AIDW_FP64_PLAIN): w = pow(d^2, -alpha/2) in float64, plain
// float64 sums, same decomposition.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "aidw_device.cuh"
#include "aidw_internal.cuh"

namespace aidw {

namespace {

constexpr int kDTile = 1024;   // points per shared-memory stage
static_assert(kDTile == kWeightTile, "weighting tiles are staged whole");
constexpr int kStages = 3;
constexpr int kChunk = 32;     // points per plain float32 partial sum
constexpr int kWaitTries = 4000;

template <bool F64>
struct WCfg;
template <>
struct WCfg<false> {
    static constexpr int kThreads = 256;
    static constexpr int kQPT = 4;
    static constexpr int kQTile = kThreads * kQPT;
    static constexpr int kMinBlocks = 2;
};
template <>
struct WCfg<true> {
    static constexpr int kThreads = 256;
    static constexpr int kQPT = 2;
    static constexpr int kQTile = kThreads * kQPT;
    static constexpr int kMinBlocks = 1;
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
    const Point *pts;  // AoS points (float64 path)
    const float *wt;   // weighting tiles {-x[], -y[], z[]} (float32 path)
    long long n_data;
    long long n_pad;   // points incl. padding (multiple of 32)
    long long D;       // data tiles
    const float *qx, *qy;
    long long nq;
    long long T;       // query tiles
    long long U;       // units = T * D
    long long G;       // CTAs
    const QRec *recs;
    int *status;
};

__device__ __forceinline__ void issue_tile(const SKArgs &a, Point *buf, uint64_t *bar, long long u)
{
    const long long d = u % a.D;
    const long long p0 = d * kDTile;
    const long long cnt = min((long long)kDTile, a.n_pad - p0);
    mbar_expect_tx(bar, (uint32_t)(cnt * sizeof(Point)));
    bulk_g2s(buf, a.pts + p0, (uint32_t)(cnt * sizeof(Point)), bar);
}

// ---------------------------------------------------------------------------
// float32 compensated weighting
// ---------------------------------------------------------------------------
constexpr int kChunk2 = 2 * kChunk;   // points per plain sum; each lane sums kChunk

// Points of tile d that the float32 kernel processes: the valid ones rounded
// up to kChunk2 (the tile's padding has weight 0).
__device__ __forceinline__ int soa_count(const SKArgs &a, long long d)
{
    const long long rem = a.n_data - d * kDTile;
    const long long c = (rem + kChunk2 - 1) / kChunk2 * kChunk2;
    return (int)min((long long)kDTile, c);
}

__device__ __forceinline__ void issue_tile_soa(const SKArgs &a, float *buf, uint64_t *bar,
                                               long long u)
{
    const long long d = u % a.D;
    const uint32_t bytes = (uint32_t)soa_count(a, d) * 4u;
    const float *src = a.wt + d * (3 * kDTile);
    mbar_expect_tx(bar, 3u * bytes);
    bulk_g2s(buf, src, bytes, bar);
    bulk_g2s(buf + kDTile, src + kDTile, bytes, bar);
    bulk_g2s(buf + 2 * kDTile, src + 2 * kDTile, bytes, bar);
}

// Each thread holds kQPT queries; every packed instruction applies one query
// to two consecutive data points (lanes), so a 16-byte shared load of the
// tile's x (or y, z) array feeds two packed operands.
__global__ void __launch_bounds__(WCfg<false>::kThreads, WCfg<false>::kMinBlocks)
    k_weight_f32(SKArgs a, float4 *__restrict__ part)
{
    using C = WCfg<false>;
    constexpr int Q = C::kQPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *buf = reinterpret_cast<float *>(smem_raw);
    __shared__ __align__(8) uint64_t full[kStages];

    const long long j = blockIdx.x;
    const long long u0 = sk_begin(j, a.U, a.G), u1 = sk_begin(j + 1, a.U, a.G);
    if (u0 >= u1) return;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < kStages; ++s)
            if (u0 + s < u1) issue_tile_soa(a, buf + s * 3 * kDTile, &full[s], u0 + s);

    const F2 zero2 = f2_pack(0.0f, 0.0f);
    long long u = u0;
    while (u < u1) {
        const long long t = u / a.D;
        const long long seg_end = min(u1, (t + 1) * a.D);

        F2 qx2[Q], qy2[Q], c2[Q], b2[Q], hw[Q], lw[Q], hz[Q], lz[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const long long q = t * C::kQTile + (long long)i * C::kThreads + threadIdx.x;
            float qx = 0.0f, qy = 0.0f, c = -1.0f, b = 0.0f;
            if (q < a.nq) {
                qx = a.qx[q];
                qy = a.qy[q];
                const QRec r = a.recs[q];
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
            const bool ok = mbar_wait_bounded(&full[s], par, kWaitTries);
            const float *X = buf + s * 3 * kDTile;
            const float *Y = X + kDTile;
            const float *Z = Y + kDTile;
            const int cnt = soa_count(a, u % a.D);
            if (ok) {
                for (int c0 = 0; c0 < cnt; c0 += kChunk2) {
                    F2 ps[Q], pz[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) ps[i] = pz[i] = zero2;
#pragma unroll 4
                    for (int jj = c0; jj < c0 + kChunk2; jj += 4) {
                        const float4 xv = *reinterpret_cast<const float4 *>(X + jj);
                        const float4 yv = *reinterpret_cast<const float4 *>(Y + jj);
                        const float4 zv = *reinterpret_cast<const float4 *>(Z + jj);
                        const F2 xs[2] = {f2_pack(xv.x, xv.y), f2_pack(xv.z, xv.w)};
                        const F2 ys[2] = {f2_pack(yv.x, yv.y), f2_pack(yv.z, yv.w)};
                        const F2 zs[2] = {f2_pack(zv.x, zv.y), f2_pack(zv.z, zv.w)};
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
#pragma unroll
                            for (int i = 0; i < Q; ++i) {
                                const F2 dx = f2_add(qx2[i], xs[h]);
                                const F2 dy = f2_add(qy2[i], ys[h]);
                                const F2 d2 = f2_fma(dy, dy, f2_mul(dx, dx));
                                float d0, d1;
                                f2_unpack(d2, d0, d1);
                                const F2 tt = f2_fma(f2_pack(lg2_sfu(d0), lg2_sfu(d1)), c2[i], b2[i]);
                                float t0, t1;
                                f2_unpack(tt, t0, t1);
                                const F2 w = f2_pack(ex2_sfu(t0), ex2_sfu(t1));
                                ps[i] = f2_add(ps[i], w);
                                pz[i] = f2_fma(w, zs[h], pz[i]);
                            }
                        }
                    }
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        f2_comp_add(hw[i], lw[i], ps[i]);
                        f2_comp_add(hz[i], lz[i], pz[i]);
                    }
                }
            }
            // every thread is done with stage s before it is refilled
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicOr(a.status, kStatusTimeout);
                // drain the copies this CTA still has in flight, then leave
                if (threadIdx.x == 0)
                    for (long long v = u; v < min(u1, u + kStages); ++v)
                        mbar_wait_bounded(&full[(v - u0) % kStages],
                                          (uint32_t)(((v - u0) / kStages) & 1), kWaitTries);
                __syncthreads();
                return;
            }
            if (threadIdx.x == 0 && u + kStages < u1)
                issue_tile_soa(a, buf + s * 3 * kDTile, &full[s], u + kStages);
        }

        const long long slot = t + j;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float w0, w1, wl0, wl1, z0, z1, zl0, zl1;
            f2_unpack(hw[i], w0, w1);
            f2_unpack(lw[i], wl0, wl1);
            f2_unpack(hz[i], z0, z1);
            f2_unpack(lz[i], zl0, zl1);
            comp_add(w0, wl0, w1);
            comp_add(z0, zl0, z1);
            part[slot * C::kQTile + (long long)i * C::kThreads + threadIdx.x] =
                make_float4(w0, add_rn(wl0, wl1), z0, add_rn(zl0, zl1));
        }
    }
}

__global__ void k_finalize_f32(const float4 *__restrict__ part, const QRec *__restrict__ recs,
                               long long nq, long long D, long long U, long long G,
                               float *__restrict__ out_z)
{
    using C = WCfg<false>;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const QRec r = recs[q];
    if (!(r.alpha == r.alpha)) {
        out_z[q] = __int_as_float(0x7fc00000);
        return;
    }
    if (r.n_hit > 0) {
        out_z[q] = (float)r.hit_z;
        return;
    }
    const long long t = q / C::kQTile, l = q % C::kQTile;
    const long long j0 = sk_owner(t * D, U, G), j1 = sk_owner((t + 1) * D - 1, U, G);
    float hw = 0.0f, lw = 0.0f, hz = 0.0f, lz = 0.0f;
    for (long long j = j0; j <= j1; ++j) {
        const float4 v = part[(t + j) * C::kQTile + l];
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
__global__ void __launch_bounds__(WCfg<true>::kThreads, WCfg<true>::kMinBlocks)
    k_weight_f64(SKArgs a, double2 *__restrict__ part)
{
    using C = WCfg<true>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Point *buf = reinterpret_cast<Point *>(smem_raw);
    __shared__ __align__(8) uint64_t full[kStages];

    const long long j = blockIdx.x;
    const long long u0 = sk_begin(j, a.U, a.G), u1 = sk_begin(j + 1, a.U, a.G);
    if (u0 >= u1) return;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < kStages; ++s)
            if (u0 + s < u1) issue_tile(a, buf + s * kDTile, &full[s], u0 + s);

    long long u = u0;
    while (u < u1) {
        const long long t = u / a.D;
        const long long seg_end = min(u1, (t + 1) * a.D);
        float qx[C::kQPT], qy[C::kQPT];
        double e[C::kQPT], sw[C::kQPT], swz[C::kQPT];
#pragma unroll
        for (int i = 0; i < C::kQPT; ++i) {
            const long long q = t * C::kQTile + (long long)i * C::kThreads + threadIdx.x;
            qx[i] = 0.0f;
            qy[i] = 0.0f;
            e[i] = -1.0;
            if (q < a.nq) {
                qx[i] = a.qx[q];
                qy[i] = a.qy[q];
                const double al = a.recs[q].alpha;
                if (al == al) e[i] = -0.5 * al;
            }
            sw[i] = swz[i] = 0.0;
        }
        for (; u < seg_end; ++u) {
            const int s = (int)((u - u0) % kStages);
            const uint32_t par = (uint32_t)(((u - u0) / kStages) & 1);
            const bool ok = mbar_wait_bounded(&full[s], par, kWaitTries);
            const Point *tile = buf + s * kDTile;
            const int cnt = (int)min((long long)kDTile, a.n_pad - (u % a.D) * kDTile);
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
                if (threadIdx.x == 0) atomicOr(a.status, kStatusTimeout);
                if (threadIdx.x == 0)
                    for (long long v = u; v < min(u1, u + kStages); ++v)
                        mbar_wait_bounded(&full[(v - u0) % kStages],
                                          (uint32_t)(((v - u0) / kStages) & 1), kWaitTries);
                __syncthreads();
                return;
            }
            if (threadIdx.x == 0 && u + kStages < u1)
                issue_tile(a, buf + s * kDTile, &full[s], u + kStages);
        }
        const long long slot = t + j;
#pragma unroll
        for (int i = 0; i < C::kQPT; ++i)
            part[slot * C::kQTile + (long long)i * C::kThreads + threadIdx.x] =
                make_double2(sw[i], swz[i]);
    }
}

__global__ void k_finalize_f64(const double2 *__restrict__ part, const QRec *__restrict__ recs,
                               long long nq, long long D, long long U, long long G,
                               double *__restrict__ out_z)
{
    using C = WCfg<true>;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const QRec r = recs[q];
    if (!(r.alpha == r.alpha)) {
        out_z[q] = r.alpha;
        return;
    }
    if (r.n_hit > 0) {
        out_z[q] = r.hit_z;
        return;
    }
    const long long t = q / C::kQTile, l = q % C::kQTile;
    const long long j0 = sk_owner(t * D, U, G), j1 = sk_owner((t + 1) * D - 1, U, G);
    double sw = 0.0, swz = 0.0;
    for (long long j = j0; j <= j1; ++j) {
        const double2 v = part[(t + j) * C::kQTile + l];
        sw += v.x;
        swz += v.y;
    }
    out_z[q] = swz / sw;
}

// Dynamic shared memory of the weighting kernels: kStages data tiles.
template <bool F64>
constexpr size_t stage_smem()
{
    return F64 ? (size_t)kStages * kDTile * sizeof(Point) : (size_t)kStages * 3 * kDTile * sizeof(float);
}

template <bool F64>
int resident_ctas(int device)
{
    static int cached[2][64] = {};
    if (device < 0 || device >= 64) return 1;
    int &c = cached[F64 ? 1 : 0][device];
    if (c) return c;
    const size_t smem = stage_smem<F64>();
    int sms = 1, per_sm = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (F64) {
        cudaFuncSetAttribute(k_weight_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_weight_f64, WCfg<true>::kThreads,
                                                      smem);
    } else {
        cudaFuncSetAttribute(k_weight_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_weight_f32,
                                                      WCfg<false>::kThreads, smem);
    }
    c = std::max(1, sms * std::max(1, per_sm));
    return c;
}

template <bool F64>
aidw_status run(const aidw_grid *g, const float *qx, const float *qy, long long nq,
                const QRec *recs, void *out_z, cudaStream_t s)
{
    using C = WCfg<F64>;
    using Part = typename std::conditional<F64, double2, float4>::type;
    SKArgs a;
    a.pts = g->pts;
    a.wt = g->wt;
    a.n_data = g->n_data;
    a.n_pad = g->n_pad;
    a.D = F64 ? (g->n_pad + kDTile - 1) / kDTile : g->n_wtiles;
    a.qx = qx;
    a.qy = qy;
    a.nq = nq;
    a.T = (nq + C::kQTile - 1) / C::kQTile;
    a.U = a.T * a.D;
    a.G = std::min<long long>(resident_ctas<F64>(g->device), a.U);
    a.recs = recs;
    a.status = &g->dev->status;

    Part *part = nullptr;
    const size_t part_bytes = sizeof(Part) * (size_t)C::kQTile * (size_t)(a.T + a.G);
    if (cudaMallocAsync((void **)&part, part_bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return AIDW_ERR_OOM;
    }
    const size_t smem = stage_smem<F64>();
    int prof = profile_begin(s);
    if (F64)
        k_weight_f64<<<(unsigned)a.G, C::kThreads, smem, s>>>(a, reinterpret_cast<double2 *>(part));
    else
        k_weight_f32<<<(unsigned)a.G, C::kThreads, smem, s>>>(a, reinterpret_cast<float4 *>(part));
    profile_end(prof, s, AIDW_STAGE_WEIGHT, 1);
    prof = profile_begin(s);
    const unsigned fb = (unsigned)((nq + 255) / 256);
    if (F64)
        k_finalize_f64<<<fb, 256, 0, s>>>(reinterpret_cast<double2 *>(part), recs, nq, a.D, a.U,
                                          a.G, static_cast<double *>(out_z));
    else
        k_finalize_f32<<<fb, 256, 0, s>>>(reinterpret_cast<float4 *>(part), recs, nq, a.D, a.U,
                                          a.G, static_cast<float *>(out_z));
    profile_end(prof, s, AIDW_STAGE_FINALIZE, 1);
    cudaFreeAsync(part, s);
    return cuda_status(cudaGetLastError());
}

template <bool F64>
aidw_status run_scratch(const aidw_grid *g, const float *qx, const float *qy, long long nq,
                        const QRec *recs, void *out_z, void *scratch, size_t scratch_bytes,
                        cudaStream_t s)
{
    using C = WCfg<F64>;
    using Part = typename std::conditional<F64, double2, float4>::type;
    SKArgs a;
    a.pts = g->pts;
    a.wt = g->wt;
    a.n_data = g->n_data;
    a.n_pad = g->n_pad;
    a.D = F64 ? (g->n_pad + kDTile - 1) / kDTile : g->n_wtiles;
    a.qx = qx;
    a.qy = qy;
    a.nq = nq;
    a.T = (nq + C::kQTile - 1) / C::kQTile;
    a.U = a.T * a.D;
    const long long slot_bytes = (long long)sizeof(Part) * C::kQTile;
    const long long g_fit = (long long)(scratch_bytes / (size_t)slot_bytes) - a.T;
    if (g_fit < 1) return AIDW_ERR_INVALID_ARG;
    a.G = std::min<long long>(std::min<long long>(resident_ctas<F64>(g->device), a.U), g_fit);
    a.recs = recs;
    a.status = &g->dev->status;
    Part *part = static_cast<Part *>(scratch);
    const size_t smem = stage_smem<F64>();
    int prof = profile_begin(s);
    if (F64)
        k_weight_f64<<<(unsigned)a.G, C::kThreads, smem, s>>>(a, reinterpret_cast<double2 *>(part));
    else
        k_weight_f32<<<(unsigned)a.G, C::kThreads, smem, s>>>(a, reinterpret_cast<float4 *>(part));
    profile_end(prof, s, AIDW_STAGE_WEIGHT, 1);
    prof = profile_begin(s);
    const unsigned fb = (unsigned)((nq + 255) / 256);
    if (F64)
        k_finalize_f64<<<fb, 256, 0, s>>>(reinterpret_cast<double2 *>(part), recs, nq, a.D, a.U,
                                          a.G, static_cast<double *>(out_z));
    else
        k_finalize_f32<<<fb, 256, 0, s>>>(reinterpret_cast<float4 *>(part), recs, nq, a.D, a.U,
                                          a.G, static_cast<float *>(out_z));
    profile_end(prof, s, AIDW_STAGE_FINALIZE, 1);
    return cuda_status(cudaGetLastError());
}

}  // namespace

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

}  // namespace aidw
