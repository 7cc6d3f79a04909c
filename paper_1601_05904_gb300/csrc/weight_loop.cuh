// Inner loop of the float32 weighting kernel (Eq. 1 over all data points):
// one chunk of kChunk2 points of a shared-memory tile against the Q queries
// a thread holds.  Shared by k_weight_f32 (weight.cu) and by the probe that
// runs this loop alone to measure the rate its instruction mix reaches
// (probe.cu), so the two compile the same code.
#pragma once

#include "aidw_device.cuh"

namespace aidw {

// Points per plain float32 partial sum (per lane) before it is folded into
// the TwoSum-compensated total.  A plain sum of n positive terms is within
// (n - 1) * 2^-24 of its magnitude, so with 64 the error budget of a
// prediction (numerator and denominator) stays under 2 * 63 * 2^-24 = 7.5e-6
// of S_q (the normalised measure) plus the SFU approximation errors, inside
// the 1e-5 bound; measured on GB300 at n = m = 1M (weighting ms, unroll of
// the point loop): chunk 32 / unroll 4: 352.3, 64 / 4: 345.4, 64 / 8:
// 341.6, 64 / 16: 334.5, 64 / 32: 389.3, 32 / 16: 346.9, 16 / 4: 367.0.
constexpr int kChunk = 64;
constexpr int kChunk2 = 2 * kChunk;  // points of one chunk (both lanes)

// Adds the weights (ps) and weighted values (pz) of points [c0, c0 + kChunk2)
// of the tile X = -x, Y = -y, Z = z to the Q queries (qx2, qy2: the query
// in both lanes; c2 = -alpha/2 and b2 = -c * log2(d1^2) of Eq. 1's
// normalised weight exp2(c * log2(d^2) + b)).  Every thread reads four
// consecutive values of each array with one broadcast 16-byte load and
// applies them, two points per packed f32x2 instruction, to its queries.
// PE, PL: how many of the 2 x Q (point pair, query) products of one inner
// step take exp2 (PE, counted from the first product) and lg2 (PL, counted
// from the last) from FMA-pipe polynomials instead of the SFU; PE2 replaces
// PE on every second step.
template <int Q, int PE, int PL, int PE2>
__device__ __forceinline__ void weight_chunk_f32(const float *X, const float *Y, const float *Z,
                                                 int c0, const F2 (&qx2)[Q], const F2 (&qy2)[Q],
                                                 const F2 (&c2)[Q], const F2 (&b2)[Q],
                                                 F2 (&ps)[Q], F2 (&pz)[Q])
{
#pragma unroll 16
    for (int st = 0; st < kChunk2 / 4; ++st) {
        // steps alternate between PE and PE2 exp2 products on the
        // FMA pipe (the parity is a constant in each unrolled copy)
        const int pe = (st & 1) ? PE2 : PE;
        const int jj = c0 + 4 * st;
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
                F2 lg;
                if (h * Q + i >= 2 * Q - PL) {
                    lg = f2_log2_poly(d2);
                } else {
                    float d0, d1;
                    f2_unpack(d2, d0, d1);
                    lg = f2_pack(lg2_sfu(d0), lg2_sfu(d1));
                }
                const F2 tt = f2_fma(lg, c2[i], b2[i]);
                F2 w;
                if (h * Q + i < pe) {
                    w = f2_exp2_poly(tt);
                } else {
                    float t0, t1;
                    f2_unpack(tt, t0, t1);
                    w = f2_pack(ex2_sfu(t0), ex2_sfu(t1));
                }
                ps[i] = f2_add(ps[i], w);
                pz[i] = f2_fma(w, zs[h], pz[i]);
            }
        }
    }
}

}  // namespace aidw
