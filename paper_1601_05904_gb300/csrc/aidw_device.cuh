// Device helpers shared by the kNN and weighting kernels.
//
// The float32 squared distance is written with explicit round-to-nearest,
// flush-to-zero PTX so that the kNN kernel and the weighting kernel compute
// bit-identical values for the same pair (the weighting stage relies on the
// nearest neighbour's d^2 being the exact minimum of the values it sees).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace aidw {

__device__ __forceinline__ float sub_rn(float a, float b)
{
    float r;
    asm("sub.rn.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float mul_rn(float a, float b)
{
    float r;
    asm("mul.rn.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float fma_rn(float a, float b, float c)
{
    float r;
    asm("fma.rn.ftz.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float add_rn(float a, float b)
{
    float r;
    asm("add.rn.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// Squared Euclidean distance in float32: fma(dy, dy, dx*dx).
__device__ __forceinline__ float dist2_f32(float qx, float qy, float px, float py)
{
    const float dx = sub_rn(qx, px);
    const float dy = sub_rn(qy, py);
    return fma_rn(dy, dy, mul_rn(dx, dx));
}

// Squared distance in float64 from float32 coordinates.  Both products are
// exact (24-bit mantissas), so the only rounding is the final add.
__device__ __forceinline__ double dist2_f64(float qx, float qy, float px, float py)
{
    const double dx = (double)qx - (double)px;
    const double dy = (double)qy - (double)py;
    return __fma_rn(dy, dy, dx * dx);
}

// SFU base-2 logarithm and exponential (PTX approx instructions).
__device__ __forceinline__ float lg2_sfu(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_sfu(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- packed float32 pairs (Blackwell f32x2 instructions) ------------------------
// Two float32 lanes in one 64-bit register pair; lane 0 is the low half.  The
// packed add/mul/fma round each lane exactly like the scalar .rn.ftz forms
// above, so a lane of dist2 computed here equals dist2_f32 bit for bit.
struct F2 {
    unsigned long long v;
};

__device__ __forceinline__ F2 f2_pack(float lo, float hi)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(F2 a, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    F2 r;
    asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b)
{
    F2 r;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b)
{
    F2 r;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c)
{
    F2 r;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
// Lane-wise compensated accumulation of x into (hi, lo) with TwoSum.
__device__ __forceinline__ void f2_comp_add(F2 &hi, F2 &lo, F2 x)
{
    const F2 s = f2_add(hi, x);
    const F2 bp = f2_sub(s, hi);
    const F2 ap = f2_sub(s, bp);
    const F2 e = f2_add(f2_sub(hi, ap), f2_sub(x, bp));
    hi = s;
    lo = f2_add(lo, e);
}

// exp2 of two float32 lanes on the FMA pipe, for moving part of the exp2
// work off the SFU.  Cody-Waite style reduction t = n + f with n = round(t)
// (adding 1.5 * 2^23 rounds t to an integer in the low mantissa bits) and
// f = t - n in [-1/2, 1/2] (exact: t and n are within a factor of two, or
// n = 0); 2^f by a degree-5 polynomial fitted to minimise the relative error
// on [-1/2, 1/2] (Lawson-iterated weighted least squares, generated by
// fit_poly.py; max relative error 7.5e-8, 1.5e-7 with the coefficients
// rounded to float32, comparable to ex2.approx); 2^n applied by adding n to
// the exponent field.  t is clamped
// below at -125 so the exponent cannot wrap; weights that small are below
// 2^-124 of the largest weight (1) and vanish in the sums.
__device__ __forceinline__ F2 f2_exp2_poly(F2 t)
{
    float t0, t1;
    f2_unpack(t, t0, t1);
    const F2 tc = f2_pack(fmaxf(t0, -125.0f), fmaxf(t1, -125.0f));
    const F2 magic = f2_pack(12582912.0f, 12582912.0f);  // 1.5 * 2^23
    const F2 r = f2_add(tc, magic);
    const F2 f = f2_sub(tc, f2_sub(r, magic));
    F2 p = f2_fma(f2_pack(1.3276444515213370e-03f, 1.3276444515213370e-03f), f,
                  f2_pack(9.6755353733897209e-03f, 9.6755353733897209e-03f));
    p = f2_fma(p, f, f2_pack(5.5507134646177292e-02f, 5.5507134646177292e-02f));
    p = f2_fma(p, f, f2_pack(2.4022120237350464e-01f, 2.4022120237350464e-01f));
    p = f2_fma(p, f, f2_pack(6.9314694404602051e-01f, 6.9314694404602051e-01f));
    p = f2_fma(p, f, f2_pack(1.0000001192092896e+00f, 1.0000001192092896e+00f));
    float r0, r1, p0, p1;
    f2_unpack(r, r0, r1);
    f2_unpack(p, p0, p1);
    const float w0 = __int_as_float(__float_as_int(p0) + (__float_as_int(r0) << 23));
    const float w1 = __int_as_float(__float_as_int(p1) + (__float_as_int(r1) << 23));
    return f2_pack(w0, w1);
}

// log2 of two positive float32 lanes on the FMA pipe, the counterpart of
// f2_exp2_poly for moving lg2 work off the SFU (which evaluates lg2 at half
// its ex2 rate).  Reduction x = 2^e * m with m in [sqrt(1/2), sqrt(2)):
// with i = bits(x) - bits(sqrt(1/2)), e = i >> 23 (arithmetic shift) and m
// has the bits (i & 0x7FFFFF) + bits(sqrt(1/2)), so both come from integer
// operations; e becomes a float by the 1.5 * 2^23 exponent-field trick.  With
// s = m - 1 in [-0.293, 0.415), log2(1 + s) = s * P(s), P of degree 7 fitted
// to minimise the absolute error (Lawson-iterated weighted least squares,
// generated by fit_poly.py; 4.8e-8 before rounding, about 1e-7 when
// evaluated in float32 on [1/2, 2], inside the 2^-22.6 bound of
// lg2.approx).  +inf maps to +inf, so padding
// points keep weight 0; x = 0 gives -127 (zero distances are never weighted:
// such queries are replaced in the finalize step).
__device__ __forceinline__ F2 f2_log2_poly(F2 x)
{
    float x0, x1;
    f2_unpack(x, x0, x1);
    const int b0 = __float_as_int(x0), b1 = __float_as_int(x1);
    const int i0 = b0 - 0x3F3504F3, i1 = b1 - 0x3F3504F3;
    const F2 m = f2_pack(__int_as_float((i0 & 0x007FFFFF) + 0x3F3504F3),
                         __int_as_float((i1 & 0x007FFFFF) + 0x3F3504F3));
    const F2 magic = f2_pack(12582912.0f, 12582912.0f);  // 1.5 * 2^23
    const F2 e = f2_sub(f2_pack(__int_as_float((i0 >> 23) + 0x4B400000),
                                __int_as_float((i1 >> 23) + 0x4B400000)),
                        magic);
    const F2 s = f2_sub(m, f2_pack(1.0f, 1.0f));
    F2 p = f2_fma(f2_pack(-1.4574408531188965e-01f, -1.4574408531188965e-01f), s,
                  f2_pack(2.3688933253288269e-01f, 2.3688933253288269e-01f));
    p = f2_fma(p, s, f2_pack(-2.5006875395774841e-01f, -2.5006875395774841e-01f));
    p = f2_fma(p, s, f2_pack(2.8670758008956909e-01f, 2.8670758008956909e-01f));
    p = f2_fma(p, s, f2_pack(-3.6008724570274353e-01f, -3.6008724570274353e-01f));
    p = f2_fma(p, s, f2_pack(4.8093944787979126e-01f, 4.8093944787979126e-01f));
    p = f2_fma(p, s, f2_pack(-7.2135716676712036e-01f, -7.2135716676712036e-01f));
    p = f2_fma(p, s, f2_pack(1.4426947832107544e+00f, 1.4426947832107544e+00f));
    float l0, l1;
    f2_unpack(f2_fma(s, p, e), l0, l1);
    const float inf = __int_as_float(0x7f800000);
    return f2_pack(b0 >= 0x7F800000 ? inf : l0, b1 >= 0x7F800000 ? inf : l1);
}

// Error-free transformation (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = add_rn(a, b);
    const float bp = sub_rn(s, a);
    const float ap = sub_rn(s, bp);
    e = add_rn(sub_rn(a, ap), sub_rn(b, bp));
}

// Adds x into the compensated pair (hi, lo).
__device__ __forceinline__ void comp_add(float &hi, float &lo, float x)
{
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo = add_rn(lo, e);
}

// ---- Eq. 4-6 on the device (float64) -----------------------------------------

// Eq. 4 with R = 0 for r_obs = 0 and R = +inf for r_exp = 0 < r_obs.
__device__ __forceinline__ double nn_statistic(double r_obs, double r_exp)
{
    if (r_obs == 0.0) return 0.0;
    if (r_exp == 0.0) return __longlong_as_double(0x7ff0000000000000LL);
    return r_obs / r_exp;
}

// Eq. 5 (cosine membership with the printed pi / R_max factor).
__device__ __forceinline__ double membership(double R, double r_min, double r_max)
{
    if (R <= r_min) return 0.0;
    if (R >= r_max) return 1.0;
    return 0.5 - 0.5 * cos((3.141592653589793 / r_max) * (R - r_min));
}

// Eq. 6 (triangular membership: linear between the knots 0.1 .. 0.9).
__device__ __forceinline__ double decay_power(double mu, double a1, double a2, double a3,
                                              double a4, double a5)
{
    if (mu <= 0.1) return a1;
    if (mu <= 0.3) return a1 * (1.0 - 5.0 * (mu - 0.1)) + 5.0 * a2 * (mu - 0.1);
    if (mu <= 0.5) return 5.0 * a3 * (mu - 0.3) + a2 * (1.0 - 5.0 * (mu - 0.3));
    if (mu <= 0.7) return a3 * (1.0 - 5.0 * (mu - 0.5)) + 5.0 * a4 * (mu - 0.5);
    if (mu <= 0.9) return 5.0 * a5 * (mu - 0.7) + a4 * (1.0 - 5.0 * (mu - 0.7));
    return a5;
}

// ---- mbarrier + bulk copy (TMA engine, 1-D) ------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy completing on an mbarrier.  dst, src 16-byte
// aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}

// Bounded wait: at most max_tries tries, each of which may suspend the
// thread for up to the 1 ms hint while the phase is incomplete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int max_tries)
{
    for (int i = 0; i < max_tries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace aidw
