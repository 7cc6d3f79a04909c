// Throughput probe of the pipes the weighting kernel runs on: SFU lg2 and
// ex2, and packed float32 FMA.  One CTA of 1024 threads per SM, each thread
// 8 independent dependency chains; the rate is lane-operations per SM per
// clock from clock64() around the loop, so it does not depend on the clock
// speed.  Used by the benchmark as the denominator of the ALU roofline.
//
// A second probe runs the weighting kernel's inner loop (weight_loop.cuh)
// alone, over a shared-memory tile filled once: no bulk copies, no waits,
// no barriers, no job logic.  Its rate is what that instruction mix reaches
// on this GPU, the reference the kernel's own rate is compared with.
#include "aidw_internal.cuh"
#include "weight_loop.cuh"

namespace aidw {
namespace {

constexpr int kProbeIters = 2048;
constexpr int kProbeThreads = 1024;

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_probe(float *out, long long *cycles, float seed)
{
    float a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = seed + 1e-3f * (float)threadIdx.x + 0.1f * (float)c;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < kProbeIters; ++i) {
        if (OP == 2) {
            unsigned long long p[4];
#pragma unroll
            for (int c = 0; c < 4; ++c)
                asm volatile("mov.b64 %0, {%1, %2};" : "=l"(p[c]) : "f"(a[2 * c]), "f"(a[2 * c + 1]));
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    asm volatile("fma.rn.ftz.f32x2 %0, %0, %1, %0;" : "+l"(p[c]) : "l"(p[(c + 1) & 3]));
#pragma unroll
            for (int c = 0; c < 4; ++c)
                asm volatile("mov.b64 {%0, %1}, %2;" : "=f"(a[2 * c]), "=f"(a[2 * c + 1]) : "l"(p[c]));
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (OP == 0) asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(a[c]));
                if (OP == 1) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[c]));
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
aidw_status probe_rate(int sms, double lane_ops_per_iter, float *out, long long *cyc, double *rate)
{
    long long *h = new long long[sms];
    double best = 0.0;
    for (int rep = 0; rep < 3; ++rep) {
        k_probe<OP><<<sms, kProbeThreads>>>(out, cyc, 0.5f);
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(h, cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            delete[] h;
            return cuda_status(e);
        }
        long long mx = 1;
        for (int i = 0; i < sms; ++i) mx = h[i] > mx ? h[i] : mx;
        const double r = (double)kProbeThreads * kProbeIters * lane_ops_per_iter / (double)mx;
        best = r > best ? r : best;
    }
    delete[] h;
    *rate = best;
    return AIDW_OK;
}

constexpr int kLoopTile = 2048;  // points of the probe's tile
constexpr int kLoopQ = 4;        // queries per thread, as the kernel
constexpr int kLoopReps = 4;     // passes over the tile (~1 ms)

template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_probe_loop(float *out, long long *cycles, float c)
{
    __shared__ __align__(16) float X[kLoopTile], Y[kLoopTile], Z[kLoopTile];
    for (int i = threadIdx.x; i < kLoopTile; i += blockDim.x) {
        // points spread over [0, 1000)^2, stored negated as in the weighting
        // tiles; no query (offsets 1/8, 3/8) coincides with a point (1/4, 1/2)
        X[i] = -(float)((i * 37) % 1000) - 0.25f;
        Y[i] = -(float)((i * 91) % 1000) - 0.5f;
        Z[i] = (float)(i % 17);
    }
    const F2 zero2 = f2_pack(0.0f, 0.0f);
    F2 qx2[kLoopQ], qy2[kLoopQ], c2[kLoopQ], b2[kLoopQ], hw[kLoopQ], lw[kLoopQ], hz[kLoopQ],
        lz[kLoopQ];
#pragma unroll
    for (int i = 0; i < kLoopQ; ++i) {
        const float qx = (float)((blockIdx.x * 13 + threadIdx.x * 7 + i * 101) % 1000) + 0.125f;
        const float qy = (float)((blockIdx.x * 29 + threadIdx.x * 3 + i * 57) % 1000) + 0.375f;
        qx2[i] = f2_pack(qx, qx);
        qy2[i] = f2_pack(qy, qy);
        c2[i] = f2_pack(c, c);
        b2[i] = f2_pack(-2.0f * c, -2.0f * c);
        hw[i] = lw[i] = hz[i] = lz[i] = zero2;
    }
    __syncthreads();
    const long long t0 = clock64();
    for (int rep = 0; rep < kLoopReps; ++rep) {
        for (int c0 = 0; c0 < kLoopTile; c0 += kChunk2) {
            F2 ps[kLoopQ], pz[kLoopQ];
#pragma unroll
            for (int i = 0; i < kLoopQ; ++i) ps[i] = pz[i] = zero2;
            // the default split of the weighting kernel: 2 of 8 exp2 on the FMA pipe
            weight_chunk_f32<kLoopQ, 2, 0, 2>(X, Y, Z, c0, qx2, qy2, c2, b2, ps, pz);
#pragma unroll
            for (int i = 0; i < kLoopQ; ++i) {
                f2_comp_add(hw[i], lw[i], ps[i]);
                f2_comp_add(hz[i], lz[i], pz[i]);
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kLoopQ; ++i) {
        float a, b, d, e;
        f2_unpack(hw[i], a, b);
        f2_unpack(hz[i], d, e);
        s += a + b + d + e;
    }
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One check of the checked build's kind, with no access behind it.
__global__ void k_bounds_hook(long long index, long long n, int *result)
{
    *result = AIDW_IN(index, n, bounds::kTestHook) ? 1 : 0;
}

}  // namespace
}  // namespace aidw

extern "C" aidw_status aidw_test_bounds_check(int64_t index, int64_t n, int *in_range)
{
    using namespace aidw;
    int *d = nullptr;
    if (cudaMalloc((void **)&d, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return AIDW_ERR_OOM;
    }
    k_bounds_hook<<<1, 1>>>((long long)index, (long long)n, d);
    int r = 0;
    cudaError_t e = cudaMemcpy(&r, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_status(e);
    if (in_range) *in_range = r;
    return AIDW_OK;
}

extern "C" aidw_status aidw_probe_weight_loop(int ctas_per_sm, double *pairs_per_sm_clk)
{
    using namespace aidw;
    if (!pairs_per_sm_clk || (ctas_per_sm != 2 && ctas_per_sm != 3)) return AIDW_ERR_INVALID_ARG;
    *pairs_per_sm_clk = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return AIDW_ERR_CUDA;
    }
    void (*k)(float *, long long *, float) =
        ctas_per_sm == 2 ? k_probe_loop<2> : k_probe_loop<3>;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, 0) != cudaSuccess ||
        occ < ctas_per_sm) {
        cudaGetLastError();
        return AIDW_ERR_CUDA;  // the form does not fit this GPU at that occupancy
    }
    const int grid = sms * ctas_per_sm;  // every CTA resident at once
    float *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc((void **)&out, sizeof(float) * (size_t)grid * 256) != cudaSuccess ||
        cudaMalloc((void **)&cyc, sizeof(long long) * (size_t)grid) != cudaSuccess) {
        if (out) cudaFree(out);
        cudaGetLastError();
        return AIDW_ERR_OOM;
    }
    long long *h = new long long[grid];
    double best = 0.0;
    aidw_status st = AIDW_OK;
    for (int rep = 0; rep < 3 && st == AIDW_OK; ++rep) {
        k<<<grid, 256>>>(out, cyc, -1.0f);
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(h, cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            st = cuda_status(e);
            break;
        }
        long long mx = 1;
        for (int i = 0; i < grid; ++i) mx = h[i] > mx ? h[i] : mx;
        const double pairs = (double)ctas_per_sm * 256.0 * kLoopQ * kLoopTile * kLoopReps;
        const double r = pairs / (double)mx;
        best = r > best ? r : best;
    }
    delete[] h;
    cudaFree(out);
    cudaFree(cyc);
    *pairs_per_sm_clk = best;
    return st;
}

extern "C" aidw_status aidw_probe_pipe_rates(double *lg2_per_sm_clk, double *ex2_per_sm_clk,
                                             double *ffma2_lanes_per_sm_clk)
{
    using namespace aidw;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return AIDW_ERR_CUDA;
    }
    float *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc((void **)&out, sizeof(float) * (size_t)sms * kProbeThreads) != cudaSuccess ||
        cudaMalloc((void **)&cyc, sizeof(long long) * (size_t)sms) != cudaSuccess) {
        if (out) cudaFree(out);
        cudaGetLastError();
        return AIDW_ERR_OOM;
    }
    double r0 = 0, r1 = 0, r2 = 0;
    aidw_status st = probe_rate<0>(sms, 8.0, out, cyc, &r0);
    if (st == AIDW_OK) st = probe_rate<1>(sms, 8.0, out, cyc, &r1);
    if (st == AIDW_OK) st = probe_rate<2>(sms, 32.0, out, cyc, &r2);
    cudaFree(out);
    cudaFree(cyc);
    if (lg2_per_sm_clk) *lg2_per_sm_clk = r0;
    if (ex2_per_sm_clk) *ex2_per_sm_clk = r1;
    if (ffma2_lanes_per_sm_clk) *ffma2_lanes_per_sm_clk = r2;
    return st;
}

extern "C" aidw_status aidw_weight_mix(int *products, int *poly_exp2, int *poly_lg2,
                                       double *fma_lanes, double *instr)
{
    aidw::weight_mix(products, poly_exp2, poly_lg2, fma_lanes, instr);
    return AIDW_OK;
}
