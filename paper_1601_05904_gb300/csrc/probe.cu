// Throughput probe of the pipes the weighting kernel runs on: SFU lg2 and
// ex2, and packed float32 FMA.  One CTA of 1024 threads per SM, each thread
// 8 independent dependency chains; the rate is lane-operations per SM per
// clock from clock64() around the loop, so it does not depend on the clock
// speed.  Used by the benchmark as the denominator of the ALU roofline.
#include "aidw_internal.cuh"

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

}  // namespace
}  // namespace aidw

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
