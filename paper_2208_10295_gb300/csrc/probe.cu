// Measured FP32 arithmetic rate of the device: the denominator of the cast
// kernel's ALU fraction (the traversal's slab and triangle tests are FP32
// adds, multiplies, fused multiply-adds and min/max).  Every SM runs eight
// resident warps per scheduler, each thread eight independent chains of fused
// multiply-adds, with no memory traffic between the first and last
// instruction; scalar (FFMA) and packed-pair (f32x2) forms are both timed and
// the faster is the rate.
#include "common.cuh"

namespace lidar {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_fma_scalar(float a, float b, int64_t rounds, float* sink)
{
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int64_t r = 0; r < rounds; ++r) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == -1.0f) sink[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) k_fma_pairs(float a, float b, int64_t rounds, float* sink)
{
    unsigned long long x[kProbeChains / 2], a2, b2;
    asm("mov.b64 %0, {%1, %1};" : "=l"(a2) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(b2) : "f"(b));
#pragma unroll
    for (int c = 0; c < kProbeChains / 2; ++c) {
        const float lo = (float)(threadIdx.x + 2 * c) * 1e-3f, hi = (float)(threadIdx.x + 2 * c + 1) * 1e-3f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
    // each packed instruction is two FMAs: half as many instructions for the
    // same FMA count as the scalar kernel
    for (int64_t r = 0; r < rounds; ++r) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < kProbeChains / 2; ++c)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(a2), "l"(b2));
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kProbeChains / 2; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == -1.0f) sink[blockIdx.x] = s;
}

}  // namespace

cudaError_t measure_fp32_rate(cudaStream_t s, int num_sms, int64_t fma_per_thread, void* sink_dev,
                              double* flops_per_s, double* ms, int* form)
{
    const int grid = num_sms * kProbeBlocksPerSm;
    // FMAs per thread per round: 8 unrolled steps x the chains
    const int64_t rounds = (fma_per_thread + 8 * kProbeChains - 1) / (8 * kProbeChains);
    const double fmas = (double)grid * kProbeThreads * rounds * 8 * kProbeChains;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    double best = 0.0, best_ms = 0.0;
    int best_form = 0;
    for (int f = 0; f < 2 && e == cudaSuccess; ++f) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first run of each form warms up
            cudaEventRecord(e0, s);
            if (f == 0)
                k_fma_scalar<<<grid, kProbeThreads, 0, s>>>(0.9999999f, 1e-7f, rounds, (float*)sink_dev);
            else
                k_fma_pairs<<<grid, kProbeThreads, 0, s>>>(0.9999999f, 1e-7f, rounds, (float*)sink_dev);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
            cudaEventRecord(e1, s);
            e = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && rep == 1 && t > 0.0f) {
                const double rate = 2.0 * fmas / (t * 1e-3);
                if (rate > best) {
                    best = rate;
                    best_ms = t;
                    best_form = f;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *flops_per_s = best;
    *ms = best_ms;
    *form = best_form;
    return e;
}

}  // namespace lidar
