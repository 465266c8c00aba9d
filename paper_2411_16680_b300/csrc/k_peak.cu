// Measured FP32 SIMT peak of the device (quark_measure_fp32_peak): the denominator of the FP32
// roofline fractions the benchmark reports (the conv block and attention of the FP32 form, the
// SIMT share of the sampling kernel), measured instead of derived from unit counts and clocks.
//
// Every thread runs 16 independent dependency chains of fused multiply-adds on registers, as
// scalar FMAs or as packed FP32x2 FMAs (the sm_100-family instruction the kernels use), long
// enough for the launch to take tens of milliseconds; FLOPs = 2 per lane-FMA.
#include <cuda_runtime.h>

#include <algorithm>

#include "api_internal.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_peak_kernel(int iters, float a, float b, float* out) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) ffma2_peak_kernel(int iters, float a, float b, float* out) {
    float2 x[kChains / 2];
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) x[i] = make_float2(threadIdx.x * 1e-3f + i, threadIdx.x * 1e-3f - i);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int i = 0; i < kChains / 2; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) s += x[i].x + x[i].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" quark_status quark_measure_fp32_peak(int device, double* fma_tflops, double* ffma2_tflops) {
    if (!fma_tflops || !ffma2_tflops) return qk_fail(nullptr, QUARK_EINVAL, "NULL argument");
    cudaError_t e = cudaSetDevice(device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return qk_fail(nullptr, QUARK_ECUDA, "device %d: %s", device, cudaGetErrorString(e));
    const int blocks = sms * 8;  // eight CTAs of 256 threads per SM: every FMA lane busy
    float* out = nullptr;
    e = cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(float));
    if (e != cudaSuccess) return qk_fail(nullptr, QUARK_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = 4096;
    // near-1 multiplier and a small addend keep the chains finite and the results data-dependent
    const float a = 0.9999f, b = 1e-4f;
    double best[2] = {0.0, 0.0};
    for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run warms the clocks
            cudaEventRecord(e0);
            if (kind == 0) fma_peak_kernel<<<blocks, kThreads>>>(iters, a, b, out);
            else ffma2_peak_kernel<<<blocks, kThreads>>>(iters, a, b, out);
            cudaEventRecord(e1);
            e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double flops = 2.0 * kChains * 8.0 * iters * (double)blocks * kThreads;
            if (ms > 0.f && rep > 0) best[kind] = std::max(best[kind], flops / (ms * 1e-3) * 1e-12);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return qk_fail(nullptr, QUARK_ECUDA, "FP32 peak kernels: %s", cudaGetErrorString(e));
    *fma_tflops = best[0];
    *ffma2_tflops = best[1];
    return QUARK_OK;
}
