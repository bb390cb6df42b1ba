// Measured arithmetic peaks of the GPU the library runs on: the denominators of the blend
// kernels' roofline (the blend is bound by FP32 instruction issue and the special-function
// unit, not by HBM).
//
// Each kernel keeps 8 independent dependency chains per thread, so that the pipe, not the
// latency of one chain, limits it, and runs a fixed number of rounds over a grid of
// SMs x 8 CTAs of 256 threads (2048 threads per SM, the most an SM holds). The instructions
// are written as inline PTX so that the count per round is exact; each result is stored
// (only when it equals an impossible value, so the store never happens but the work cannot
// be removed).
#include <cuda_runtime.h>

#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 8;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(float *sink, int rounds, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int r = 0; r < rounds; r++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == -1.2345f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed pairs: one fma.rn.f32x2 is two FP32 FMAs.
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma2(float *sink, int rounds, float a, float b) {
    unsigned long long x[kChains], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        const float v = (float)(threadIdx.x + c) * 1e-3f;
        asm("mov.b64 %0, {%1, %1};" : "=l"(x[c]) : "f"(v));
    }
    for (int r = 0; r < rounds; r++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == -1.2345f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Special-function unit: x <- 2^(-x) converges to a fixed point near 0.64 (no overflow); the
// negation runs on another pipe beside the SFU.
__global__ void __launch_bounds__(kPeakThreads) k_peak_ex2(float *sink, int rounds) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int r = 0; r < rounds; r++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
            float y;
            asm volatile("neg.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(y));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == -1.2345f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// x <- 1 / (x + 1) converges to 0.618...; the add runs on the FMA pipe beside the SFU.
__global__ void __launch_bounds__(kPeakThreads) k_peak_rcp(float *sink, int rounds) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int r = 0; r < rounds; r++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
            float y;
            asm volatile("add.rn.f32 %0, %1, 0f3F800000;" : "=f"(y) : "f"(x[c]));
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(y));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == -1.2345f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace tgs

using namespace tgs;

extern "C" tgs_status tgs_measure_peaks(tgs_peaks *out, tgs_stream stream) {
    if (!out) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return TGS_ERR_CUDA;
    }
    const int blocks = sms * kPeakBlocksPerSM;
    const double threads = (double)blocks * kPeakThreads;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tgs_status s = TGS_OK;
    if (cudaMalloc(&sink, sizeof(float) * (size_t)blocks * kPeakThreads) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        s = TGS_ERR_CUDA;
    }
    // rounds sized for a few milliseconds per kernel at the GB300's nominal rates
    const int r_fma = 65536, r_sfu = 8192;
    double ms[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4 && s == TGS_OK; k++) {
        for (int rep = 0; rep < 2 && s == TGS_OK; rep++) {  // the first launch is a warm-up
            cudaEventRecord(e0, st);
            switch (k) {
                case 0: k_peak_fma<<<blocks, kPeakThreads, 0, st>>>(sink, r_fma, 0.9999f, 1e-4f); break;
                case 1: k_peak_fma2<<<blocks, kPeakThreads, 0, st>>>(sink, r_fma, 0.9999f, 1e-4f); break;
                case 2: k_peak_ex2<<<blocks, kPeakThreads, 0, st>>>(sink, r_sfu); break;
                default: k_peak_rcp<<<blocks, kPeakThreads, 0, st>>>(sink, r_sfu); break;
            }
            cudaEventRecord(e1, st);
            float t = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
                cudaGetLastError() != cudaSuccess)
                s = TGS_ERR_CUDA;
            ms[k] = t;
        }
    }
    if (s == TGS_OK) {
        out->fp32_fma_per_s = threads * r_fma * kChains / (ms[0] * 1e-3);
        out->fp32x2_fma_per_s = 2.0 * threads * r_fma * kChains / (ms[1] * 1e-3);
        out->ex2_per_s = threads * r_sfu * kChains / (ms[2] * 1e-3);
        out->rcp_per_s = threads * r_sfu * kChains / (ms[3] * 1e-3);
        out->sms = sms;
        out->ms = ms[0] + ms[1] + ms[2] + ms[3];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return s;
}
