// FP32 FMA throughput of the current GPU, measured (reg_fp32_peak in
// include/reg.h).
//
// The transport solves run their FFT butterflies and RK2 updates on the FP32
// CUDA cores, so the arithmetic ceiling of a Hessian matvec is the FP32 FMA
// rate.  This measures that rate on the device instead of deriving it from the
// SM count and a nominal clock: one wave of 256-thread CTAs (SM count x CTAs
// resident per SM), every thread running independent FMA recurrences on
// registers, timed with CUDA events on a stream of its own.
#include <string>

#include "internal.h"

namespace {
constexpr int kChains = 16;   // independent recurrences per thread (covers the FMA latency)
constexpr int kThreads = 256;
constexpr int kIters = 2048;  // recurrence steps per chain and launch
constexpr int kWarmup = 2, kWindows = 3, kPerWindow = 5;

// x <- a x + b with b = 1 - a and 0 < a < 1 keeps every x in (0, 1] (fixed
// point 1), so the sum of the chains stays below 2 kChains and the store below
// never runs; a and b arrive at run time, so the compiler keeps every FMA.
__global__ void __launch_bounds__(kThreads) k_fma_rate(float a, float b, float* sink) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (float)(i + 1) + 1e-7f * (float)threadIdx.x;
#pragma unroll 4
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s > 2.0f * kChains) sink[0] = s;
}
}  // namespace

extern "C" int reg_fp32_peak(double* tflops, double* ms_per_launch) {
    if (!tflops) return reg_fail(REG_ERR_ARG, "tflops is NULL");
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate, kThreads, 0);
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
    if (sms < 1 || per_sm < 1) return reg_fail(REG_ERR_CUDA, "no resident CTA of the FMA kernel fits an SM");
    const int grid = sms * per_sm;

    float* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return reg_fail(REG_ERR_NOMEM, "fp32 peak: 4-byte sink");
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    const float a = 0.999f, b = 1.0f - a;
    for (int i = 0; ok && i < kWarmup; ++i) {
        k_fma_rate<<<grid, kThreads, 0, st>>>(a, b, sink);
        ok = cudaGetLastError() == cudaSuccess;
    }
    double best = -1.0;
    for (int w = 0; ok && w < kWindows; ++w) {
        ok = cudaEventRecord(e0, st) == cudaSuccess;
        for (int i = 0; ok && i < kPerWindow; ++i) {
            k_fma_rate<<<grid, kThreads, 0, st>>>(a, b, sink);
            ok = cudaGetLastError() == cudaSuccess;
        }
        float t = 0.f;
        ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
        const double ms = t / (double)kPerWindow;
        if (ok && (best < 0.0 || ms < best)) best = ms;
    }
    std::string err = ok ? std::string() : std::string(cudaGetErrorString(cudaGetLastError()));
    if (st) cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    if (!ok || best <= 0.0) return reg_fail(REG_ERR_CUDA, "fp32 peak: " + err);
    const double flops = 2.0 * kChains * (double)kIters * kThreads * (double)grid;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms_per_launch) *ms_per_launch = best;
    return REG_OK;
}
