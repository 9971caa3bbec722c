// Complex arithmetic on float2 and the twiddle table shared by the FFT kernels
// of the pseudospectral discretization (Sec. 4 of Mang & Biros: Fourier basis
// in space); the transforms themselves are in fft_reg.cuh.
//
// Twiddles w^t = exp(-2 pi i t / 1024) for t < 1024 come from a table the host
// fills once from FP64 sin/cos; a transform of length L reads entry
// t * (1024 / L).
#pragma once
#include <cuda_runtime.h>

#define REG_TW_N 1024
#define REG_LOG_TW_N 10

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by i
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }
