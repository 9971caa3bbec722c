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

// Per-pass twiddle tables.  Pass i (stride s = 8^i) of a radix-8 transform of length
// L = 2^logl multiplies output k (1..7) of butterfly group p (p < P_i = L / (8 s)) by
// w^(p k s), w = exp(-2 pi i / L).  Entry (i, k, p) sits at tw_off(logl, i) + (k - 1) P_i + p,
// so the threads of a warp (consecutive p, or one p) read consecutive entries.  The tables
// of the lengths 16 .. 1024 follow the 1024-entry table, at twp_base(logl); REG_TW_TOTAL
// entries in all.
__host__ __device__ constexpr int tw_groups(int logl, int i) { return 1 << (logl - 3 * i - 3); }
__host__ __device__ constexpr int tw_off(int logl, int i) {
    return i == 0 ? 0 : tw_off(logl, i - 1) + 7 * tw_groups(logl, i - 1);
}
// passes that apply twiddles: every radix-8 pass except a final one
__host__ __device__ constexpr int tw_passes(int logl) { return (logl % 3 == 0) ? logl / 3 - 1 : logl / 3; }
__host__ __device__ constexpr int tw_entries(int logl) { return tw_off(logl, tw_passes(logl)); }
__host__ __device__ constexpr int twp_base(int logl) {
    return logl <= 4 ? REG_TW_N : twp_base(logl - 1) + tw_entries(logl - 1);
}
#define REG_TW_TOTAL (twp_base(11))

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by i
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }
