// Shared-memory FFT building blocks for the pseudospectral discretization
// (Sec. 4 of Mang & Biros: Fourier basis in space).
//
// Transforms are unnormalized Stockham auto-sort FFTs (decimation in
// frequency, radix 4 with a final radix-2 pass when log2(L) is odd) over
// `nfft` contiguous sequences of length L that live in shared memory.  The
// caller's whole CTA cooperates; the function ends with __syncthreads() and
// returns the buffer that holds the result.
//
// Twiddles w^t = exp(-2 pi i t / 1024) for t < 1024 come from a table the host
// fills once from FP64 sin/cos; length L reads entry t * (1024 / L).
//
// Real transforms use the "two real sequences in one complex FFT" identity:
// z = a + i b has Z[k] = A[k] + i B[k], so A[k] = (Z[k] + conj Z[L-k]) / 2 and
// B[k] = (Z[k] - conj Z[L-k]) / (2i).  A real row's half spectrum is stored
// "packed": entry 0 holds A[0] (real) in .x and A[L/2] (real) in .y, entries
// 1..L/2-1 hold A[k].  Packed spectra are stored transposed, [L/2][n1].
#pragma once
#include <cuda_runtime.h>

#define REG_TW_N 1024
#define REG_LOG_TW_N 10

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by i
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }

// Radix-4/2 Stockham FFT of nfft sequences of length L = 2^LOGL stored at
// x[f*L + i].  y is scratch of the same size.  INV selects the conjugate
// transform (no 1/L factor).
template <int LOGL, bool INV>
__device__ __forceinline__ float2* smem_fft(float2* x, float2* y, int nfft, const float2* __restrict__ tw) {
    constexpr int L = 1 << LOGL;
    constexpr int L4 = L >> 2;
    constexpr int TWSHIFT = REG_LOG_TW_N - LOGL;
    int ls = 0;  // log2 of stride s
#pragma unroll 1
    for (int logn = LOGL; logn >= 2; logn -= 2) {
        const int s = 1 << ls;
        const int m = 1 << (logn - 2);
        const int items = nfft * L4;
        for (int t = threadIdx.x; t < items; t += blockDim.x) {
            const int f = t >> (LOGL - 2);
            const int r = t & (L4 - 1);
            const int p = r >> ls;
            const int q = r & (s - 1);
            const float2* xf = x + f * L;
            float2* yf = y + f * L;
            const float2 a0 = xf[q + s * p];
            const float2 a1 = xf[q + s * (p + m)];
            const float2 a2 = xf[q + s * (p + 2 * m)];
            const float2 a3 = xf[q + s * (p + 3 * m)];
            const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
            const float2 t2 = cadd(a1, a3), t3 = csub(a1, a3);
            // forward: -i * t3 ; inverse: +i * t3
            const float2 jt3 = INV ? make_float2(-t3.y, t3.x) : make_float2(t3.y, -t3.x);
            const float2 b0 = cadd(t0, t2), b2 = csub(t0, t2);
            const float2 b1 = cadd(t1, jt3), b3 = csub(t1, jt3);
            const int e = (p << ls) << TWSHIFT;  // p*s in units of 1/L, scaled to the table
            float2 w1 = __ldg(&tw[e]);
            float2 w2 = __ldg(&tw[2 * e]);
            float2 w3 = __ldg(&tw[3 * e]);
            if (INV) { w1 = cconj(w1); w2 = cconj(w2); w3 = cconj(w3); }
            const int o = q + s * 4 * p;
            yf[o] = b0;
            yf[o + s] = cmul(b1, w1);
            yf[o + 2 * s] = cmul(b2, w2);
            yf[o + 3 * s] = cmul(b3, w3);
        }
        __syncthreads();
        float2* tmp = x; x = y; y = tmp;
        ls += 2;
    }
    if (LOGL & 1) {
        constexpr int L2 = L >> 1;
        const int items = nfft * L2;
        for (int t = threadIdx.x; t < items; t += blockDim.x) {
            const int f = t >> (LOGL - 1);
            const int q = t & (L2 - 1);
            const float2 a = x[f * L + q];
            const float2 b = x[f * L + q + L2];
            y[f * L + q] = cadd(a, b);
            y[f * L + q + L2] = csub(a, b);
        }
        __syncthreads();
        float2* tmp = x; x = y; y = tmp;
    }
    return x;
}

// Split the spectrum Z of z = a + i b (length L) at wavenumber k in [1, L/2)
// into A[k], B[k].
__device__ __forceinline__ void split_pair(float2 Zk, float2 Zm, float2& A, float2& B) {
    A = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
    B = make_float2(0.5f * (Zk.y + Zm.y), -0.5f * (Zk.x - Zm.x));
}

// Merge packed half spectra entries A[k], B[k] (k in [1, L/2)) into Z[k] and Z[L-k].
__device__ __forceinline__ void merge_pair(float2 A, float2 B, float2& Zk, float2& Zm) {
    Zk = make_float2(A.x - B.y, A.y + B.x);
    Zm = make_float2(A.x + B.y, -A.y + B.x);
}
