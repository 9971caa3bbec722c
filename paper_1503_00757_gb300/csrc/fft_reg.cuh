// Register-resident radix-8 FFTs for the pseudospectral operators (Sec. 4 of
// Mang & Biros: Fourier basis in space).
//
// A length-L transform (L = 2^LOGL, 16 <= L <= 1024) is computed by T = L/8
// threads that each hold 8 complex values.  On entry thread t holds
// x[k] = in[t + k T]; on exit x[k] = out[t + k T] (k = 0..7).  The algorithm
// is a Stockham auto-sort FFT (decimation in frequency): floor(LOGL/3)
// radix-8 passes computed in registers, then one radix-2 or radix-4 pass if
// LOGL is not a multiple of 3.  Passes exchange data through two shared-memory
// buffers of L complex values (one __syncthreads per exchange).  Unnormalized
// in both directions (the 1/(n1 n2) factor is applied with the Fourier
// multiplier).
//
// Twiddles come from per-pass tables (fft.cuh) filled once by the host from FP64
// sin/cos, laid out so that a warp reads consecutive entries.  The exchange
// buffers are padded (fft_pad) so that a pass's stores are free of bank
// conflicts.
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"

// Packed half spectra are stored in row-quad tiles: the entry of row i and
// wavenumber e (0 <= e < W = n2/2) lives at ((i / 4) * W + e) * 4 + i % 4, so
// the spectra of 4 consecutive rows form one contiguous block and a column of
// the spectrum is read in 32-byte pieces per 4 rows.
__device__ __forceinline__ size_t sp_idx(int i, int e, int W) { return ((size_t)(i >> 2) * W + e) * 4 + (i & 3); }

template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {  // forward: -i a ; inverse: +i a
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// In-register DFT of length 8 (radix-2 split into even / odd DFT-4).
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&x)[8]) {
    const float r = 0.70710678118654752440f;
    const float2 b0 = cadd(x[0], x[4]), b1 = csub(x[0], x[4]);
    const float2 b2 = cadd(x[2], x[6]), b3 = mul_mi<INV>(csub(x[2], x[6]));
    const float2 b4 = cadd(x[1], x[5]), b5 = csub(x[1], x[5]);
    const float2 b6 = cadd(x[3], x[7]), b7 = mul_mi<INV>(csub(x[3], x[7]));
    const float2 E0 = cadd(b0, b2), E2 = csub(b0, b2), E1 = cadd(b1, b3), E3 = csub(b1, b3);
    const float2 O0 = cadd(b4, b6), O2 = csub(b4, b6), O1 = cadd(b5, b7), O3 = csub(b5, b7);
    // w1 = exp(-/+ i pi/4), w3 = exp(-/+ 3 i pi/4)
    const float2 w1 = INV ? make_float2(r, r) : make_float2(r, -r);
    const float2 w3 = INV ? make_float2(-r, r) : make_float2(-r, -r);
    const float2 t1 = cmul(w1, O1), t2 = mul_mi<INV>(O2), t3 = cmul(w3, O3);
    x[0] = cadd(E0, O0); x[4] = csub(E0, O0);
    x[1] = cadd(E1, t1); x[5] = csub(E1, t1);
    x[2] = cadd(E2, t2); x[6] = csub(E2, t2);
    x[3] = cadd(E3, t3); x[7] = csub(E3, t3);
}

// twiddle w^(p k s) of pass i (see fft.cuh), from the per-pass table of length 2^LOGL
template <int LOGL, bool INV>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int i, int k, int p) {
    float2 w = __ldg(&tw[twp_base(LOGL) + tw_off(LOGL, i) + (k - 1) * tw_groups(LOGL, i) + p]);
    if (INV) w.y = -w.y;
    return w;
}

// Exchange-buffer index with one padding slot every 8 entries: a radix-8 pass stores 8
// consecutive entries per thread (stride 8 between threads), which without the padding puts
// 16 threads of a warp on the same shared-memory banks.  A buffer holds fft_buf(L) entries.
__host__ __device__ constexpr int fft_buf(int L) { return L + L / 8; }
__device__ __forceinline__ int fft_pad(int i) { return i + (i >> 3); }

// All threads of the CTA must call this together (it contains __syncthreads).
// bA, bB: this FFT's two exchange buffers of fft_buf(L) float2 each.  Threads with
// active == false take part in the barriers only.
template <int LOGL, bool INV>
__device__ __forceinline__ void reg_fft(float2 (&x)[8], int t, bool active, float2* bA, float2* bB,
                                        const float2* __restrict__ tw) {
    constexpr int L = 1 << LOGL;
    constexpr int T = L >> 3;
    constexpr int NP8 = LOGL / 3;
    constexpr int REM = LOGL - 3 * NP8;
    float2* cur = bA;
    float2* nxt = bB;
#pragma unroll
    for (int i = 0; i < NP8; ++i) {
        const int ls = 3 * i;
        const int s = 1 << ls;
        const int q = t & (s - 1);
        const int p = t >> ls;
        const int m = L >> (ls + 3);
        const bool last = (i == NP8 - 1) && (REM == 0);
        if (active) {
            if (i > 0) {
#pragma unroll
                for (int k = 0; k < 8; ++k) x[k] = cur[fft_pad(q + s * (p + k * m))];
            }
            dft8<INV>(x);
            if (!last) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float2 y = (k == 0) ? x[k] : cmul(x[k], twiddle<LOGL, INV>(tw, i, k, p));
                    nxt[fft_pad(q + s * (8 * p + k))] = y;
                }
            }
        }
        if (!last) {
            __syncthreads();
            float2* tmp = cur; cur = nxt; nxt = tmp;
        }
    }
    if (REM == 1) {
        // radix 2, stride s = L/2 = 4T: butterflies q = t + jT (j < 4)
        if (active) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 a = cur[fft_pad(t + j * T)], b = cur[fft_pad(t + j * T + 4 * T)];
                x[j] = cadd(a, b);
                x[j + 4] = csub(a, b);
            }
        }
    } else if (REM == 2) {
        // radix 4, stride s = L/4 = 2T: butterflies q = t + jT (j < 2)
        if (active) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int q = t + j * T;
                const float2 a0 = cur[fft_pad(q)], a1 = cur[fft_pad(q + 2 * T)], a2 = cur[fft_pad(q + 4 * T)],
                             a3 = cur[fft_pad(q + 6 * T)];
                const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
                x[j] = cadd(t0, t2);
                x[j + 2] = cadd(t1, t3);
                x[j + 4] = csub(t0, t2);
                x[j + 6] = csub(t1, t3);
            }
        }
    }
}

// Z[e] of z = a + i b, where a and b are real rows whose packed half spectra
// are rows ra of Sa and rb of Sb of a tiled chunk (W = L/2 wavenumbers).
template <int LOGL>
__device__ __forceinline__ float2 merged_entry(const float2* Sa, int ra, const float2* Sb, int rb, int e) {
    constexpr int L = 1 << LOGL, H = L >> 1;
    if (e == 0) {
        const float2 A = Sa[sp_idx(ra, 0, H)], B = Sb[sp_idx(rb, 0, H)];
        return make_float2(A.x, B.x);
    }
    if (e == H) {
        const float2 A = Sa[sp_idx(ra, 0, H)], B = Sb[sp_idx(rb, 0, H)];
        return make_float2(A.y, B.y);
    }
    const int ee = (e < H) ? e : L - e;
    const float2 A = Sa[sp_idx(ra, ee, H)], B = Sb[sp_idx(rb, ee, H)];
    return (e < H) ? make_float2(A.x - B.y, A.y + B.x) : make_float2(A.x + B.y, -A.y + B.x);
}

// As merged_entry, with the imaginary-part row given implicitly as the x^2
// derivative of another row: B[e] = i e c S[e] (c = 1/n2), which is zero at
// e = 0 and at the Nyquist entry (odd symbol).
template <int LOGL>
__device__ __forceinline__ float2 merged_entry_d2(const float2* Sa, int ra, const float2* Sd, int rd, int e, float c) {
    constexpr int L = 1 << LOGL, H = L >> 1;
    if (e == 0) return make_float2(Sa[sp_idx(ra, 0, H)].x, 0.f);
    if (e == H) return make_float2(Sa[sp_idx(ra, 0, H)].y, 0.f);
    const int ee = (e < H) ? e : L - e;
    const float2 A = Sa[sp_idx(ra, ee, H)], S = Sd[sp_idx(rd, ee, H)];
    const float ce = c * (float)ee;
    const float2 B = make_float2(-ce * S.y, ce * S.x);
    return (e < H) ? make_float2(A.x - B.y, A.y + B.x) : make_float2(A.x + B.y, -A.y + B.x);
}

// Packed half-spectrum entry e of the real part (part 0) or imaginary part
// (part 1) of z, given the full spectrum Z (natural order, L entries).
template <int LOGL>
__device__ __forceinline__ float2 split_entry(const float2* Z, int part, int e) {
    constexpr int L = 1 << LOGL, H = L >> 1;
    if (e == 0) {
        const float2 z0 = Z[0], zh = Z[H];
        return part == 0 ? make_float2(z0.x, zh.x) : make_float2(z0.y, zh.y);
    }
    const float2 zk = Z[e], zm = Z[L - e];
    return part == 0 ? make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y))
                     : make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
}
