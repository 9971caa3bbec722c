// Three-dimensional registration operators on the GPU: the reduced gradient and the
// Gauss-Newton Hessian matvec of the H1-regularized problem on an n1 x n2 x n3 periodic
// box (the paper's equations of Sec. 3 for d = 3: state Eq. (e:state-eq-elim), adjoint
// Eq. (e:adj-eq-elim), incremental state and adjoint Eqs. (e:inc-state-eq-elim),
// (e:inc-adj-eq-elim), body forces and the projection K of Eq. (e:project-body-force)),
// with the same discretization as the 2-D path: Heun's RK2 in pseudo-time, trapezoidal
// time quadrature, pseudospectral derivatives with odd symbols k~ (Nyquist entry zero)
// and the full even symbol |k|^2.
//
// Layout: real fields are n1 x n2 x n3 floats, index (i1 n2 + i2) n3 + i3; vector fields
// three such fields back to back.  Spectra are full complex (float2) fields in the same
// order.  A 3-D transform is three passes of batched 1-D radix-2 Stockham FFTs
// (k3_fft_pass), one per axis: a CTA stages a tile of 32 lines in shared memory (loads
// coalesced along the contiguous direction), runs the log2(L) butterfly stages between
// two shared buffers (row stride padded by one element against bank conflicts; twiddles
// from a per-CTA table built once from exact fractions) and writes the tile back in
// natural order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "internal.h"

namespace {

constexpr int R3_THREADS = 256;
constexpr int R3_TILE = 32;  // lines per CTA in an FFT pass

// line l of a pass starts at (l / Q) P + (l % Q) R; elements are S apart
struct LineMap {
    int L, S, Q, P, R, TWL;
};

// one pass of length-L transforms (forward exp(-2 pi i jk / L), or inverse exp(+...),
// unnormalized) over TWL consecutive lines per CTA
template <bool INV>
__global__ void __launch_bounds__(R3_THREADS) k3_fft_pass(float2* __restrict__ data, LineMap m) {
    extern __shared__ float2 sbuf[];
    const int TWL = m.TWL, L = m.L, SP = m.TWL + 1;  // padded stride: line elements fall in distinct banks
    float2* b0 = sbuf;
    float2* b1 = sbuf + L * SP;
    float2* tw = sbuf + 2 * L * SP;  // tw[k] = exp(-2 pi i k / L), k < L / 2
    const int tile = blockIdx.x;
    auto base = [&](int w) {
        const long long l = (long long)tile * TWL + w;
        return (l / m.Q) * (long long)m.P + (l % m.Q) * (long long)m.R;
    };
    for (int k = threadIdx.x; k < L / 2; k += blockDim.x) {
        float sn, cs;
        sincospif(2.f * (float)k / (float)L, &sn, &cs);
        tw[k] = make_float2(cs, -sn);
    }
    // stage the tile: b0[p SP + w] = element p of line w (the contiguous direction fastest)
    for (int e = threadIdx.x; e < L * TWL; e += blockDim.x) {
        int p, w;
        if (m.S == 1) { p = e % L; w = e / L; } else { w = e % TWL; p = e / TWL; }
        b0[p * SP + w] = data[base(w) + (long long)p * m.S];
    }
    __syncthreads();
    float2* src = b0;
    float2* dst = b1;
    for (int Ns = 1; Ns < L; Ns <<= 1) {
        const int step = L / (2 * Ns);  // exp(-i pi k / Ns) = tw[k step]
        for (int e = threadIdx.x; e < (L / 2) * TWL; e += blockDim.x) {
            const int w = e % TWL, j = e / TWL;
            const int k = j & (Ns - 1);
            const float2 a = src[j * SP + w];
            const float2 c = src[(j + L / 2) * SP + w];
            const float2 t0 = tw[k * step];
            const float ws = INV ? -t0.y : t0.y;
            const float2 t = make_float2(c.x * t0.x - c.y * ws, c.x * ws + c.y * t0.x);
            const int d = (j / Ns) * 2 * Ns + k;
            dst[d * SP + w] = make_float2(a.x + t.x, a.y + t.y);
            dst[(d + Ns) * SP + w] = make_float2(a.x - t.x, a.y - t.y);
        }
        __syncthreads();
        float2* tmp = src;
        src = dst;
        dst = tmp;
    }
    for (int e = threadIdx.x; e < L * TWL; e += blockDim.x) {
        int p, w;
        if (m.S == 1) { p = e % L; w = e / L; } else { w = e % TWL; p = e / TWL; }
        data[base(w) + (long long)p * m.S] = src[p * SP + w];
    }
}

struct Dims3 {
    int n1, n2, n3;
    long long N;
};

// odd (Nyquist zero) and even (Nyquist n/2) wavenumbers of index i on an axis of length n
__device__ __forceinline__ float k_odd(int i, int n) { return i < n / 2 ? (float)i : (i == n / 2 ? 0.f : (float)(i - n)); }
__device__ __forceinline__ float k_even(int i, int n) { return i < n / 2 ? (float)i : (float)(i - n); }

__device__ __forceinline__ void wave3(const Dims3& D, long long idx, float& k1, float& k2, float& k3, float& kk) {
    const int i3 = (int)(idx % D.n3);
    const long long r = idx / D.n3;
    const int i2 = (int)(r % D.n2), i1 = (int)(r / D.n2);
    k1 = k_odd(i1, D.n1);
    k2 = k_odd(i2, D.n2);
    k3 = k_odd(i3, D.n3);
    const float e1 = k_even(i1, D.n1), e2 = k_even(i2, D.n2), e3 = k_even(i3, D.n3);
    kk = e1 * e1 + e2 * e2 + e3 * e3;
}

#define GRID_STRIDE(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// F = (f, 0) for nf fields of N points
__global__ void k3_real2c(const float* __restrict__ f, float2* __restrict__ F, long long n) {
    GRID_STRIDE(i, n) F[i] = make_float2(f[i], 0.f);
}

// G_d = i k~_d F (three spectra)
__global__ void k3_grad_spec(const float2* __restrict__ F, float2* __restrict__ G, Dims3 D) {
    GRID_STRIDE(i, D.N) {
        float k1, k2, k3, kk;
        wave3(D, i, k1, k2, k3, kk);
        const float2 f = F[i];
        G[i] = make_float2(-k1 * f.y, k1 * f.x);
        G[D.N + i] = make_float2(-k2 * f.y, k2 * f.x);
        G[2 * D.N + i] = make_float2(-k3 * f.y, k3 * f.x);
    }
}

// F = sum_d i k~_d U_d
__global__ void k3_div_spec(const float2* __restrict__ U, float2* __restrict__ F, Dims3 D) {
    GRID_STRIDE(i, D.N) {
        float k1, k2, k3, kk;
        wave3(D, i, k1, k2, k3, kk);
        const float2 a = U[i], b = U[D.N + i], c = U[2 * D.N + i];
        const float re = k1 * a.x + k2 * b.x + k3 * c.x, im = k1 * a.y + k2 * b.y + k3 * c.y;
        F[i] = make_float2(-im, re);
    }
}

// out = beta |k|^2 V + K^ B (three spectra); mode 0: K = I, 1: incompressible, 2: mass source
// (K^ = I - k~ k~^T / (|k~|^2 + beta |k|^2 / (beta_w (1 + |k|^2))))
__global__ void k3_assemble(const float2* __restrict__ V, const float2* Bs, float2* out,  // out may be Bs
                            Dims3 D, float beta, int mode, float beta_w) {
    GRID_STRIDE(i, D.N) {
        float k1, k2, k3, kk;
        wave3(D, i, k1, k2, k3, kk);
        float2 b[3] = {Bs[i], Bs[D.N + i], Bs[2 * D.N + i]};
        if (mode != 0) {
            const float ko = k1 * k1 + k2 * k2 + k3 * k3;
            if (ko > 0.f) {
                const float denom = mode == 1 ? ko : ko + beta * kk / (beta_w * (1.f + kk));
                const float cre = (k1 * b[0].x + k2 * b[1].x + k3 * b[2].x) / denom;
                const float cim = (k1 * b[0].y + k2 * b[1].y + k3 * b[2].y) / denom;
                const float kd[3] = {k1, k2, k3};
#pragma unroll
                for (int d = 0; d < 3; ++d) b[d] = make_float2(b[d].x - kd[d] * cre, b[d].y - kd[d] * cim);
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float2 v = V[d * D.N + i];
            out[d * D.N + i] = make_float2(beta * kk * v.x + b[d].x, beta * kk * v.y + b[d].y);
        }
    }
}

// f = Re(F) / N
__global__ void k3_c2real(const float2* __restrict__ F, float* __restrict__ f, long long n, float invN) {
    GRID_STRIDE(i, n) f[i] = F[i].x * invN;
}

// advection stage of the state (src == nullptr) or incremental state equation:
//   k = -grad y . v - src . vt  (grad y = Re(G) / N);  gm_out (optional) = grad y
//   stage 1: kbuf = k, y_out = y + h k;  stage 2: y_out = y + h / 2 (kbuf + k)
__global__ void k3_adv_stage(const float2* __restrict__ G, const float* __restrict__ v, const float* __restrict__ src,
                             const float* __restrict__ vt, const float* y, float* __restrict__ kbuf,
                             float* y_out, float* __restrict__ gm_out, long long N, float invN, float h,  // y_out may be y
                             int stage) {
    GRID_STRIDE(i, N) {
        const float g0 = G[i].x * invN, g1 = G[N + i].x * invN, g2 = G[2 * N + i].x * invN;
        if (gm_out) {
            gm_out[i] = g0;
            gm_out[N + i] = g1;
            gm_out[2 * N + i] = g2;
        }
        float k = -(g0 * v[i] + g1 * v[N + i] + g2 * v[2 * N + i]);
        if (src) k -= src[i] * vt[i] + src[N + i] * vt[N + i] + src[2 * N + i] * vt[2 * N + i];
        if (stage == 1) {
            kbuf[i] = k;
            y_out[i] = y[i] + h * k;
        } else {
            y_out[i] = y[i] + 0.5f * h * (kbuf[i] + k);
        }
    }
}

// U_d = (lam v_d, 0): the flux of the adjoint transport, ready for the forward transforms
__global__ void k3_flux(const float* __restrict__ lam, const float* __restrict__ v, float2* __restrict__ U, long long N) {
    GRID_STRIDE(i, N) {
        const float l = lam[i];
        U[i] = make_float2(l * v[i], 0.f);
        U[N + i] = make_float2(l * v[N + i], 0.f);
        U[2 * N + i] = make_float2(l * v[2 * N + i], 0.f);
    }
}

// adjoint stage, k = div(lam v) = Re(F) / N (time reversed: d_tau lam = div(lam v))
__global__ void k3_adj_stage(const float2* __restrict__ F, const float* y, float* __restrict__ kbuf,
                             float* y_out, long long N, float invN, float h, int stage) {  // y_out may be y
    GRID_STRIDE(i, N) {
        const float k = F[i].x * invN;
        if (stage == 1) {
            kbuf[i] = k;
            y_out[i] = y[i] + h * k;
        } else {
            y_out[i] = y[i] + 0.5f * h * (kbuf[i] + k);
        }
    }
}

// b (+)= w lam grad m (trapezoid weight w; first = 1 overwrites)
__global__ void k3_body_force(const float* __restrict__ lam, const float* __restrict__ gm, float* __restrict__ b,
                              long long N, float w, int first) {
    GRID_STRIDE(i, N) {
        const float l = w * lam[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) b[d * N + i] = (first ? 0.f : b[d * N + i]) + l * gm[d * N + i];
    }
}

// y = a x (scale), used for lam(1) = m_R - m(1) and lam~(1) = -m~(1)
__global__ void k3_axpy(const float* __restrict__ x, const float* __restrict__ z, float* __restrict__ y, long long N,
                        float a, float c) {
    GRID_STRIDE(i, N) y[i] = a * x[i] + (z ? c * z[i] : 0.f);
}

// per-block FP64 partial sums of the objective terms, reduced in a fixed order by k3_reduce:
// data: sum (mR - m1)^2; reg: sum_k |k|^2 |V_d|^2; w: sum_k (1 + |k|^2) |i k~ . V|^2
__global__ void __launch_bounds__(R3_THREADS) k3_energy_part(const float* __restrict__ mR, const float* __restrict__ m1,
                                                             const float2* __restrict__ V, Dims3 D, double* part) {
    __shared__ double s[3][R3_THREADS];
    double a = 0.0, r = 0.0, wv = 0.0;
    GRID_STRIDE(i, D.N) {
        const double d = (double)mR[i] - (double)m1[i];
        a += d * d;
        float k1, k2, k3, kk;
        wave3(D, i, k1, k2, k3, kk);
        double e = 0.0;
        float2 vv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            vv[c] = V[c * D.N + i];
            e += (double)vv[c].x * vv[c].x + (double)vv[c].y * vv[c].y;
        }
        r += (double)kk * e;
        const double wre = (double)k1 * vv[0].x + (double)k2 * vv[1].x + (double)k3 * vv[2].x;
        const double wim = (double)k1 * vv[0].y + (double)k2 * vv[1].y + (double)k3 * vv[2].y;
        wv += (1.0 + kk) * (wre * wre + wim * wim);
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = r;
    s[2][threadIdx.x] = wv;
    __syncthreads();
    for (int o = R3_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 3; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[blockIdx.x * 3 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k3_reduce(const double* __restrict__ part, int nblk, double* out) {
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int b = 0; b < nblk; ++b) t += part[b * 3 + threadIdx.x];
        out[threadIdx.x] = t;
    }
}

// per-block FP64 partial sums of sum_i a_i b_i (fixed-order reduction by k3_reduce)
__global__ void __launch_bounds__(R3_THREADS) k3_dot_part(const float* __restrict__ a, const float* __restrict__ b,
                                                          long long n, double* part) {
    __shared__ double sh[R3_THREADS];
    double t = 0.0;
    GRID_STRIDE(i, n) t += (double)a[i] * (double)b[i];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int o = R3_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x * 3] = sh[0];
        part[blockIdx.x * 3 + 1] = 0.0;
        part[blockIdx.x * 3 + 2] = 0.0;
    }
}

// y = a x + b y
__global__ void k3_axpby(const float* x, float* y, long long n, float a, float b) {  // x may be y
    GRID_STRIDE(i, n) y[i] = a * x[i] + b * y[i];
}

// (beta A)^-1 on three spectra, the k = 0 symbol of A replaced by 1 (App. E)
__global__ void k3_precond_spec(float2* X, Dims3 D, float beta) {
    GRID_STRIDE(i, D.N) {
        float k1, k2, k3, kk;
        wave3(D, i, k1, k2, k3, kk);
        const float s = 1.f / (beta * (kk > 0.f ? kk : 1.f));
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float2 x = X[d * D.N + i];
            X[d * D.N + i] = make_float2(x.x * s, x.y * s);
        }
    }
}

}  // namespace

struct reg3_ctx {
    Dims3 D;
    int nt;
    double beta, gamma;
    int kmode;  // 0: K = I (gamma = 0), 1: incompressible (gamma = inf), 2: mass source
    cudaStream_t stream;
    float *mT, *mR, *v, *gm, *y, *ys, *kb, *lam, *g3, *bt, *mt;
    float2 *F, *G;  // one spectrum, three spectra
    double *d_part, *d_sum, *h_sum;
    bool have_images, have_lin;
};

namespace {

constexpr int R3_BLOCKS = 608;  // 4 per SM of a GB300 for the grid-stride kernels

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

LineMap line_map(const Dims3& D, int axis) {
    LineMap m;
    if (axis == 2) {
        m.L = D.n3; m.S = 1; m.Q = D.n1 * D.n2; m.P = 0; m.R = D.n3; m.TWL = R3_TILE;
    } else if (axis == 1) {
        m.L = D.n2; m.S = D.n3; m.Q = D.n3; m.P = D.n2 * D.n3; m.R = 1; m.TWL = D.n3 < R3_TILE ? D.n3 : R3_TILE;
    } else {
        m.L = D.n1; m.S = D.n2 * D.n3; m.Q = D.n2 * D.n3; m.P = 0; m.R = 1; m.TWL = R3_TILE;
    }
    return m;
}

size_t pass_smem(const LineMap& m) { return ((size_t)2 * m.L * (m.TWL + 1) + m.L / 2) * sizeof(float2); }

// in-place 3-D transform of `count` consecutive spectra
void fft3(reg3_ctx* c, float2* X, int count, bool inverse) {
    for (int f = 0; f < count; ++f)
        for (int axis = 2; axis >= 0; --axis) {
            const LineMap m = line_map(c->D, axis);
            const int tiles = (int)(c->D.N / m.L / m.TWL);
            if (inverse)
                k3_fft_pass<true><<<tiles, R3_THREADS, pass_smem(m), c->stream>>>(X + f * c->D.N, m);
            else
                k3_fft_pass<false><<<tiles, R3_THREADS, pass_smem(m), c->stream>>>(X + f * c->D.N, m);
        }
}

// G = the three spectra of grad f (still to be inverse-transformed and scaled by 1 / N)
void grad_spectra(reg3_ctx* c, const float* f) {
    k3_real2c<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(f, c->F, c->D.N);
    fft3(c, c->F, 1, false);
    k3_grad_spec<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->F, c->G, c->D);
    fft3(c, c->G, 3, true);
}

// state (src == nullptr, from y0 into c->y, gradient history into c->gm) or incremental
// state (source grad m_j . vt from the stored history, from 0, into c->mt)
void forward_solve(reg3_ctx* c, const float* y0, const float* vt) {
    const long long N = c->D.N;
    const float h = 1.f / c->nt, invN = 1.f / (float)N;
    float* y = vt ? c->mt : c->y;
    if (y0) cudaMemcpyAsync(y, y0, sizeof(float) * N, cudaMemcpyDeviceToDevice, c->stream);
    else cudaMemsetAsync(y, 0, sizeof(float) * N, c->stream);
    for (int j = 0; j < c->nt; ++j) {
        grad_spectra(c, y);
        k3_adv_stage<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->G, c->v, vt ? c->gm + 3 * N * j : nullptr, vt, y,
                                                              c->kb, c->ys, vt ? nullptr : c->gm + 3 * N * j, N,
                                                              invN, h, 1);
        grad_spectra(c, c->ys);
        k3_adv_stage<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->G, c->v, vt ? c->gm + 3 * N * (j + 1) : nullptr, vt,
                                                              y, c->kb, y, nullptr, N, invN, h, 2);
    }
    if (!vt) {  // grad m(t = 1) completes the history
        grad_spectra(c, y);
        k3_adv_stage<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->G, c->v, nullptr, nullptr, y, c->kb, c->ys,
                                                              c->gm + 3 * N * c->nt, N, invN, h, 1);
    }
}

// adjoint transport backward from c->lam = lam(1), accumulating out = int lam grad m dt
void adjoint_solve(reg3_ctx* c, float* out) {
    const long long N = c->D.N;
    const int nt = c->nt;
    const float h = 1.f / nt, invN = 1.f / (float)N;
    for (int j = nt; j >= 1; --j) {
        k3_body_force<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->lam, c->gm + 3 * N * j, out, N,
                                                               j == nt ? 0.5f * h : h, j == nt);
        k3_flux<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->lam, c->v, c->G, N);
        fft3(c, c->G, 3, false);
        k3_div_spec<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->G, c->F, c->D);
        fft3(c, c->F, 1, true);
        k3_adj_stage<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->F, c->lam, c->kb, c->ys, N, invN, h, 1);
        k3_flux<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->ys, c->v, c->G, N);
        fft3(c, c->G, 3, false);
        k3_div_spec<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->G, c->F, c->D);
        fft3(c, c->F, 1, true);
        k3_adj_stage<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->F, c->lam, c->kb, c->lam, N, invN, h, 2);
    }
    k3_body_force<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->lam, c->gm, out, N, 0.5f * h, 0);
}

// out = beta A x + K b (x, b vector fields); leaves the spectra of x in c->G
void assemble(reg3_ctx* c, const float* x, const float* b, float* out) {
    const long long N = c->D.N;
    // spectra of b in c->G, of x in the scratch g3 (3 complex fields)
    k3_real2c<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(b, c->G, 3 * N);
    fft3(c, c->G, 3, false);
    float2* X = reinterpret_cast<float2*>(c->g3);  // 3 complex fields of scratch (6N floats)
    k3_real2c<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(x, X, 3 * N);
    fft3(c, X, 3, false);
    k3_assemble<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(X, c->G, c->G, c->D, (float)c->beta, c->kmode,
                                                         (float)c->gamma);
    fft3(c, c->G, 3, true);
    k3_c2real<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->G, out, 3 * N, 1.f / (float)N);
    k3_energy_part<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->mR, c->y, X, c->D, c->d_part);
    k3_reduce<<<1, 32, 0, c->stream>>>(c->d_part, R3_BLOCKS, c->d_sum);
}

int r3_err(const char* what) {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? REG_OK : reg_fail(REG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" void reg3_destroy(reg3_ctx* c) {
    if (!c) return;
    void* ptrs[] = {c->mT, c->mR, c->v, c->gm, c->y, c->ys, c->kb, c->lam, c->g3, c->bt, c->mt, c->F, c->G,
                    c->d_part, c->d_sum};
    for (void* p : ptrs) cudaFree(p);
    cudaFreeHost(c->h_sum);
    delete c;
}

extern "C" int reg3_create(int n1, int n2, int n3, int nt, double beta, double gamma, reg3_ctx** out) {
    if (!out) return reg_fail(REG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!pow2_in(n1, 8, 256) || !pow2_in(n2, 8, 256) || !pow2_in(n3, 8, 256))
        return reg_fail(REG_ERR_ARG, "n1, n2, n3 must be powers of two in [8, 256]");
    if (nt < 1 || nt > 1024) return reg_fail(REG_ERR_ARG, "nt must be in [1, 1024]");
    if (!(beta > 0.0) || !std::isfinite(beta)) return reg_fail(REG_ERR_ARG, "beta must be positive and finite");
    if (!(gamma >= 0.0)) return reg_fail(REG_ERR_ARG, "gamma must be >= 0 (INFINITY: incompressible)");
    reg3_ctx* c = new reg3_ctx();
    c->D = Dims3{n1, n2, n3, (long long)n1 * n2 * n3};
    c->nt = nt;
    c->beta = beta;
    c->gamma = gamma;
    c->kmode = gamma == 0.0 ? 0 : (std::isinf(gamma) ? 1 : 2);
    c->stream = 0;
    const size_t N = (size_t)c->D.N;
    bool ok = true;
    auto M = [&](void** p, size_t bytes) { if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false; };
    M((void**)&c->mT, sizeof(float) * N);
    M((void**)&c->mR, sizeof(float) * N);
    M((void**)&c->v, sizeof(float) * 3 * N);
    M((void**)&c->gm, sizeof(float) * 3 * N * (nt + 1));
    M((void**)&c->y, sizeof(float) * N);
    M((void**)&c->ys, sizeof(float) * N);
    M((void**)&c->kb, sizeof(float) * N);
    M((void**)&c->lam, sizeof(float) * N);
    M((void**)&c->g3, sizeof(float) * 6 * N);
    M((void**)&c->bt, sizeof(float) * 3 * N);
    M((void**)&c->mt, sizeof(float) * N);
    M((void**)&c->F, sizeof(float2) * N);
    M((void**)&c->G, sizeof(float2) * 3 * N);
    M((void**)&c->d_part, sizeof(double) * 3 * R3_BLOCKS);
    M((void**)&c->d_sum, sizeof(double) * 3);
    if (ok && cudaMallocHost((void**)&c->h_sum, sizeof(double) * 3) != cudaSuccess) ok = false;
    if (!ok) {
        cudaGetLastError();
        reg3_destroy(c);
        return reg_fail(REG_ERR_NOMEM, "3-D context allocation failed");
    }
    // the opt-in is a per-kernel, per-device attribute shared by every context: always the
    // largest tile any legal grid needs (256-point lines, 32 per CTA), so that a smaller context
    // created later never lowers it under a larger one
    LineMap mmax;
    mmax.L = 256;
    mmax.TWL = R3_TILE;
    const size_t smax = pass_smem(mmax);
    cudaFuncSetAttribute(k3_fft_pass<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    cudaFuncSetAttribute(k3_fft_pass<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    const int st = r3_err("3-D context set-up");
    if (st != REG_OK) {
        reg3_destroy(c);
        return st;
    }
    *out = c;
    return REG_OK;
}

extern "C" int reg3_set_stream(reg3_ctx* c, void* stream) {
    if (!c) return reg_fail(REG_ERR_ARG, "ctx is NULL");
    c->stream = (cudaStream_t)stream;
    return REG_OK;
}

extern "C" int reg3_set_images(reg3_ctx* c, const float* mT, const float* mR) {
    if (!c || !mT || !mR) return reg_fail(REG_ERR_ARG, "NULL argument");
    cudaMemcpyAsync(c->mT, mT, sizeof(float) * c->D.N, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->mR, mR, sizeof(float) * c->D.N, cudaMemcpyDeviceToDevice, c->stream);
    c->have_images = true;
    c->have_lin = false;
    return r3_err("reg3_set_images");
}

extern "C" int reg3_gradient(reg3_ctx* c, const float* v, float* g, double* J) {
    if (!c || !v || !g) return reg_fail(REG_ERR_ARG, "NULL argument");
    if (!c->have_images) return reg_fail(REG_ERR_STATE, "reg3_set_images first");
    const long long N = c->D.N;
    cudaMemcpyAsync(c->v, v, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, c->stream);
    forward_solve(c, c->mT, nullptr);                                                         // m, grad m history
    k3_axpy<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->mR, c->y, c->lam, N, 1.f, -1.f);     // lam(1) = mR - m(1)
    adjoint_solve(c, c->bt);                                                                   // b
    assemble(c, c->v, c->bt, g);                                                               // beta A v + K b, J parts
    cudaMemcpyAsync(c->h_sum, c->d_sum, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream);
    int st = r3_err("reg3_gradient");
    if (st != REG_OK) return st;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return r3_err("reg3_gradient");
    const double hv = std::pow(2.0 * M_PI, 3) / (double)N;
    double Jv = 0.5 * hv * c->h_sum[0] + 0.5 * c->beta * hv / (double)N * c->h_sum[1];
    if (c->kmode == 2) Jv += 0.5 * c->gamma * hv / (double)N * c->h_sum[2];
    if (J) *J = Jv;
    if (!std::isfinite(Jv)) return reg_fail(REG_ERR_NAN, "objective is not finite");
    c->have_lin = true;
    return REG_OK;
}

extern "C" int reg3_hessian_matvec(reg3_ctx* c, const float* vt, float* Hvt) {
    if (!c || !vt || !Hvt) return reg_fail(REG_ERR_ARG, "NULL argument");
    if (!c->have_lin) return reg_fail(REG_ERR_STATE, "reg3_gradient first (it fixes the linearization point)");
    const long long N = c->D.N;
    float* vtc = c->g3;  // the direction, kept while the solves run (the assembly reuses g3 after)
    cudaMemcpyAsync(vtc, vt, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, c->stream);
    forward_solve(c, nullptr, vtc);                                                           // m~ history end
    k3_axpy<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->mt, nullptr, c->lam, N, -1.f, 0.f);  // lam~(1) = -m~(1)
    adjoint_solve(c, c->bt);                                                                   // b~
    // the assembly transforms x into g3 in place: give it vt from the caller's buffer
    assemble(c, vt, c->bt, Hvt);
    return r3_err("reg3_hessian_matvec");
}

namespace {

// <a, b> on the grid (trapezoidal weight (2 pi)^3 / N) over 3 N values; synchronous
double inner3(reg3_ctx* c, const float* a, const float* b) {
    k3_dot_part<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(a, b, 3 * c->D.N, c->d_part);
    k3_reduce<<<1, 32, 0, c->stream>>>(c->d_part, R3_BLOCKS, c->d_sum);
    cudaMemcpyAsync(c->h_sum, c->d_sum, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    return std::pow(2.0 * M_PI, 3) / (double)c->D.N * c->h_sum[0];
}

void precond3(reg3_ctx* c, const float* r, float* out) {
    const long long N = c->D.N;
    k3_real2c<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(r, c->G, 3 * N);
    fft3(c, c->G, 3, false);
    k3_precond_spec<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->G, c->D, (float)c->beta);
    fft3(c, c->G, 3, true);
    k3_c2real<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->G, out, 3 * N, 1.f / (float)N);
}

// J at x (one state solve; the gradient history is overwritten, which Algorithm 1 allows:
// the next gradient evaluation rebuilds it at the accepted point)
double objective3(reg3_ctx* c, const float* x) {
    const long long N = c->D.N;
    cudaMemcpyAsync(c->v, x, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, c->stream);
    forward_solve(c, c->mT, nullptr);
    float2* X = reinterpret_cast<float2*>(c->g3);
    k3_real2c<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(x, X, 3 * N);
    fft3(c, X, 3, false);
    k3_energy_part<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(c->mR, c->y, X, c->D, c->d_part);
    k3_reduce<<<1, 32, 0, c->stream>>>(c->d_part, R3_BLOCKS, c->d_sum);
    cudaMemcpyAsync(c->h_sum, c->d_sum, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    const double hv = std::pow(2.0 * M_PI, 3) / (double)N;
    double J = 0.5 * hv * c->h_sum[0] + 0.5 * c->beta * hv / (double)N * c->h_sum[1];
    if (c->kmode == 2) J += 0.5 * c->gamma * hv / (double)N * c->h_sum[2];
    c->have_lin = false;
    return J;
}

}  // namespace

extern "C" int reg3_solve(reg3_ctx* c, float* v, double tol, int maxit_newton, int maxit_pcg, double* stats) {
    if (!c || !v) return reg_fail(REG_ERR_ARG, "NULL argument");
    if (!c->have_images) return reg_fail(REG_ERR_STATE, "reg3_set_images first");
    if (!(tol > 0.0) || maxit_newton < 0 || maxit_pcg < 1) return reg_fail(REG_ERR_ARG, "tol > 0, maxit_pcg >= 1");
    const long long N3 = 3 * c->D.N;
    float *g, *vt, *r, *z, *sd, *Hs, *vtrial;
    float** bufs[] = {&g, &vt, &r, &z, &sd, &Hs, &vtrial};
    for (float** b : bufs) *b = nullptr;
    for (float** b : bufs)
        if (cudaMalloc((void**)b, sizeof(float) * N3) != cudaSuccess) {
            cudaGetLastError();
            for (float** q : bufs) cudaFree(*q);
            return reg_fail(REG_ERR_NOMEM, "reg3_solve work vectors");
        }
    int k = 0, nmv = 0, nls = 0, status = REG_OK;
    double J = 0.0, J0 = 0.0, g0 = 0.0, gn = 0.0;
    auto done = [&](int st) {
        if (stats) {
            stats[0] = k;
            stats[1] = nmv;
            stats[2] = nls;
            stats[3] = g0 > 0.0 ? gn / g0 : 0.0;
            stats[4] = J;
            stats[5] = st;
            stats[6] = J0;
        }
        for (float** q : bufs) cudaFree(*q);
        return st;
    };
    const double c1 = 1e-4, rho = 0.5;
    const int max_ls = 20;
    // Algorithm 1 from v = 0: the stopping test is relative to ||g(0)||
    cudaMemsetAsync(v, 0, sizeof(float) * N3, c->stream);
    int st = reg3_gradient(c, v, g, &J);
    if (st != REG_OK) return done(st);
    J0 = J;
    g0 = gn = std::sqrt(inner3(c, g, g));
    while (g0 > 0.0 && gn / g0 > tol) {
        if (k >= maxit_newton) { status = REG_ERR_MAXIT; break; }
        // Algorithm 2: preconditioned CG on H v~ = -g to ||r|| < eta ||g||
        const double eta = std::fmin(0.5, std::sqrt(gn / g0));
        cudaMemsetAsync(vt, 0, sizeof(float) * N3, c->stream);
        cudaMemsetAsync(r, 0, sizeof(float) * N3, c->stream);
        k3_axpby<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(g, r, N3, -1.f, 0.f);  // r = -g
        precond3(c, r, z);
        cudaMemcpyAsync(sd, z, sizeof(float) * N3, cudaMemcpyDeviceToDevice, c->stream);
        double rz = inner3(c, r, z);
        for (int it = 1; it <= maxit_pcg; ++it) {
            st = reg3_hessian_matvec(c, sd, Hs);
            if (st != REG_OK) return done(st);
            ++nmv;
            const double sHs = inner3(c, sd, Hs);
            if (!(sHs > 0.0)) {
                if (it == 1) cudaMemcpyAsync(vt, sd, sizeof(float) * N3, cudaMemcpyDeviceToDevice, c->stream);
                break;
            }
            const float kappa = (float)(rz / sHs);
            k3_axpby<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(sd, vt, N3, kappa, 1.f);
            k3_axpby<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(Hs, r, N3, -kappa, 1.f);
            if (std::sqrt(inner3(c, r, r)) < eta * gn) break;
            precond3(c, r, z);
            const double rz_new = inner3(c, z, r);
            k3_axpby<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(z, sd, N3, 1.f, (float)(rz_new / rz));
            rz = rz_new;
        }
        double gv = inner3(c, g, vt);
        if (gv >= 0.0) {  // not a descent direction: the preconditioned steepest descent step
            precond3(c, g, vt);
            k3_axpby<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(vt, vt, N3, 0.f, -1.f);
            gv = inner3(c, g, vt);
        }
        // Armijo backtracking on J
        double alpha = 1.0;
        bool accepted = false;
        for (int l = 0; l < max_ls; ++l) {
            cudaMemcpyAsync(vtrial, v, sizeof(float) * N3, cudaMemcpyDeviceToDevice, c->stream);
            k3_axpby<<<R3_BLOCKS, R3_THREADS, 0, c->stream>>>(vt, vtrial, N3, (float)alpha, 1.f);
            ++nls;
            // a trial beyond the explicit scheme's stability gives a non-finite J: rejected like any
            // other trial that fails the sufficient-decrease test
            const double Jt = objective3(c, vtrial);
            if (std::isfinite(Jt) && Jt <= J + c1 * alpha * gv) {
                accepted = true;
                break;
            }
            alpha *= rho;
        }
        if (!accepted) { status = REG_ERR_LINESEARCH; break; }
        cudaMemcpyAsync(v, vtrial, sizeof(float) * N3, cudaMemcpyDeviceToDevice, c->stream);
        ++k;
        st = reg3_gradient(c, v, g, &J);
        if (st != REG_OK) return done(st);
        gn = std::sqrt(inner3(c, g, g));
    }
    const int e = r3_err("reg3_solve");
    if (e != REG_OK) return done(e);
    if (status == REG_ERR_LINESEARCH) return done(reg_fail(status, "line search failed"));
    if (status == REG_ERR_MAXIT) return done(reg_fail(status, "Newton iteration cap reached before the tolerance"));
    return done(REG_OK);
}
