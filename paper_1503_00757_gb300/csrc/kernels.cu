// CUDA kernels (sm_103a) for the pseudospectral Gauss-Newton-Krylov
// registration solver of Mang & Biros (arXiv 1503.00757).
//
// A 2-D transform of an n1 x n2 real field is split into two passes over HBM:
//   * row kernels: one CTA owns R consecutive rows; real FFTs along x^2
//     (two real rows, or two real fields of one row, per complex FFT), fused
//     with the pointwise work of an RK2 stage (Sec. 5) on the physical side;
//   * column kernels: one CTA owns CPB columns of the packed half spectrum
//     (stored transposed, so a column is contiguous); forward FFT along x^1,
//     a Fourier multiplier (gradient, divergence, A, K, preconditioner,
//     Eq. (e:var-reg-v), (e:project-body-force), Appendix E), inverse FFT.
// Pointwise and reduction kernels serve the PCG (Algorithm 2) and the
// deformation gradient (Eq. (e:def-grad)); FP64 accumulation for all sums.
#include <cmath>
#include <cstdio>
#include <unordered_map>
#include <vector>

#include "fft.cuh"
#include "internal.h"

#define NTHREADS 256
#define NBLK_RED 304  // 2 x 152 SMs

// ---------------------------------------------------------------------------
// timing hooks
// ---------------------------------------------------------------------------
void ktimer_begin(reg_ctx* ctx, int kclass, double bytes) {
    ctx->launches++;
    if (!ctx->timing) return;
    EventPair ep;
    size_t need = ctx->events.size() * 2 + 2;
    while (ctx->event_pool.size() < need) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ctx->event_pool.push_back(e);
    }
    ep.a = ctx->event_pool[need - 2];
    ep.b = ctx->event_pool[need - 1];
    ep.kclass = kclass;
    ep.bytes = bytes;
    cudaEventRecord(ep.a, ctx->stream);
    ctx->events.push_back(ep);
}

void ktimer_end(reg_ctx* ctx) {
    if (!ctx->timing) return;
    cudaEventRecord(ctx->events.back().b, ctx->stream);
}

cudaError_t k_init_twiddles(reg_ctx* ctx) {
    std::vector<float2> h(REG_TW_N);
    for (int t = 0; t < REG_TW_N; ++t) {
        double a = -2.0 * M_PI * (double)t / (double)REG_TW_N;
        h[t] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    return cudaMemcpy(ctx->tw, h.data(), sizeof(float2) * REG_TW_N, cudaMemcpyHostToDevice);
}

// ---------------------------------------------------------------------------
// helpers: block reductions (FP64)
// ---------------------------------------------------------------------------
template <int OPR>
__device__ __forceinline__ double red_op(double a, double b) {
    if (OPR == 0) return a + b;
    if (OPR == 1) return fmax(a, b);
    return fmin(a, b);
}

template <int OPR>
__device__ double block_reduce(double v) {
    __shared__ double red_sm[32];
    for (int o = 16; o > 0; o >>= 1) v = red_op<OPR>(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red_sm[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        v = (l < nw) ? red_sm[l] : (OPR == 0 ? 0.0 : red_sm[0]);
        for (int o = 16; o > 0; o >>= 1) v = red_op<OPR>(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// packed-spectrum row helpers (transposed layout [L/2][n1])
// ---------------------------------------------------------------------------
// Build full complex spectra of nseq sequences.  pairs_of_rows: sequence sq
// merges rows row0+2sq (real part) and row0+2sq+1 (imag part) of SA;
// otherwise it merges row row0+sq of SA (real part) and of SB (imag part).
template <int LOGL>
__device__ __forceinline__ void load_merge(float2* buf, int nseq, const float2* __restrict__ SA,
                                           const float2* __restrict__ SB, int n1, int row0, bool pairs_of_rows) {
    constexpr int L = 1 << LOGL, H = L >> 1;
    for (int t = threadIdx.x; t < nseq * H; t += blockDim.x) {
        const int sq = t % nseq, k = t / nseq;
        int ra, rb;
        const float2* pb;
        if (pairs_of_rows) { ra = row0 + 2 * sq; rb = ra + 1; pb = SA; }
        else { ra = rb = row0 + sq; pb = SB; }
        const float2 A = SA[(size_t)k * n1 + ra];
        const float2 B = pb[(size_t)k * n1 + rb];
        float2* z = buf + sq * L;
        if (k == 0) {
            z[0] = make_float2(A.x, B.x);
            z[H] = make_float2(A.y, B.y);
        } else {
            float2 zk, zm;
            merge_pair(A, B, zk, zm);
            z[k] = zk;
            z[L - k] = zm;
        }
    }
}

template <int LOGL>
__device__ __forceinline__ void split_store(const float2* buf, int nseq, float2* __restrict__ SA,
                                            float2* __restrict__ SB, int n1, int row0, bool pairs_of_rows) {
    constexpr int L = 1 << LOGL, H = L >> 1;
    for (int t = threadIdx.x; t < nseq * H; t += blockDim.x) {
        const int sq = t % nseq, k = t / nseq;
        const float2* z = buf + sq * L;
        float2 A, B;
        if (k == 0) {
            const float2 z0 = z[0], zh = z[H];
            A = make_float2(z0.x, zh.x);
            B = make_float2(z0.y, zh.y);
        } else {
            split_pair(z[k], z[L - k], A, B);
        }
        if (pairs_of_rows) {
            const int ra = row0 + 2 * sq;
            SA[(size_t)k * n1 + ra] = A;
            SA[(size_t)k * n1 + ra + 1] = B;
        } else {
            SA[(size_t)k * n1 + row0 + sq] = A;
            SB[(size_t)k * n1 + row0 + sq] = B;
        }
    }
}

// ---------------------------------------------------------------------------
// generic row kernels: real <-> packed spectrum along x^2
// ---------------------------------------------------------------------------
template <int LOGL, bool VEC>
__global__ void __launch_bounds__(NTHREADS) k_r2c(const float* __restrict__ f1, const float* __restrict__ f2,
                                                  float2* S1, float2* S2, int n1, int R, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int L = 1 << LOGL;
    float2* A = sm;
    float2* B = sm + R * L;
    const int row0 = blockIdx.x * R;
    const int nseq = VEC ? R : R / 2;
    for (int t = threadIdx.x; t < R * L; t += blockDim.x) {
        const int r = t >> LOGL, j = t & (L - 1);
        const size_t idx = (size_t)(row0 + r) * L + j;
        if (VEC) {
            A[r * L + j] = make_float2(f1[idx], f2[idx]);
        } else {
            float* a = reinterpret_cast<float*>(A);
            a[2 * ((r >> 1) * L + j) + (r & 1)] = f1[idx];
        }
    }
    __syncthreads();
    float2* X = smem_fft<LOGL, false>(A, B, nseq, tw);
    split_store<LOGL>(X, nseq, S1, VEC ? S2 : S1, n1, row0, !VEC);
}

template <int LOGL, bool VEC>
__global__ void __launch_bounds__(NTHREADS) k_c2r(const float2* S1, const float2* S2, float* __restrict__ f1,
                                                  float* __restrict__ f2, int n1, int R, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int L = 1 << LOGL;
    float2* A = sm;
    float2* B = sm + R * L;
    const int row0 = blockIdx.x * R;
    const int nseq = VEC ? R : R / 2;
    load_merge<LOGL>(A, nseq, S1, VEC ? S2 : S1, n1, row0, !VEC);
    __syncthreads();
    float2* X = smem_fft<LOGL, true>(A, B, nseq, tw);
    for (int t = threadIdx.x; t < R * L; t += blockDim.x) {
        const int r = t >> LOGL, j = t & (L - 1);
        const size_t idx = (size_t)(row0 + r) * L + j;
        if (VEC) {
            const float2 z = X[r * L + j];
            f1[idx] = z.x;
            f2[idx] = z.y;
        } else {
            const float* x = reinterpret_cast<const float*>(X);
            f1[idx] = x[2 * ((r >> 1) * L + j) + (r & 1)];
        }
    }
}

// ---------------------------------------------------------------------------
// RK2 (Heun) advection stage, state and incremental state equations
// (Eq. (e:state-eq-elim), (e:inc-state-eq-elim)):
//   k = -v . grad u_s - v~ . grad m(t)         (source only for the incremental state)
//   stage 1: u* = u_j + h k ;  stage 2: u_{j+1} = (u_j + u* + h k) / 2
// ---------------------------------------------------------------------------
template <int LOGL>
__global__ void __launch_bounds__(NTHREADS) k_row_adv(AdvArgs a, int n1, int N, int R, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int L = 1 << LOGL;
    float2* A = sm;
    float2* B = sm + R * L;
    const int row0 = blockIdx.x * R;
    float2* X = nullptr;
    if (a.G1) {
        load_merge<LOGL>(A, R, a.G1, a.G2, n1, row0, false);
        __syncthreads();
        X = smem_fft<LOGL, true>(A, B, R, tw);
    }
    float2* P = (X == A) ? B : A;  // pack buffer for the forward FFT of u_out
    float* pk = reinterpret_cast<float*>(P);
    for (int t = threadIdx.x; t < R * L; t += blockDim.x) {
        const int r = t >> LOGL, j = t & (L - 1);
        const size_t idx = (size_t)(row0 + r) * L + j;
        float d1 = 0.f, d2 = 0.f;
        if (X) {
            const float2 g = X[r * L + j];
            d1 = g.x;
            d2 = g.y;
        }
        if (a.grad_out) {
            a.grad_out[idx] = d1;
            a.grad_out[N + idx] = d2;
        }
        float k = -(a.v[idx] * d1 + a.v[N + idx] * d2);
        if (a.gm) k -= a.vt[idx] * a.gm[idx] + a.vt[N + idx] * a.gm[N + idx];
        const float uj = a.uj[idx];
        const float out = (a.stage == 1) ? fmaf(a.h, k, uj) : 0.5f * (uj + a.us[idx] + a.h * k);
        a.u_out[idx] = out;
        if (a.S_out) pk[2 * ((r >> 1) * L + j) + (r & 1)] = out;
    }
    if (!a.S_out) return;
    __syncthreads();
    float2* Y = smem_fft<LOGL, false>(P, P + (R / 2) * L, R / 2, tw);
    split_store<LOGL>(Y, R / 2, a.S_out, a.S_out, n1, row0, true);
}

// ---------------------------------------------------------------------------
// RK2 (Heun) stage of the adjoint / incremental adjoint equation, backward in
// time (Eq. (e:adj-eq-elim), (e:inc-adj-eq-elim) without the lambda term):
//   k = div(lam_s v); stage 1: lam* = lam_j + h k; stage 2: lam_{j-1} = (lam_j + lam* + h k) / 2
// Stage 2 also accumulates the body force b += w lam_{j-1} grad m_{j-1}
// (trapezoidal rule, Sec. 4.1 / Sec. 5) and both stages emit the packed
// spectra of the flux lam_out v for the next divergence.
// ---------------------------------------------------------------------------
template <int LOGL>
__global__ void __launch_bounds__(NTHREADS) k_row_adj(AdjArgs a, int n1, int N, int R, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int L = 1 << LOGL;
    float2* A = sm;
    float2* B = sm + R * L;
    const int row0 = blockIdx.x * R;
    load_merge<LOGL>(A, R / 2, a.D, a.D, n1, row0, true);
    __syncthreads();
    float2* X = smem_fft<LOGL, true>(A, A + (R / 2) * L, R / 2, tw);
    const float* xd = reinterpret_cast<const float*>(X);
    for (int t = threadIdx.x; t < R * L; t += blockDim.x) {
        const int r = t >> LOGL, j = t & (L - 1);
        const size_t idx = (size_t)(row0 + r) * L + j;
        const float dv = xd[2 * ((r >> 1) * L + j) + (r & 1)];
        const float lj = a.lj[idx];
        const float out = (a.stage == 1) ? fmaf(a.h, dv, lj) : 0.5f * (lj + a.ls[idx] + a.h * dv);
        a.l_out[idx] = out;
        if (a.b) {
            const float wl = a.w * out;
            a.b[idx] = fmaf(wl, a.gm[idx], a.b[idx]);
            a.b[N + idx] = fmaf(wl, a.gm[N + idx], a.b[N + idx]);
        }
        if (a.F1) B[r * L + j] = make_float2(out * a.v[idx], out * a.v[N + idx]);
    }
    if (!a.F1) return;
    __syncthreads();
    float2* Y = smem_fft<LOGL, false>(B, A, R, tw);
    split_store<LOGL>(Y, R, a.F1, a.F2, n1, row0, false);
}

// lam = ca*a + cb*c; b = w lam gm; flux spectra; partial 0.5*sum(lam^2)
template <int LOGL>
__global__ void __launch_bounds__(NTHREADS) k_adj_init(const float* __restrict__ a, float ca, const float* __restrict__ c,
                                                       float cb, const float* __restrict__ v, float* lam, float* b,
                                                       const float* __restrict__ gm, float w, float2* F1, float2* F2,
                                                       double* part, int n1, int N, int R, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int L = 1 << LOGL;
    float2* A = sm;
    float2* B = sm + R * L;
    const int row0 = blockIdx.x * R;
    double acc = 0.0;
    for (int t = threadIdx.x; t < R * L; t += blockDim.x) {
        const int r = t >> LOGL, j = t & (L - 1);
        const size_t idx = (size_t)(row0 + r) * L + j;
        float l = cb * c[idx];
        if (a) l = fmaf(ca, a[idx], l);
        lam[idx] = l;
        acc += 0.5 * (double)l * (double)l;
        if (b) {
            b[idx] = w * l * gm[idx];
            b[N + idx] = w * l * gm[N + idx];
        }
        A[r * L + j] = make_float2(l * v[idx], l * v[N + idx]);
    }
    if (part) {
        double s = block_reduce<0>(acc);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
    __syncthreads();
    float2* Y = smem_fft<LOGL, false>(A, B, R, tw);
    split_store<LOGL>(Y, R, F1, F2, n1, row0, false);
}

// ---------------------------------------------------------------------------
// column kernel: FFT along x^1, Fourier multiplier, inverse FFT
// ---------------------------------------------------------------------------
struct ColArgs {
    const float2* in[5];
    float2* out[2];
    SpecParams P;
    double* part;
    int cpb;
    int n2;
};

__device__ __forceinline__ float reg_sym(int regnorm, float kk) { return regnorm == 1 ? kk : kk * kk; }

__device__ __forceinline__ void proj_sym(const SpecParams& P, int pmode, float k1o, float k2o, float kk, float& K11,
                                         float& K12, float& K22) {
    K11 = 1.f; K12 = 0.f; K22 = 1.f;
    if (pmode == PROJ_IDENTITY) return;
    const float kko = k1o * k1o + k2o * k2o;
    if (kko == 0.f) return;
    float d = kko;
    if (pmode == PROJ_MASS) d += P.beta_v * reg_sym(P.regnorm, kk) / (P.beta_w * (1.f + kk));
    const float c = 1.f / d;
    K11 = 1.f - c * k1o * k1o;
    K12 = -c * k1o * k2o;
    K22 = 1.f - c * k2o * k2o;
}

template <int OP>
__device__ __forceinline__ void spec_apply(const SpecParams& P, float k1o, float k2o, float kk, const float2* x,
                                           float2* y, double& eacc, float ew) {
    const float s = P.scale;
    if (OP == OP_GRAD) {
        y[0] = cscale(cmuli(x[0]), k1o * s);
        y[1] = cscale(cmuli(x[0]), k2o * s);
    } else if (OP == OP_DIV) {
        y[0] = cscale(cmuli(cadd(cscale(x[0], k1o), cscale(x[1], k2o))), s);
    } else if (OP == OP_REG) {
        const float c = P.coefA * reg_sym(P.regnorm, kk) * s;
        y[0] = cscale(x[0], c);
        y[1] = cscale(x[1], c);
    } else if (OP == OP_PROJ) {
        float K11, K12, K22;
        proj_sym(P, P.pmode, k1o, k2o, kk, K11, K12, K22);
        y[0] = cscale(cadd(cscale(x[0], K11), cscale(x[1], K12)), s);
        y[1] = cscale(cadd(cscale(x[0], K12), cscale(x[1], K22)), s);
    } else if (OP == OP_PRECOND) {
        float a = reg_sym(P.regnorm, kk);
        if (kk == 0.f) a = 1.f;
        const float c = s / (P.beta_v * a);
        y[0] = cscale(x[0], c);
        y[1] = cscale(x[1], c);
    } else if (OP == OP_ASSEMBLE) {
        float K11, K12, K22;
        proj_sym(P, P.pmode, k1o, k2o, kk, K11, K12, K22);
        const float ca = P.coefA * reg_sym(P.regnorm, kk);
        y[0] = cscale(cadd(cscale(x[0], ca), cadd(cscale(x[2], K11), cscale(x[3], K12))), s);
        y[1] = cscale(cadd(cscale(x[1], ca), cadd(cscale(x[2], K12), cscale(x[3], K22))), s);
    } else if (OP == OP_ENERGY) {
        const double a = reg_sym(P.regnorm, kk);
        double e = P.ebv * a * ((double)x[0].x * x[0].x + (double)x[0].y * x[0].y + (double)x[1].x * x[1].x +
                                (double)x[1].y * x[1].y);
        if (P.ebw != 0.0) {
            const double dr = (double)k1o * x[0].x + (double)k2o * x[1].x;
            const double di = (double)k1o * x[0].y + (double)k2o * x[1].y;
            e += P.ebw * (1.0 + kk) * (dr * dr + di * di);
        }
        eacc += ew * e;
    } else if (OP == OP_DIVT_PROJ) {
        // d = div T:  d1 = i k1 T11 + i k2 T12 ; d2 = i k1 T12 + i k2 T22
        const float2 d1 = cmuli(cadd(cscale(x[0], k1o), cscale(x[1], k2o)));
        const float2 d2 = cmuli(cadd(cscale(x[1], k1o), cscale(x[2], k2o)));
        const float2 u0 = cadd(cscale(d1, P.coefA), x[3]);
        const float2 u1 = cadd(cscale(d2, P.coefA), x[4]);
        float K11, K12, K22;
        proj_sym(P, PROJ_LERAY, k1o, k2o, kk, K11, K12, K22);
        y[0] = cscale(cadd(cscale(u0, K11), cscale(u1, K12)), s);
        y[1] = cscale(cadd(cscale(u0, K12), cscale(u1, K22)), s);
    }
}

template <int LOGL, int NIN, int NOUT, int OP>
__global__ void __launch_bounds__(NTHREADS) k_col(ColArgs a, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int L = 1 << LOGL, H = L >> 1;
    constexpr int NF = NIN > NOUT ? NIN : NOUT;
    const int CPB = a.cpb;
    float2* A = sm;
    float2* B = sm + NF * CPB * L;
    const int j0 = blockIdx.x * CPB;
    for (int t = threadIdx.x; t < NIN * CPB * L; t += blockDim.x) {
        const int f = t / (CPB * L);
        const int rem = t - f * CPB * L;
        const int c = rem >> LOGL, i = rem & (L - 1);
        A[t] = a.in[f][(size_t)(j0 + c) * L + i];
    }
    __syncthreads();
    float2* X = smem_fft<LOGL, false>(A, B, NIN * CPB, tw);
    float2* Y = (X == A) ? B : A;
    double eacc = 0.0;
    const float kny2 = 0.5f * (float)a.n2;  // |k2| of the Nyquist column (even symbols)
    for (int t = threadIdx.x; t < CPB * L; t += blockDim.x) {
        const int c = t >> LOGL, p = t & (L - 1);
        const int j = j0 + c;
        const float k1 = (p < H) ? (float)p : (float)(p - L);
        const float k1o = (p == H) ? 0.f : k1;
        float2 x[NIN > 0 ? NIN : 1], y[NOUT > 0 ? NOUT : 1];
        if (j > 0) {
            const float k2 = (float)j;
#pragma unroll
            for (int f = 0; f < NIN; ++f) x[f] = X[(f * CPB + c) * L + p];
            spec_apply<OP>(a.P, k1o, k2, k1 * k1 + k2 * k2, x, y, eacc, 2.f);
#pragma unroll
            for (int o = 0; o < NOUT; ++o) Y[(o * CPB + c) * L + p] = y[o];
        } else {
            // packed column: A-part is k2 = 0, B-part is k2 = n2/2 (odd symbol 0)
            if (p > H) continue;
            const int pm = (L - p) & (L - 1);
            const bool self = (p == 0) || (p == H);
            float2 xa[NIN > 0 ? NIN : 1], xb[NIN > 0 ? NIN : 1], ya[NOUT > 0 ? NOUT : 1], yb[NOUT > 0 ? NOUT : 1];
#pragma unroll
            for (int f = 0; f < NIN; ++f) {
                const float2 zp = X[(f * CPB + c) * L + p];
                if (self) {
                    xa[f] = make_float2(zp.x, 0.f);
                    xb[f] = make_float2(zp.y, 0.f);
                } else {
                    split_pair(zp, X[(f * CPB + c) * L + pm], xa[f], xb[f]);
                }
            }
            const float ew = self ? 1.f : 2.f;
            spec_apply<OP>(a.P, k1o, 0.f, k1 * k1, xa, ya, eacc, ew);
            spec_apply<OP>(a.P, k1o, 0.f, k1 * k1 + kny2 * kny2, xb, yb, eacc, ew);
#pragma unroll
            for (int o = 0; o < NOUT; ++o) {
                if (self) {
                    Y[(o * CPB + c) * L + p] = make_float2(ya[o].x - yb[o].y, ya[o].y + yb[o].x);
                } else {
                    float2 zk, zm;
                    merge_pair(ya[o], yb[o], zk, zm);
                    Y[(o * CPB + c) * L + p] = zk;
                    Y[(o * CPB + c) * L + pm] = zm;
                }
            }
        }
    }
    if (OP == OP_ENERGY) {
        const double s = block_reduce<0>(eacc);
        if (threadIdx.x == 0) a.part[blockIdx.x] = s * a.P.escale;
        return;
    }
    __syncthreads();
    float2* Z = smem_fft<LOGL, true>(Y, X, NOUT * CPB, tw);
    for (int t = threadIdx.x; t < NOUT * CPB * L; t += blockDim.x) {
        const int o = t / (CPB * L);
        const int rem = t - o * CPB * L;
        const int c = rem >> LOGL, i = rem & (L - 1);
        a.out[o][(size_t)(j0 + c) * L + i] = Z[t];
    }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
static int rows_per_cta(int n1, int L) {
    int R = 4;
    while (R * L < 1024 && R * 2 <= n1) R *= 2;
    return R;
}

static int cols_per_cta(int W, int L) {
    int c = 1;
    while (c * L < 1024 && c * 2 <= W) c *= 2;
    return c;
}

// Opt in to more than 48 KB of dynamic shared memory once per kernel instantiation and size.
template <typename K>
static void set_smem(K kern, size_t bytes) {
    if (bytes <= 48 * 1024) return;
    static std::unordered_map<const void*, size_t> done;
    auto it = done.find((const void*)kern);
    if (it != done.end() && it->second >= bytes) return;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done[(const void*)kern] = bytes;
}

#define DISPATCH_LOG(LOG, ...)                        \
    switch (LOG) {                                    \
        case 4: { constexpr int LG = 4; __VA_ARGS__; } break;   \
        case 5: { constexpr int LG = 5; __VA_ARGS__; } break;   \
        case 6: { constexpr int LG = 6; __VA_ARGS__; } break;   \
        case 7: { constexpr int LG = 7; __VA_ARGS__; } break;   \
        case 8: { constexpr int LG = 8; __VA_ARGS__; } break;   \
        case 9: { constexpr int LG = 9; __VA_ARGS__; } break;   \
        case 10: { constexpr int LG = 10; __VA_ARGS__; } break; \
        default: break;                               \
    }

void launch_r2c_scalar(reg_ctx* ctx, const float* f, float2* S) {
    const int L = ctx->n2, R = rows_per_cta(ctx->n1, L);
    const size_t smem = 2 * (size_t)R * L * sizeof(float2);
    ktimer_begin(ctx, KC_ROW, 8.0 * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_r2c<LG, false>;
        set_smem(kern, smem);
        kern<<<ctx->n1 / R, NTHREADS, smem, ctx->stream>>>(f, nullptr, S, nullptr, ctx->n1, R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_r2c_vec(reg_ctx* ctx, const float* u1, const float* u2, float2* S1, float2* S2) {
    const int L = ctx->n2, R = rows_per_cta(ctx->n1, L);
    const size_t smem = 2 * (size_t)R * L * sizeof(float2);
    ktimer_begin(ctx, KC_ROW, 16.0 * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_r2c<LG, true>;
        set_smem(kern, smem);
        kern<<<ctx->n1 / R, NTHREADS, smem, ctx->stream>>>(u1, u2, S1, S2, ctx->n1, R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_c2r_scalar(reg_ctx* ctx, const float2* S, float* f) {
    const int L = ctx->n2, R = rows_per_cta(ctx->n1, L);
    const size_t smem = 2 * (size_t)R * L * sizeof(float2);
    ktimer_begin(ctx, KC_ROW, 8.0 * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_c2r<LG, false>;
        set_smem(kern, smem);
        kern<<<ctx->n1 / R, NTHREADS, smem, ctx->stream>>>(S, nullptr, f, nullptr, ctx->n1, R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_c2r_vec(reg_ctx* ctx, const float2* S1, const float2* S2, float* u1, float* u2) {
    const int L = ctx->n2, R = rows_per_cta(ctx->n1, L);
    const size_t smem = 2 * (size_t)R * L * sizeof(float2);
    ktimer_begin(ctx, KC_ROW, 16.0 * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_c2r<LG, true>;
        set_smem(kern, smem);
        kern<<<ctx->n1 / R, NTHREADS, smem, ctx->stream>>>(S1, S2, u1, u2, ctx->n1, R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_row_adv(reg_ctx* ctx, const AdvArgs& a) {
    const int L = ctx->n2, R = rows_per_cta(ctx->n1, L);
    const size_t smem = 2 * (size_t)R * L * sizeof(float2);
    // floats per node read/written: G 2 (complex half spectra = 1 float per node each), u_j 1,
    // u* 1 (stage 2), v 2, source gm + v~ 4, u_out 1, grad_out 2, S_out 1
    double fl = 1 + 2 + 1 + (a.G1 ? 2 : 0) + (a.stage == 2 ? 1 : 0) + (a.gm ? 4 : 0) + (a.grad_out ? 2 : 0) +
                (a.S_out ? 1 : 0);
    ktimer_begin(ctx, KC_ROWSTAGE, 4.0 * fl * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_row_adv<LG>;
        set_smem(kern, smem);
        kern<<<ctx->n1 / R, NTHREADS, smem, ctx->stream>>>(a, ctx->n1, ctx->N, R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_row_adj(reg_ctx* ctx, const AdjArgs& a) {
    const int L = ctx->n2, R = rows_per_cta(ctx->n1, L);
    const size_t smem = 2 * (size_t)R * L * sizeof(float2);
    // D 1, lam_j 1, lam* 1 (stage 2), v 2, l_out 1, body force b read+write 4 and gm 2, flux spectra 2
    double fl = 1 + 1 + 2 + 1 + (a.stage == 2 ? 1 : 0) + (a.b ? 6 : 0) + (a.F1 ? 2 : 0);
    ktimer_begin(ctx, KC_ROWSTAGE, 4.0 * fl * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_row_adj<LG>;
        set_smem(kern, smem);
        kern<<<ctx->n1 / R, NTHREADS, smem, ctx->stream>>>(a, ctx->n1, ctx->N, R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_adj_init(reg_ctx* ctx, const float* a, float ca, const float* c, float cb, const float* v, float* lam,
                     float* b, const float* gm, float w, float2* F1, float2* F2, double* part) {
    const int L = ctx->n2, R = rows_per_cta(ctx->n1, L);
    const size_t smem = 2 * (size_t)R * L * sizeof(float2);
    // a 1 (optional), c 1, v 2, lam 1, b 2 + gm 2, flux spectra 2
    ktimer_begin(ctx, KC_ROW, 4.0 * ((a ? 1 : 0) + 1 + 2 + 1 + 4 + 2) * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_adj_init<LG>;
        set_smem(kern, smem);
        kern<<<ctx->n1 / R, NTHREADS, smem, ctx->stream>>>(a, ca, c, cb, v, lam, b, gm, w, F1, F2, part, ctx->n1,
                                                            ctx->N, R, ctx->tw);
    });
    ktimer_end(ctx);
}

template <int NIN, int NOUT, int OP>
static void launch_col_t(reg_ctx* ctx, const float2* const* in, float2* const* out, const SpecParams& P,
                         double* part) {
    const int L = ctx->n1, W = ctx->n2 / 2;
    const int cpb = cols_per_cta(W, L);
    constexpr int NF = NIN > NOUT ? NIN : NOUT;
    const size_t smem = 2 * (size_t)NF * cpb * L * sizeof(float2);
    ColArgs a;
    for (int f = 0; f < 5; ++f) a.in[f] = (f < NIN) ? in[f] : nullptr;
    for (int o = 0; o < 2; ++o) a.out[o] = (o < NOUT) ? out[o] : nullptr;
    a.P = P;
    a.part = part;
    a.cpb = cpb;
    a.n2 = ctx->n2;
    ktimer_begin(ctx, KC_COL, 4.0 * (NIN + NOUT) * ctx->N);
    DISPATCH_LOG(ctx->log1, {
        auto kern = k_col<LG, NIN, NOUT, OP>;
        set_smem(kern, smem);
        kern<<<W / cpb, NTHREADS, smem, ctx->stream>>>(a, ctx->tw);
    });
    ktimer_end(ctx);
}

int col_blocks(reg_ctx* ctx) {
    const int L = ctx->n1, W = ctx->n2 / 2;
    return W / cols_per_cta(W, L);
}

void launch_col(reg_ctx* ctx, int op, const float2* const* in, float2* const* out, const SpecParams& P,
                double* part) {
    switch (op) {
        case OP_GRAD: launch_col_t<1, 2, OP_GRAD>(ctx, in, out, P, part); break;
        case OP_DIV: launch_col_t<2, 1, OP_DIV>(ctx, in, out, P, part); break;
        case OP_REG: launch_col_t<2, 2, OP_REG>(ctx, in, out, P, part); break;
        case OP_PROJ: launch_col_t<2, 2, OP_PROJ>(ctx, in, out, P, part); break;
        case OP_PRECOND: launch_col_t<2, 2, OP_PRECOND>(ctx, in, out, P, part); break;
        case OP_ASSEMBLE: launch_col_t<4, 2, OP_ASSEMBLE>(ctx, in, out, P, part); break;
        case OP_ENERGY: launch_col_t<2, 0, OP_ENERGY>(ctx, in, out, P, part); break;
        case OP_DIVT_PROJ: launch_col_t<5, 2, OP_DIVT_PROJ>(ctx, in, out, P, part); break;
        default: break;
    }
}

// ---------------------------------------------------------------------------
// pointwise and reduction kernels
// ---------------------------------------------------------------------------
__global__ void k_dot_partial(const float* __restrict__ x, const float* __restrict__ y, long long n, double* part) {
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)x[i] * (double)y[i];
    const double s = block_reduce<0>(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

int launch_dot_partial(reg_ctx* ctx, const float* x, const float* y, long long n, double* part) {
    ktimer_begin(ctx, KC_POINT, 8.0 * n);
    k_dot_partial<<<NBLK_RED, NTHREADS, 0, ctx->stream>>>(x, y, n, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

__global__ void k_maxnorm_partial(const float* __restrict__ v, int N, double* part) {
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double a = v[i], b = v[N + i];
        m = fmax(m, sqrt(a * a + b * b));
    }
    const double s = block_reduce<1>(m);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

int launch_maxnorm_partial(reg_ctx* ctx, const float* v, int N, double* part) {
    ktimer_begin(ctx, KC_POINT, 8.0 * N);
    k_maxnorm_partial<<<NBLK_RED, NTHREADS, 0, ctx->stream>>>(v, N, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

template <int OPR>
__global__ void k_finalize(const double* __restrict__ part, int np, double* out, double scale, int accumulate) {
    double acc = (OPR == 0) ? 0.0 : part[0];
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc = red_op<OPR>(acc, part[i]);
    const double s = block_reduce<OPR>(acc);
    if (threadIdx.x == 0) *out = scale * s + (accumulate ? *out : 0.0);
}

void launch_finalize(reg_ctx* ctx, const double* part, int np, double* out, double scale, int accumulate, int op) {
    ktimer_begin(ctx, KC_POINT, 8.0 * np);
    if (op == 0) k_finalize<0><<<1, NTHREADS, 0, ctx->stream>>>(part, np, out, scale, accumulate);
    else if (op == 1) k_finalize<1><<<1, NTHREADS, 0, ctx->stream>>>(part, np, out, scale, accumulate);
    else k_finalize<2><<<1, NTHREADS, 0, ctx->stream>>>(part, np, out, scale, accumulate);
    ktimer_end(ctx);
}

__global__ void k_axpby(long long n, float a, const float* __restrict__ x, float b, const float* y, float* out,
                        const double* __restrict__ scal, int num, int den) {
    float aa = a;
    if (num >= 0) aa = (float)((double)a * scal[num] / scal[den]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        // terms with a zero coefficient are skipped so that uninitialized (possibly NaN) inputs are never read
        const float yi = (b != 0.f) ? b * y[i] : 0.f;
        out[i] = (aa != 0.f) ? fmaf(aa, x[i], yi) : yi;
    }
}

void launch_axpby(reg_ctx* ctx, long long n, float a, const float* x, float b, float* y, int num, int den, float* out) {
    ktimer_begin(ctx, KC_POINT, 4.0 * n * ((a != 0.f) + (b != 0.f) + 1));
    k_axpby<<<NBLK_RED, NTHREADS, 0, ctx->stream>>>(n, a, x, b, y, out ? out : y, ctx->d_scal, num, den);
    ktimer_end(ctx);
}

__global__ void k_pcg_update(long long n, float* vt, const float* __restrict__ s, float* r, const float* __restrict__ Hs,
                             const double* __restrict__ scal, double* part) {
    const float kappa = (float)(scal[SL_RZ] / scal[SL_SHS]);
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        vt[i] = fmaf(kappa, s[i], vt[i]);
        const float ri = fmaf(-kappa, Hs[i], r[i]);
        r[i] = ri;
        acc += (double)ri * (double)ri;
    }
    const double t = block_reduce<0>(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

int launch_pcg_update(reg_ctx* ctx, long long n, float* vt, const float* s, float* r, const float* Hs, double* part) {
    ktimer_begin(ctx, KC_POINT, 4.0 * n * 6);
    k_pcg_update<<<NBLK_RED, NTHREADS, 0, ctx->stream>>>(n, vt, s, r, Hs, ctx->d_scal, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

__global__ void k_pcg_dir(long long n, const float* __restrict__ z, float* s, const double* __restrict__ scal) {
    const float mu = (float)(scal[SL_RZNEW] / scal[SL_RZ]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s[i] = fmaf(mu, s[i], z[i]);
}

void launch_pcg_dir(reg_ctx* ctx, long long n, const float* z, float* s) {
    ktimer_begin(ctx, KC_POINT, 4.0 * n * 3);
    k_pcg_dir<<<NBLK_RED, NTHREADS, 0, ctx->stream>>>(n, z, s, ctx->d_scal);
    ktimer_end(ctx);
}

__global__ void k_fill(long long n, float* y, float val) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = val;
}

void launch_fill(reg_ctx* ctx, long long n, float* y, float val) {
    ktimer_begin(ctx, KC_POINT, 4.0 * n);
    k_fill<<<NBLK_RED, NTHREADS, 0, ctx->stream>>>(n, y, val);
    ktimer_end(ctx);
}

// deformation gradient stage (Eq. (e:def-grad)); F planes (F11, F12, F21, F22),
// gF planes (d1 F11, d2 F11, d1 F12, d2 F12, ...), gv planes (d1 v1, d2 v1, d1 v2, d2 v2)
__global__ void k_defgrad_stage(int N, int stage, const float* __restrict__ F, const float* __restrict__ Fs,
                                const float* __restrict__ gF, const float* __restrict__ gv,
                                const float* __restrict__ v, float h, float* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float* Fin = (stage == 1) ? F : Fs;
        float Fv[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) Fv[c] = Fin[(size_t)c * N + i];
        const float v1 = v[i], v2 = v[N + i];
        const float g[4] = {gv[i], gv[(size_t)N + i], gv[2 * (size_t)N + i], gv[3 * (size_t)N + i]};
#pragma unroll
        for (int a = 0; a < 2; ++a) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int c = 2 * a + b;
                float rhs = -(v1 * gF[(size_t)(2 * c) * N + i] + v2 * gF[(size_t)(2 * c + 1) * N + i]);
                rhs += g[2 * a] * Fv[b] + g[2 * a + 1] * Fv[2 + b];
                const float f0 = F[(size_t)c * N + i];
                out[(size_t)c * N + i] = (stage == 1) ? fmaf(h, rhs, f0) : 0.5f * (f0 + Fs[(size_t)c * N + i] + h * rhs);
            }
        }
    }
}

void launch_defgrad_stage(reg_ctx* ctx, int stage, const float* F, const float* Fs, const float* gF, const float* gv,
                          const float* v, float h, float* out) {
    ktimer_begin(ctx, KC_POINT, 4.0 * (4 + (stage == 2 ? 4 : 0) + 8 + 4 + 2 + 4) * ctx->N);
    k_defgrad_stage<<<NBLK_RED, NTHREADS, 0, ctx->stream>>>(ctx->N, stage, F, Fs, gF, gv, v, h, out);
    ktimer_end(ctx);
}

__global__ void k_det_stats(int N, const float* __restrict__ F, float* detF, double* part) {
    double mn = 1e300, mx = -1e300, sm = 0.0, dmx = 0.0, dsm = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double f11 = F[i], f12 = F[(size_t)N + i], f21 = F[2 * (size_t)N + i], f22 = F[3 * (size_t)N + i];
        const double det = f11 * f22 - f12 * f21;
        const double D = sqrt((f11 - 1) * (f11 - 1) + f12 * f12 + f21 * f21 + (f22 - 1) * (f22 - 1));
        if (detF) detF[i] = (float)det;
        mn = fmin(mn, det);
        mx = fmax(mx, det);
        sm += det;
        dmx = fmax(dmx, D);
        dsm += D;
    }
    double r;
    r = block_reduce<2>(mn);
    if (threadIdx.x == 0) part[0 * gridDim.x + blockIdx.x] = r;
    r = block_reduce<0>(sm);
    if (threadIdx.x == 0) part[1 * gridDim.x + blockIdx.x] = r;
    r = block_reduce<1>(mx);
    if (threadIdx.x == 0) part[2 * gridDim.x + blockIdx.x] = r;
    r = block_reduce<1>(dmx);
    if (threadIdx.x == 0) part[3 * gridDim.x + blockIdx.x] = r;
    r = block_reduce<0>(dsm);
    if (threadIdx.x == 0) part[4 * gridDim.x + blockIdx.x] = r;
}

int launch_det_stats(reg_ctx* ctx, const float* F, float* detF, double* part) {
    ktimer_begin(ctx, KC_POINT, 4.0 * (4 + (detF ? 1 : 0)) * ctx->N);
    k_det_stats<<<NBLK_RED, NTHREADS, 0, ctx->stream>>>(ctx->N, F, detF, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

// shear control: strain rate, viscosity, stress (Eqs. (e:shear-control-reg-v), (e:1st-var-reg-v-nls))
#define SHEAR_EPS2 1.0e-6f
__global__ void k_shear_strain(int N, const float* __restrict__ gv, float nu, float* E, float* eta, float* T,
                               double* part) {
    const float pe = (1.f - nu) / (2.f * nu);
    const float pw = (1.f + nu) / (2.f * nu);
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float e11 = gv[i];
        const float e12 = 0.5f * (gv[(size_t)N + i] + gv[2 * (size_t)N + i]);
        const float e22 = gv[3 * (size_t)N + i];
        const float ee = e11 * e11 + 2.f * e12 * e12 + e22 * e22 + SHEAR_EPS2;
        const float et = powf(ee, pe);
        if (E) {
            E[i] = e11;
            E[(size_t)N + i] = e12;
            E[2 * (size_t)N + i] = e22;
        }
        if (eta) eta[i] = et;
        if (T) {
            T[i] = 2.f * et * e11;
            T[(size_t)N + i] = 2.f * et * e12;
            T[2 * (size_t)N + i] = 2.f * et * e22;
        }
        if (part) acc += (double)powf(ee, pw);
    }
    if (part) {
        const double s = block_reduce<0>(acc);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

int launch_shear_strain(reg_ctx* ctx, const float* gv, float nu, float* E, float* eta, float* T, double* part) {
    ktimer_begin(ctx, KC_POINT, 4.0 * (4 + (E ? 3 : 0) + (eta ? 1 : 0) + (T ? 3 : 0)) * ctx->N);
    k_shear_strain<<<NBLK_RED, NTHREADS, 0, ctx->stream>>>(ctx->N, gv, nu, E, eta, T, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

__global__ void k_shear_second(int N, const float* __restrict__ gvt, const float* __restrict__ E,
                               const float* __restrict__ eta, float nu, float* T) {
    const float cq = (1.f - nu) / nu;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float t11 = gvt[i];
        const float t12 = 0.5f * (gvt[(size_t)N + i] + gvt[2 * (size_t)N + i]);
        const float t22 = gvt[3 * (size_t)N + i];
        const float e11 = E[i], e12 = E[(size_t)N + i], e22 = E[2 * (size_t)N + i];
        const float ee = e11 * e11 + 2.f * e12 * e12 + e22 * e22 + SHEAR_EPS2;
        const float q = cq * (e11 * t11 + 2.f * e12 * t12 + e22 * t22) / ee;
        const float c = 2.f * eta[i];
        T[i] = c * (t11 + q * e11);
        T[(size_t)N + i] = c * (t12 + q * e12);
        T[2 * (size_t)N + i] = c * (t22 + q * e22);
    }
}

void launch_shear_second(reg_ctx* ctx, const float* gvt, const float* E, const float* eta, float nu, float* T) {
    ktimer_begin(ctx, KC_POINT, 4.0 * (4 + 3 + 1 + 3) * ctx->N);
    k_shear_second<<<NBLK_RED, NTHREADS, 0, ctx->stream>>>(ctx->N, gvt, E, eta, nu, T);
    ktimer_end(ctx);
}
