// CUDA kernels (sm_103a) for the pseudospectral Gauss-Newton-Krylov
// registration solver of Mang & Biros (arXiv 1503.00757).
//
// A 2-D transform of an n1 x n2 real field is split into two passes over HBM:
//   * row kernels: one CTA owns R consecutive rows; real FFTs along x^2
//     (two real rows, or two real fields of one row, per complex FFT), fused
//     with the pointwise work of an RK2 stage (Sec. 4) on the physical side;
//   * column kernels: one CTA owns C consecutive columns of the packed half
//     spectra (row-quad tiled layout, see fft_reg.cuh); forward FFT along x^1,
//     a Fourier multiplier (gradient, divergence, A, K, preconditioner,
//     Eq. (e:var-reg-v), (e:project-body-force), Appendix E), inverse FFT.
// All transforms are register-resident radix-8 FFTs (fft_reg.cuh).
// Pointwise and reduction kernels serve the PCG (Algorithm 2) and the
// deformation gradient (Eq. (e:def-grad)); FP64 accumulation for all sums.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "fft.cuh"
#include "fft_reg.cuh"
#include "internal.h"

#define NTHREADS 256
#define NBLK_RED 304  // 2 x 152 SMs

// Programmatic dependent launch: every kernel waits for the grid it depends
// on (it has completed and its writes are visible after the wait) and then
// lets the next kernel in the stream begin launching, so the launch, CTA
// scheduling and prologue of kernel k+1 overlap the tail of kernel k.  Since
// each kernel triggers only after its own wait, a kernel that starts early
// may read, before its wait, anything written two or more launches back
// (the RK2 row-stage kernels prefetch their pointwise operands that way).
// Without a programmatic dependency both instructions are no-ops.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch with the programmatic-stream-serialization attribute (ctx->pdl) or plainly.
template <typename... KArgs, typename... Args>
static void launch_k(reg_ctx* ctx, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = ctx->pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// timing hooks
// ---------------------------------------------------------------------------
// Inside a stream capture an external record becomes an event-record node of
// the graph; outside a capture the plain record is used.
static void ktimer_record(reg_ctx* ctx, cudaEvent_t e) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cs);
    if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, ctx->stream, cudaEventRecordExternal);
    else cudaEventRecord(e, ctx->stream);
}

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
    ktimer_record(ctx, ep.a);
    ctx->events.push_back(ep);
}

void ktimer_end(reg_ctx* ctx) {
    if (!ctx->timing) return;
    ktimer_record(ctx, ctx->events.back().b);
}

void fill_twiddles(float2* h) {
    // w^t = exp(-2 pi i t / 1024), t < 1024
    for (int t = 0; t < REG_TW_N; ++t) {
        const double a = -2.0 * M_PI * (double)t / (double)REG_TW_N;
        h[t] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    // per-pass tables of the lengths 2^4 .. 2^10 (layout in fft.cuh), from the exact angles
    for (int logl = 4; logl <= 10; ++logl) {
        const int L = 1 << logl;
        for (int i = 0; i < tw_passes(logl); ++i) {
            const int P = tw_groups(logl, i), s = 1 << (3 * i);
            for (int k = 1; k <= 7; ++k)
                for (int p = 0; p < P; ++p) {
                    const double a = -2.0 * M_PI * (double)(p * k * s) / (double)L;
                    h[twp_base(logl) + tw_off(logl, i) + (k - 1) * P + p] =
                        make_float2((float)std::cos(a), (float)std::sin(a));
                }
        }
    }
}

cudaError_t k_init_twiddles(reg_ctx* ctx) {
    std::vector<float2> h(REG_TW_TOTAL);
    fill_twiddles(h.data());
    return cudaMemcpy(ctx->tw, h.data(), sizeof(float2) * REG_TW_TOTAL, cudaMemcpyHostToDevice);
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
    if (blockDim.x < 32) {
        // a partial warp: no shuffles across lanes that do not exist
        __syncthreads();
        red_sm[threadIdx.x] = v;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int i = 1; i < (int)blockDim.x; ++i) v = red_op<OPR>(v, red_sm[i]);
        return v;  // valid in thread 0
    }
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
// row kernels: real rows <-> packed half spectra along x^2, fused with the
// pointwise work of the RK2 stages.  A CTA owns R consecutive rows (R a
// multiple of 4, so its packed spectra form one contiguous tiled chunk of
// R * L/2 entries starting at row0 * L/2); T = L/8 threads per row FFT.
// Shared memory: region A (R*L float2: staging) + region X (2*R*L float2:
// FFT exchange buffers, 2*L per FFT).
// ---------------------------------------------------------------------------
// The RK2 row kernels come in two variants.  PRE = true loads the operands
// written two or more launches back (u_j, u*, v, grad m, v~, lambda, b)
// before waiting on the preceding column kernel, which overlaps those loads
// with its tail but holds ~40 more registers per thread (one CTA of 512
// threads per SM).  PRE = false loads them after the FFT and is compiled for
// two CTAs of 512 threads per SM (64 registers), which is what concurrent
// solves and 1024-point rows want.  The autotuner chooses per grid.
// Elements per batch of late operand loads in the RK2 row kernels: the largest
// batch that stays within 64 registers without spills (advection 8, adjoint 4).
constexpr int ADV_LOAD_BATCH = 8;
constexpr int ADJ_LOAD_BATCH = 4;

template <bool PRE>
struct RowBlocks {
    static constexpr int value = PRE ? 1 : 2;
};

template <int LOGL>
__device__ __forceinline__ void stage_chunk(float2* dst, const float2* __restrict__ src, int n) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int i = threadIdx.x; i < n / 2; i += blockDim.x) d4[i] = s4[i];
}

template <int LOGL, bool VEC>
__global__ void __launch_bounds__(512) k_r2c(const float* __restrict__ f1, const float* __restrict__ f2,
                                             float2* S1, float2* S2, int R, const float2* __restrict__ tw) {
    pdl_entry();
    extern __shared__ __align__(16) float2 sm[];
    constexpr int L = 1 << LOGL, T = L >> 3, W = L >> 1;
    float2* A = sm;
    float2* X = sm + R * L;
    const int q = threadIdx.x / T, t = threadIdx.x - q * T;
    const int row0 = blockIdx.x * R;
    const int nfft = VEC ? R : R / 2;
    const bool active = q < nfft;
    float2 x[8];
    if (active) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int j = t + k * T;
            if (VEC) {
                const size_t idx = (size_t)(row0 + q) * L + j;
                x[k] = make_float2(f1[idx], f2[idx]);
            } else {
                const size_t idx = (size_t)(row0 + 2 * q) * L + j;
                x[k] = make_float2(f1[idx], f1[idx + L]);
            }
        }
    }
    reg_fft<LOGL, false>(x, t, active, X + 2 * q * fft_buf(L), X + 2 * q * fft_buf(L) + fft_buf(L), tw);
    if (active) {
#pragma unroll
        for (int k = 0; k < 8; ++k) A[q * L + t + k * T] = x[k];
    }
    __syncthreads();
    const size_t base = (size_t)row0 * W;
    for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x) {
        const int r = ((idx / (4 * W)) << 2) | (idx & 3);
        const int e = (idx >> 2) & (W - 1);
        if (VEC) {
            S1[base + idx] = split_entry<LOGL>(A + r * L, 0, e);
            S2[base + idx] = split_entry<LOGL>(A + r * L, 1, e);
        } else {
            S1[base + idx] = split_entry<LOGL>(A + (r >> 1) * L, r & 1, e);
        }
    }
}

template <int LOGL, bool VEC>
__global__ void __launch_bounds__(512) k_c2r(const float2* __restrict__ S1, const float2* __restrict__ S2,
                                             float* __restrict__ f1, float* __restrict__ f2, int R,
                                             const float2* __restrict__ tw) {
    pdl_entry();
    extern __shared__ __align__(16) float2 sm[];
    constexpr int L = 1 << LOGL, T = L >> 3, W = L >> 1;
    float2* A = sm;
    float2* X = sm + R * L;
    const int q = threadIdx.x / T, t = threadIdx.x - q * T;
    const int row0 = blockIdx.x * R;
    const size_t base = (size_t)row0 * W;
    stage_chunk<LOGL>(A, S1 + base, R * W);
    if (VEC) stage_chunk<LOGL>(A + R * W, S2 + base, R * W);
    __syncthreads();
    const int nfft = VEC ? R : R / 2;
    const bool active = q < nfft;
    float2 x[8];
    if (active) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            x[k] = VEC ? merged_entry<LOGL>(A, q, A + R * W, q, t + k * T)
                       : merged_entry<LOGL>(A, 2 * q, A, 2 * q + 1, t + k * T);
    }
    reg_fft<LOGL, true>(x, t, active, X + 2 * q * fft_buf(L), X + 2 * q * fft_buf(L) + fft_buf(L), tw);
    if (active) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int j = t + k * T;
            if (VEC) {
                const size_t idx = (size_t)(row0 + q) * L + j;
                f1[idx] = x[k].x;
                f2[idx] = x[k].y;
            } else {
                const size_t idx = (size_t)(row0 + 2 * q) * L + j;
                f1[idx] = x[k].x;
                f1[idx + L] = x[k].y;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// RK2 (Heun) advection stage of the state and incremental state equations
// (Eq. (e:state-eq-elim), (e:inc-state-eq-elim)):
//   k = -v . grad u_s - v~ . grad m(t)         (source only for the incremental state)
//   stage 1: u* = u_j + h k ;  stage 2: u_{j+1} = (u_j + u* + h k) / 2
// grad u_s arrives as packed spectra (G1, G2) from the column pass; the stage
// result u_out leaves as its packed spectrum S_out for the next column pass.
// ---------------------------------------------------------------------------
template <int LOGL, bool PRE>
__global__ void __launch_bounds__(512, RowBlocks<PRE>::value) k_row_adv(AdvArgs a, int N, int R,
                                                                           const float2* __restrict__ tw) {
    extern __shared__ __align__(16) float2 sm[];
    constexpr int L = 1 << LOGL, T = L >> 3, W = L >> 1;
    float2* A = sm;
    float2* X = sm + R * L;
    const int q = threadIdx.x / T, t = threadIdx.x - q * T;
    const int row0 = blockIdx.x * R;
    const size_t base = (size_t)row0 * W;
    const size_t rowbase = (size_t)(row0 + q) * L;
    // Operands written at least two launches earlier (u_j, u*, v, grad m, v~) are
    // loaded before waiting on the preceding column kernel; only G depends on it.
    // u_j == nullptr stands for u_j = 0 (the incremental state at t = 0).  With
    // PRE = false the operands are read after the FFT instead, which keeps the
    // register count low enough for two CTAs per SM.
    float pv1[8], pv2[8], puj[8], pus[8], psrc[8];
    auto load_ops = [&](int k) {
        const size_t idx = rowbase + t + k * T;
        pv1[k] = a.v[idx];
        pv2[k] = a.v[N + idx];
        puj[k] = a.uj ? a.uj[idx] : 0.f;
        pus[k] = (a.stage == 2) ? a.us[idx] : 0.f;
        psrc[k] = a.gm ? -(a.vt[idx] * a.gm[idx] + a.vt[N + idx] * a.gm[N + idx]) : 0.f;
    };
    const bool early = PRE && !a.late;
    if (early) {
#pragma unroll
        for (int k = 0; k < 8; ++k) load_ops(k);
    }
    pdl_entry();
    float2 x[8];
    if (a.G1) {
        stage_chunk<LOGL>(A, a.G1 + base, R * W);
        stage_chunk<LOGL>(A + R * W, (a.G2 ? a.G2 : a.Sd2) + base, R * W);
        __syncthreads();
        if (a.G2) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = merged_entry<LOGL>(A, q, A + R * W, q, t + k * T);
        } else {
            const float c = 1.0f / (float)L;
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = merged_entry_d2<LOGL>(A, q, A + R * W, q, t + k * T, c);
        }
        reg_fft<LOGL, true>(x, t, true, X + 2 * q * fft_buf(L), X + 2 * q * fft_buf(L) + fft_buf(L), tw);
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = make_float2(0.f, 0.f);
    }
    // Late operands are loaded a batch of elements at a time before any of those
    // elements' results is stored, so that the loads of a batch are in flight together
    // (the compiler cannot move a load above a store to a pointer that may alias it).
    float out[8];
#pragma unroll
    for (int k0 = 0; k0 < 8; k0 += ADV_LOAD_BATCH) {
        if (!early) {
#pragma unroll
            for (int k = k0; k < k0 + ADV_LOAD_BATCH; ++k) load_ops(k);
        }
#pragma unroll
        for (int k = k0; k < k0 + ADV_LOAD_BATCH; ++k) {
            const size_t idx = rowbase + t + k * T;
            const float d1 = x[k].x, d2 = x[k].y;
            if (a.grad_out) {
                a.grad_out[idx] = d1;
                a.grad_out[N + idx] = d2;
            }
            const float kk = psrc[k] - (pv1[k] * d1 + pv2[k] * d2);
            out[k] = (a.stage == 1) ? fmaf(a.h, kk, puj[k]) : 0.5f * (puj[k] + pus[k] + a.h * kk);
            a.u_out[idx] = out[k];
        }
    }
    if (!a.S_out) return;
    float* O = reinterpret_cast<float*>(A);
#pragma unroll
    for (int k = 0; k < 8; ++k) O[q * L + t + k * T] = out[k];
    __syncthreads();
    const bool act2 = q < R / 2;
    if (act2) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = t + k * T;
            x[k] = make_float2(O[2 * q * L + e], O[(2 * q + 1) * L + e]);
        }
    }
    reg_fft<LOGL, false>(x, t, act2, X + 2 * q * fft_buf(L), X + 2 * q * fft_buf(L) + fft_buf(L), tw);
    if (act2) {
#pragma unroll
        for (int k = 0; k < 8; ++k) A[q * L + t + k * T] = x[k];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x) {
        const int r = ((idx / (4 * W)) << 2) | (idx & 3);
        const int e = (idx >> 2) & (W - 1);
        a.S_out[base + idx] = split_entry<LOGL>(A + (r >> 1) * L, r & 1, e);
    }
}

// ---------------------------------------------------------------------------
// RK2 (Heun) stage of the adjoint / incremental adjoint equation, backward in
// time (Eq. (e:adj-eq-elim), (e:inc-adj-eq-elim) without the lambda term):
//   k = div(lam_s v); stage 1: lam* = lam_j + h k; stage 2: lam_{j-1} = (lam_j + lam* + h k) / 2
// Stage 2 also accumulates the body force b += w lam_{j-1} grad m_{j-1}
// (trapezoidal rule, Sec. 3.1 / Sec. 4); the flux lam_out v leaves as two
// packed spectra for the next divergence.
// ---------------------------------------------------------------------------
template <int LOGL>
__device__ __forceinline__ void flux_fft_store(float2 (&x)[8], int q, int t, int R, int row0, float2* A, float2* X,
                                               float2* F1, float2* F2, const float2* __restrict__ tw) {
    constexpr int L = 1 << LOGL, T = L >> 3, W = L >> 1;
    reg_fft<LOGL, false>(x, t, true, X + 2 * q * fft_buf(L), X + 2 * q * fft_buf(L) + fft_buf(L), tw);
#pragma unroll
    for (int k = 0; k < 8; ++k) A[q * L + t + k * T] = x[k];
    __syncthreads();
    const size_t base = (size_t)row0 * W;
    for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x) {
        const int r = ((idx / (4 * W)) << 2) | (idx & 3);
        const int e = (idx >> 2) & (W - 1);
        F1[base + idx] = split_entry<LOGL>(A + r * L, 0, e);
        F2[base + idx] = split_entry<LOGL>(A + r * L, 1, e);
    }
}

// FULL (full Newton, Eq. (e:inc-adj-eq-elim) with the lambda term): the flux of the next
// divergence is lam_out v + lam_src v~ (lam_src: the adjoint state at the time that divergence
// is evaluated) and stage 2 adds w lam_src grad m~ to the body force.  Compiled only without
// prefetch, with a smaller load batch (more operands per element).
template <int LOGL, bool PRE, bool FULL>
__global__ void __launch_bounds__(512, RowBlocks<PRE>::value) k_row_adj(AdjArgs a, int N, int R,
                                                                           const float2* __restrict__ tw) {
    extern __shared__ __align__(16) float2 sm[];
    constexpr int L = 1 << LOGL, T = L >> 3, W = L >> 1;
    constexpr int BATCH = FULL ? 2 : ADJ_LOAD_BATCH;
    float2* A = sm;
    float2* X = sm + R * L;
    const int q = threadIdx.x / T, t = threadIdx.x - q * T;
    const int row0 = blockIdx.x * R;
    const size_t rowbase = (size_t)(row0 + q) * L;
    // Operands written at least two launches earlier (lam_j, lam*, v, b, grad m)
    // are loaded before waiting on the preceding column kernel, which writes D
    // (after the FFT with PRE = false, as in k_row_adv).
    float plj[8], pls[8], pv1[8], pv2[8], pb1[8], pb2[8], pg1[8], pg2[8];
    float psrc[8], pt1[8], pt2[8], ph1[8], ph2[8];
    auto load_ops = [&](int k) {
        const size_t idx = rowbase + t + k * T;
        plj[k] = a.lj[idx];
        pls[k] = (a.stage == 2) ? a.ls[idx] : 0.f;
        pv1[k] = a.v[idx];
        pv2[k] = a.v[N + idx];
        if (a.b) {
            pb1[k] = a.b[idx];
            pb2[k] = a.b[N + idx];
            pg1[k] = a.gm[idx];
            pg2[k] = a.gm[N + idx];
        }
        if (FULL) {
            psrc[k] = a.lsrc[idx];
            pt1[k] = a.vt[idx];
            pt2[k] = a.vt[N + idx];
            if (a.b) {
                ph1[k] = a.gmt[idx];
                ph2[k] = a.gmt[N + idx];
            }
        }
    };
    if (PRE && !FULL) {
#pragma unroll
        for (int k = 0; k < 8; ++k) load_ops(k);
    }
    pdl_entry();
    stage_chunk<LOGL>(A, a.D + (size_t)row0 * W, R * W);
    __syncthreads();
    const bool act1 = q < R / 2;
    float2 x[8];
    if (act1) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = merged_entry<LOGL>(A, 2 * q, A, 2 * q + 1, t + k * T);
    }
    reg_fft<LOGL, true>(x, t, act1, X + 2 * q * fft_buf(L), X + 2 * q * fft_buf(L) + fft_buf(L), tw);
    float* O = reinterpret_cast<float*>(A);
    if (act1) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            O[2 * q * L + t + k * T] = x[k].x;
            O[(2 * q + 1) * L + t + k * T] = x[k].y;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k0 = 0; k0 < 8; k0 += BATCH) {
        if (!PRE || FULL) {
#pragma unroll
            for (int k = k0; k < k0 + BATCH; ++k) load_ops(k);  // batched, as in k_row_adv
        }
#pragma unroll
        for (int k = k0; k < k0 + BATCH; ++k) {
            const int j = t + k * T;
            const size_t idx = rowbase + j;
            const float dv = O[q * L + j];
            const float out = (a.stage == 1) ? fmaf(a.h, dv, plj[k]) : 0.5f * (plj[k] + pls[k] + a.h * dv);
            a.l_out[idx] = out;
            if (a.b) {
                const float wl = a.w * out;
                float b1 = fmaf(wl, pg1[k], pb1[k]), b2 = fmaf(wl, pg2[k], pb2[k]);
                if (FULL) {
                    const float ws = a.w * psrc[k];
                    b1 = fmaf(ws, ph1[k], b1);
                    b2 = fmaf(ws, ph2[k], b2);
                }
                a.b[idx] = b1;
                a.b[N + idx] = b2;
            }
            x[k] = FULL ? make_float2(fmaf(out, pv1[k], psrc[k] * pt1[k]), fmaf(out, pv2[k], psrc[k] * pt2[k]))
                        : make_float2(out * pv1[k], out * pv2[k]);
        }
    }
    if (!a.F1) return;
    flux_fft_store<LOGL>(x, q, t, R, row0, A, X, a.F1, a.F2, tw);
}

// lam = ca*a + cb*c; b = w lam gm; flux spectra; partial 0.5*sum(lam^2).  With lsrc (full
// Newton): b += w lsrc gmt and the flux is lam v + lsrc v~.
template <int LOGL>
__global__ void __launch_bounds__(512) k_adj_init(const float* __restrict__ a, float ca, const float* __restrict__ c,
                                                  float cb, const float* __restrict__ v, float* lam, float* b,
                                                  const float* __restrict__ gm, float w, float2* F1, float2* F2,
                                                  double* part, int N, int R, const float2* __restrict__ tw,
                                                  const float* __restrict__ lsrc, const float* __restrict__ vt,
                                                  const float* __restrict__ gmt) {
    pdl_entry();
    extern __shared__ __align__(16) float2 sm[];
    constexpr int L = 1 << LOGL, T = L >> 3;
    float2* A = sm;
    float2* X = sm + R * L;
    const int q = threadIdx.x / T, t = threadIdx.x - q * T;
    const int row0 = blockIdx.x * R;
    const size_t rowbase = (size_t)(row0 + q) * L;
    double acc = 0.0;
    float2 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const size_t idx = rowbase + t + k * T;
        float l = cb * c[idx];
        if (a) l = fmaf(ca, a[idx], l);
        lam[idx] = l;
        acc += 0.5 * (double)l * (double)l;
        if (lsrc) {
            const float ls = lsrc[idx];
            b[idx] = fmaf(w * ls, gmt[idx], w * l * gm[idx]);
            b[N + idx] = fmaf(w * ls, gmt[N + idx], w * l * gm[N + idx]);
            x[k] = make_float2(fmaf(l, v[idx], ls * vt[idx]), fmaf(l, v[N + idx], ls * vt[N + idx]));
        } else {
            b[idx] = w * l * gm[idx];
            b[N + idx] = w * l * gm[N + idx];
            x[k] = make_float2(l * v[idx], l * v[N + idx]);
        }
    }
    if (part) {
        const double s = block_reduce<0>(acc);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
    flux_fft_store<LOGL>(x, q, t, R, row0, A, X, F1, F2, tw);
}

// ---------------------------------------------------------------------------
// column kernel: FFT along x^1, Fourier multiplier, inverse FFT.  A CTA owns
// C consecutive columns e0..e0+C-1 of the packed half spectra (T = n1/8
// threads per column FFT); each 4-row tile contributes C*32 contiguous bytes.
// Column 0 holds the k2 = 0 column (real part) and the k2 = n2/2 column
// (imaginary part) of each real field; they are separated per wavenumber with
// the partner entry at -k1 before the multiplier is applied.
// ---------------------------------------------------------------------------
struct ColArgs {
    const float2* in[5];
    float2* out[2];
    SpecParams P;
    double* part;
    int cpb;
    int lcpb;       // log2(cpb): cpb is a power of two (reg_set_tiles / reg_autotune limits)
    int n2;
};

// |k|^2 (H1), |k|^4 (H2) or |k|^6 (H3): the regularization symbol A^(k)
__device__ __forceinline__ float reg_sym(int regnorm, float kk) {
    return regnorm == 1 ? kk : (regnorm == 2 ? kk * kk : kk * kk * kk);
}

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
    } else if (OP == OP_QINV || OP == OP_QMUL) {
        const float a = (kk == 0.f) ? 1.f : reg_sym(P.regnorm, kk);
        const float q = sqrtf(P.beta_v * a);
        const float c = (OP == OP_QINV) ? s / q : s * q;
        y[0] = cscale(x[0], c);
        y[1] = cscale(x[1], c);
    } else if (OP == OP_ASSEMBLE_Y) {
        float K11, K12, K22;
        proj_sym(P, P.pmode, k1o, k2o, kk, K11, K12, K22);
        const float a = (kk == 0.f) ? 1.f : reg_sym(P.regnorm, kk);
        const float qi = s / sqrtf(P.beta_v * a);
        const float c0 = (kk == 0.f) ? 0.f : s;
        y[0] = cadd(cscale(x[0], c0), cscale(cadd(cscale(x[2], K11), cscale(x[3], K12)), qi));
        y[1] = cadd(cscale(x[1], c0), cscale(cadd(cscale(x[2], K12), cscale(x[3], K22)), qi));
    } else if (OP == OP_QNORM) {
        const double a = (kk == 0.f) ? 1.0 : (double)reg_sym(P.regnorm, kk);
        eacc += ew * (double)P.beta_v * a *
                ((double)x[0].x * x[0].x + (double)x[0].y * x[0].y + (double)x[1].x * x[1].x + (double)x[1].y * x[1].y);
    } else if (OP == OP_ENERGY_Y) {
        // (beta_v / 2) <A v, v> = |Pi0 y|^2 / 2 ; mass-source term (beta_w / 2) (1 + |k|^2) |k~ . v^|^2 with v^ = y^ / Q^
        double e = (kk == 0.f) ? 0.0
                               : 0.5 * ((double)x[0].x * x[0].x + (double)x[0].y * x[0].y + (double)x[1].x * x[1].x +
                                        (double)x[1].y * x[1].y);
        if (P.ebw != 0.0) {
            const double a = (kk == 0.f) ? 1.0 : (double)reg_sym(P.regnorm, kk);
            const double dr = (double)k1o * x[0].x + (double)k2o * x[1].x;
            const double di = (double)k1o * x[0].y + (double)k2o * x[1].y;
            e += P.ebw * (1.0 + kk) * (dr * dr + di * di) / ((double)P.beta_v * a);
        }
        eacc += ew * e;
    } else if (OP == OP_MASSP) {
        const float kko = k1o * k1o + k2o * k2o;
        if (kko == 0.f) {
            y[0] = make_float2(0.f, 0.f);
            y[1] = make_float2(0.f, 0.f);
        } else {
            const float m = 1.f + 2.f * P.beta_v * (float)__ldg(P.eta_bar) / (P.beta_w * (1.f + kk));
            const float c = s / (kko * m);
            const float2 pr = cadd(cscale(x[0], k1o), cscale(x[1], k2o));
            y[0] = cscale(pr, c * k1o);
            y[1] = cscale(pr, c * k2o);
        }
    } else if (OP == OP_SMOOTH) {
        y[0] = cscale(x[0], expf(-P.coefA * kk) * s);
    } else if (OP == OP_SMOOTH_PROJ) {
        float K11, K12, K22;
        proj_sym(P, PROJ_LERAY, k1o, k2o, kk, K11, K12, K22);
        const float gs = expf(-P.coefA * kk) * s;
        y[0] = cscale(cadd(cscale(x[0], K11), cscale(x[1], K12)), gs);
        y[1] = cscale(cadd(cscale(x[0], K12), cscale(x[1], K22)), gs);
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
    } else if (OP == OP_GRAD1 || OP == OP_DIV1) {
        y[0] = cscale(cmuli(x[0]), k1o * s);
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
__global__ void __launch_bounds__(256) k_col(ColArgs a, const float2* __restrict__ tw) {
    pdl_entry();
    extern __shared__ __align__(16) float2 sm[];
    constexpr int L = 1 << LOGL, T = L >> 3, H = L >> 1;
    const int C = a.cpb;
    const int g_shift = a.lcpb + 2, g_mask = 4 * C - 1;  // idx -> (4-row group, column in CTA, row in group)
    const int W = a.n2 >> 1;
    float2* A = sm;
    float2* X = sm + C * L;
    float2* B2 = X + 2 * C * fft_buf(L);  // OP_DIV1: the untransformed second input, staged with the first
    const int c = threadIdx.x / T, t = threadIdx.x - c * T;
    const int e0 = blockIdx.x * C;
    const int e = e0 + c;
    float2 xin[NIN][8];
#pragma unroll
    for (int f = 0; f < NIN; ++f) {
        const float2* src = a.in[f];
        for (int idx = threadIdx.x; idx < C * L; idx += blockDim.x) {
            const int g = idx >> g_shift;
            const int rem = idx & g_mask;
            const int cc = rem >> 2, rr = rem & 3;
            const size_t gi = ((size_t)g * W + e0 + cc) * 4 + rr;
            A[cc * L + 4 * g + rr] = src[gi];
            if (OP == OP_DIV1 && f == 0) B2[cc * L + 4 * g + rr] = a.in[1][gi];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; ++k) xin[f][k] = A[c * L + t + k * T];
        reg_fft<LOGL, false>(xin[f], t, true, X + 2 * c * fft_buf(L), X + 2 * c * fft_buf(L) + fft_buf(L), tw);
    }
    float2 y[NOUT > 0 ? NOUT : 1][8];
    double eacc = 0.0;
    if (e0 == 0) {
        // packed column 0: stage every input's column-0 spectrum (natural order) for the -k1 partner
        float2* Zs = sm;  // NIN * L <= C * L + 2 * C * fft_buf(L) entries
        __syncthreads();
        if (c == 0) {
#pragma unroll
            for (int f = 0; f < NIN; ++f)
#pragma unroll
                for (int k = 0; k < 8; ++k) Zs[f * L + t + k * T] = xin[f][k];
        }
        __syncthreads();
    }
    const float kny2 = 0.5f * (float)a.n2;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int p = t + k * T;
        const float k1 = (p < H) ? (float)p : (float)(p - L);
        const float k1o = (p == H) ? 0.f : k1;
        float2 xv[NIN], yv[NOUT > 0 ? NOUT : 1];
        if (e > 0) {
#pragma unroll
            for (int f = 0; f < NIN; ++f) xv[f] = xin[f][k];
            const float k2 = (float)e;
            spec_apply<OP>(a.P, k1o, k2, k1 * k1 + k2 * k2, xv, yv, eacc, 2.f);
        } else {
            const int pm = (L - p) & (L - 1);
            float2 xb[NIN], yb[NOUT > 0 ? NOUT : 1];
#pragma unroll
            for (int f = 0; f < NIN; ++f) {
                const float2 zp = xin[f][k], zm = sm[f * L + pm];
                xv[f] = make_float2(0.5f * (zp.x + zm.x), 0.5f * (zp.y - zm.y));
                xb[f] = make_float2(0.5f * (zp.y + zm.y), -0.5f * (zp.x - zm.x));
            }
            spec_apply<OP>(a.P, k1o, 0.f, k1 * k1, xv, yv, eacc, 1.f);
            spec_apply<OP>(a.P, k1o, 0.f, k1 * k1 + kny2 * kny2, xb, yb, eacc, 1.f);
#pragma unroll
            for (int o = 0; o < NOUT; ++o) yv[o] = make_float2(yv[o].x - yb[o].y, yv[o].y + yb[o].x);
        }
#pragma unroll
        for (int o = 0; o < NOUT; ++o) y[o][k] = yv[o];
    }
    if (OP == OP_ENERGY || OP == OP_QNORM || OP == OP_ENERGY_Y) {
        const double s = block_reduce<0>(eacc);
        if (threadIdx.x == 0) a.part[blockIdx.x] = s * a.P.escale;
        return;
    }
#pragma unroll
    for (int o = 0; o < NOUT; ++o) {
        __syncthreads();
        reg_fft<LOGL, true>(y[o], t, true, X + 2 * c * fft_buf(L), X + 2 * c * fft_buf(L) + fft_buf(L), tw);
#pragma unroll
        for (int k = 0; k < 8; ++k) A[c * L + t + k * T] = y[o][k];
        __syncthreads();
        float2* dst = a.out[o];
        const float cd2 = 1.0f / (float)a.n2;
        for (int idx = threadIdx.x; idx < C * L; idx += blockDim.x) {
            const int g = idx >> g_shift;
            const int rem = idx & g_mask;
            const int cc = rem >> 2, rr = rem & 3;
            const size_t gi = ((size_t)g * W + e0 + cc) * 4 + rr;
            float2 val = A[cc * L + 4 * g + rr];
            if (OP == OP_DIV1) {
                // + (i k2~ / n2) F2, diagonal in the row spectra; k2~ = 0 in the packed column 0
                const float2 f2 = B2[cc * L + 4 * g + rr];
                const float ce = cd2 * (float)(e0 + cc);
                val = make_float2(val.x - ce * f2.y, val.y + ce * f2.x);
            }
            dst[gi] = val;
        }
    }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
// Default tile choices.  R rows per row CTA: a multiple of 4 with at least 64
// threads (T = L/8 per row); C spectrum columns per column CTA: at least 2
// (64-byte segments) and 64 threads.  reg_autotune may replace both per grid.
void default_tiles(int n1, int n2, int* R_out, int* C_out, int* P_out) {
    if (P_out) *P_out = n2 <= 512 ? 1 : 0;
    int R = 4;
    while (R * (n2 / 8) < 64 && R * 2 <= n1) R *= 2;
    const int W = n2 / 2;
    int C = 2;
    while (C * (n1 / 8) < 64 && C * 2 <= W) C *= 2;
    *R_out = R;
    *C_out = C > W ? W : C;
}

// Shared memory of a row kernel with R rows of length L (staging: R L; exchange: two padded
// buffers per transform, at most R transforms) and of the column kernel with C columns of
// length L (staging C L, two padded buffers per column, and C L more for OP_DIV1).
size_t row_smem(int R, int L) { return ((size_t)R * L + 2 * (size_t)R * fft_buf(L)) * sizeof(float2); }
size_t col_smem(int C, int L, bool div1) {
    return ((size_t)C * L * (div1 ? 2 : 1) + 2 * (size_t)C * fft_buf(L)) * sizeof(float2);
}

// Launch limits of the row kernels (32 to 512 threads; 2 CTAs per SM for
// 1024-point rows) and the column kernel (32 to 256 threads), and 227 KB of
// shared memory.
bool tiles_valid(int n1, int n2, int R, int C, int P) {
    const size_t smax = 227 * 1024;
    if (P != 0 && (P != 1 || n2 > 512)) return false;
    const int W = n2 / 2;
    if (R < 4 || (R & 3) || R > n1 || (n1 % R)) return false;
    if (R * (n2 / 8) < 32 || R * (n2 / 8) > 512 || row_smem(R, n2) > smax) return false;
    if (C < 2 || (C & (C - 1)) || C > W || (W % C)) return false;
    if (C * (n1 / 8) < 32 || C * (n1 / 8) > 256 || col_smem(C, n1, true) > smax) return false;
    return true;
}

static int rows_per_cta(const reg_ctx* ctx) {
    int R, C, P;
    default_tiles(ctx->n1, ctx->n2, &R, &C, &P);
    return ctx->tileR > 0 ? ctx->tileR : R;
}

static int cols_per_cta(const reg_ctx* ctx) {
    int R, C, P;
    default_tiles(ctx->n1, ctx->n2, &R, &C, &P);
    return ctx->tileC > 0 ? ctx->tileC : C;
}

static bool prefetch_rows(const reg_ctx* ctx) {
    int R, C, P;
    default_tiles(ctx->n1, ctx->n2, &R, &C, &P);
    return (ctx->tileR > 0 ? ctx->tileP : P) != 0;
}

// Opt in to more than 48 KB of dynamic shared memory once per (device, kernel instantiation)
// and size: the attribute applies to the current device only (contexts on several host
// threads launch concurrently, hence the lock).
struct SmemKey {
    int dev;
    const void* kern;
    bool operator==(const SmemKey& o) const { return dev == o.dev && kern == o.kern; }
};
struct SmemKeyHash {
    size_t operator()(const SmemKey& k) const { return std::hash<const void*>()(k.kern) * 31u + (size_t)k.dev; }
};
template <typename K>
static void set_smem(K kern, size_t bytes) {
    if (bytes <= 32 * 1024) return;  // static shared memory (reductions) also counts toward the 48 KB default
    static std::mutex mu;
    static std::unordered_map<SmemKey, size_t, SmemKeyHash> done;
    int dev = 0;
    cudaGetDevice(&dev);
    const SmemKey key{dev, (const void*)kern};
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done[key] = bytes;
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

struct RowCfg { int R, threads; size_t smem; int grid; bool pre; };
static RowCfg row_cfg(reg_ctx* ctx) {
    RowCfg c;
    const int L = ctx->n2;
    c.R = rows_per_cta(ctx);
    c.pre = prefetch_rows(ctx);
    c.threads = c.R * (L / 8);
    c.smem = row_smem(c.R, L);
    c.grid = ctx->n1 / c.R;
    return c;
}

void launch_r2c_scalar(reg_ctx* ctx, const float* f, float2* S) {
    const RowCfg g = row_cfg(ctx);
    ktimer_begin(ctx, KC_ROW, 8.0 * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_r2c<LG, false>;
        set_smem(kern, g.smem);
        launch_k(ctx, kern, g.grid, g.threads, g.smem, f, nullptr, S, nullptr, g.R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_r2c_vec(reg_ctx* ctx, const float* u1, const float* u2, float2* S1, float2* S2) {
    const RowCfg g = row_cfg(ctx);
    ktimer_begin(ctx, KC_ROW, 16.0 * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_r2c<LG, true>;
        set_smem(kern, g.smem);
        launch_k(ctx, kern, g.grid, g.threads, g.smem, u1, u2, S1, S2, g.R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_c2r_scalar(reg_ctx* ctx, const float2* S, float* f) {
    const RowCfg g = row_cfg(ctx);
    ktimer_begin(ctx, KC_ROW, 8.0 * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_c2r<LG, false>;
        set_smem(kern, g.smem);
        launch_k(ctx, kern, g.grid, g.threads, g.smem, S, nullptr, f, nullptr, g.R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_c2r_vec(reg_ctx* ctx, const float2* S1, const float2* S2, float* u1, float* u2) {
    const RowCfg g = row_cfg(ctx);
    ktimer_begin(ctx, KC_ROW, 16.0 * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_c2r<LG, true>;
        set_smem(kern, g.smem);
        launch_k(ctx, kern, g.grid, g.threads, g.smem, S1, S2, u1, u2, g.R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_row_adv(reg_ctx* ctx, const AdvArgs& a) {
    const RowCfg g = row_cfg(ctx);
    // floats per node read/written: G 2 (complex half spectra = 1 float per node each), u_j 1,
    // u* 1 (stage 2), v 2, source gm + v~ 4, u_out 1, grad_out 2, S_out 1
    double fl = 1 + 2 + 1 + (a.G1 ? 2 : 0) + (a.stage == 2 ? 1 : 0) + (a.gm ? 4 : 0) + (a.grad_out ? 2 : 0) +
                (a.S_out ? 1 : 0);
    ktimer_begin(ctx, KC_ROWSTAGE, 4.0 * fl * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = (g.pre && LG <= 9) ? k_row_adv<LG, (LG <= 9)> : k_row_adv<LG, false>;
        set_smem(kern, g.smem);
        launch_k(ctx, kern, g.grid, g.threads, g.smem, a, ctx->N, g.R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_row_adj(reg_ctx* ctx, const AdjArgs& a) {
    const RowCfg g = row_cfg(ctx);
    // D 1, lam_j 1, lam* 1 (stage 2), v 2, l_out 1, body force b read+write 4 and gm 2, flux spectra 2;
    // full Newton: lam_src 1, v~ 2, grad m~ 2 (stage 2)
    double fl = 1 + 1 + 2 + 1 + (a.stage == 2 ? 1 : 0) + (a.b ? 6 : 0) + (a.F1 ? 2 : 0) +
                (a.lsrc ? 3 + (a.b ? 2 : 0) : 0);
    ktimer_begin(ctx, KC_ROWSTAGE, 4.0 * fl * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = a.lsrc ? k_row_adj<LG, false, true>
                           : ((g.pre && LG <= 9) ? k_row_adj<LG, (LG <= 9), false> : k_row_adj<LG, false, false>);
        set_smem(kern, g.smem);
        launch_k(ctx, kern, g.grid, g.threads, g.smem, a, ctx->N, g.R, ctx->tw);
    });
    ktimer_end(ctx);
}

void launch_adj_init(reg_ctx* ctx, const float* a, float ca, const float* c, float cb, const float* v, float* lam,
                     float* b, const float* gm, float w, float2* F1, float2* F2, double* part, const float* lsrc,
                     const float* vt, const float* gmt) {
    const RowCfg g = row_cfg(ctx);
    // a 1 (optional), c 1, v 2, lam 1, b 2 + gm 2, flux spectra 2; full Newton: lsrc 1, v~ 2, grad m~ 2
    ktimer_begin(ctx, KC_ROW, 4.0 * ((a ? 1 : 0) + 1 + 2 + 1 + 4 + 2 + (lsrc ? 5 : 0)) * ctx->N);
    DISPATCH_LOG(ctx->log2, {
        auto kern = k_adj_init<LG>;
        set_smem(kern, g.smem);
        launch_k(ctx, kern, g.grid, g.threads, g.smem, a, ca, c, cb, v, lam, b, gm, w, F1, F2, part, ctx->N, g.R,
                 ctx->tw, lsrc, vt, gmt);
    });
    ktimer_end(ctx);
}

int row_blocks(reg_ctx* ctx) { return row_cfg(ctx).grid; }

template <int NIN, int NOUT, int OP>
static void launch_col_t(reg_ctx* ctx, const float2* const* in, float2* const* out, const SpecParams& P,
                         double* part) {
    const int L = ctx->n1, W = ctx->n2 / 2;
    const int cpb = cols_per_cta(ctx);
    const size_t smem = col_smem(cpb, L, OP == OP_DIV1);
    ColArgs a;
    for (int f = 0; f < 5; ++f) a.in[f] = (f < NIN) ? in[f] : nullptr;
    if (OP == OP_DIV1) a.in[1] = in[1];  // read untransformed in the store phase
    for (int o = 0; o < 2; ++o) a.out[o] = (o < NOUT) ? out[o] : nullptr;
    a.P = P;
    a.part = part;
    a.cpb = cpb;
    a.lcpb = 0;
    while ((1 << a.lcpb) < cpb) ++a.lcpb;
    a.n2 = ctx->n2;
    ktimer_begin(ctx, KC_COL, 4.0 * (NIN + NOUT + (OP == OP_DIV1 ? 1 : 0)) * ctx->N);
    DISPATCH_LOG(ctx->log1, {
        auto kern = k_col<LG, NIN, NOUT, OP>;
        set_smem(kern, smem);
        launch_k(ctx, kern, W / cpb, cpb * (L / 8), smem, a, ctx->tw);
    });
    ktimer_end(ctx);
}

int col_blocks(reg_ctx* ctx) { return (ctx->n2 / 2) / cols_per_cta(ctx); }

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
        case OP_GRAD1: launch_col_t<1, 1, OP_GRAD1>(ctx, in, out, P, part); break;
        case OP_DIV1: launch_col_t<1, 1, OP_DIV1>(ctx, in, out, P, part); break;
        case OP_SMOOTH_PROJ: launch_col_t<2, 2, OP_SMOOTH_PROJ>(ctx, in, out, P, part); break;
        case OP_SMOOTH: launch_col_t<1, 1, OP_SMOOTH>(ctx, in, out, P, part); break;
        case OP_MASSP: launch_col_t<2, 2, OP_MASSP>(ctx, in, out, P, part); break;
        case OP_QINV: launch_col_t<2, 2, OP_QINV>(ctx, in, out, P, part); break;
        case OP_QMUL: launch_col_t<2, 2, OP_QMUL>(ctx, in, out, P, part); break;
        case OP_ASSEMBLE_Y: launch_col_t<4, 2, OP_ASSEMBLE_Y>(ctx, in, out, P, part); break;
        case OP_QNORM: launch_col_t<2, 0, OP_QNORM>(ctx, in, out, P, part); break;
        case OP_ENERGY_Y: launch_col_t<2, 0, OP_ENERGY_Y>(ctx, in, out, P, part); break;
        default: break;
    }
}

// ---------------------------------------------------------------------------
// pointwise and reduction kernels
// ---------------------------------------------------------------------------
__global__ void k_dot_partial(const float* __restrict__ x, const float* __restrict__ y, long long n, double* part) {
    pdl_entry();
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)x[i] * (double)y[i];
    const double s = block_reduce<0>(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

int launch_dot_partial(reg_ctx* ctx, const float* x, const float* y, long long n, double* part) {
    ktimer_begin(ctx, KC_POINT, 8.0 * n);
    launch_k(ctx, k_dot_partial, NBLK_RED, NTHREADS, 0, x, y, n, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

__global__ void k_sum_partial(const float* __restrict__ x, long long n, double* part) {
    pdl_entry();
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)x[i];
    const double s = block_reduce<0>(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

int launch_sum_partial(reg_ctx* ctx, const float* x, long long n, double* part) {
    ktimer_begin(ctx, KC_POINT, 4.0 * n);
    launch_k(ctx, k_sum_partial, NBLK_RED, NTHREADS, 0, x, n, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

__global__ void k_maxnorm_partial(const float* __restrict__ v, int N, double* part) {
    pdl_entry();
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
    launch_k(ctx, k_maxnorm_partial, NBLK_RED, NTHREADS, 0, v, N, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

template <int OPR>
__global__ void k_finalize(const double* __restrict__ part, int np, double* out, double scale, int accumulate) {
    pdl_entry();
    double acc = (OPR == 0) ? 0.0 : part[0];
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc = red_op<OPR>(acc, part[i]);
    const double s = block_reduce<OPR>(acc);
    if (threadIdx.x == 0) *out = scale * s + (accumulate ? *out : 0.0);
}

void launch_finalize(reg_ctx* ctx, const double* part, int np, double* out, double scale, int accumulate, int op) {
    ktimer_begin(ctx, KC_POINT, 8.0 * np);
    if (op == 0) launch_k(ctx, k_finalize<0>, 1, NTHREADS, 0, part, np, out, scale, accumulate);
    else if (op == 1) launch_k(ctx, k_finalize<1>, 1, NTHREADS, 0, part, np, out, scale, accumulate);
    else launch_k(ctx, k_finalize<2>, 1, NTHREADS, 0, part, np, out, scale, accumulate);
    ktimer_end(ctx);
}

__global__ void k_axpby(long long n, float a, const float* __restrict__ x, float b, const float* y, float* out,
                        const double* __restrict__ scal, int num, int den) {
    pdl_entry();
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
    launch_k(ctx, k_axpby, NBLK_RED, NTHREADS, 0, n, a, x, b, y, out ? out : y, ctx->d_scal, num, den);
    ktimer_end(ctx);
}

__global__ void k_pcg_update(long long n, float* vt, const float* __restrict__ s, float* r, const float* __restrict__ Hs,
                             const double* __restrict__ scal, double* part) {
    pdl_entry();
    const double shs = scal[SL_SHS];
    const float kappa = (float)(scal[SL_RZ] / shs);
    double acc = 0.0;
    if (!(shs > 0.0)) {  // non-positive curvature: leave vt and r unchanged (the host stops PCG)
        if (threadIdx.x == 0) part[blockIdx.x] = 0.0;
        return;
    }
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
    launch_k(ctx, k_pcg_update, NBLK_RED, NTHREADS, 0, n, vt, s, r, Hs, ctx->d_scal, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

__global__ void k_pcg_dir(long long n, const float* __restrict__ z, float* s, const double* __restrict__ scal) {
    pdl_entry();
    const float mu = (float)(scal[SL_RZNEW] / scal[SL_RZ]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s[i] = fmaf(mu, s[i], z[i]);
}

void launch_pcg_dir(reg_ctx* ctx, long long n, const float* z, float* s) {
    ktimer_begin(ctx, KC_POINT, 4.0 * n * 3);
    launch_k(ctx, k_pcg_dir, NBLK_RED, NTHREADS, 0, n, z, s, ctx->d_scal);
    ktimer_end(ctx);
}

__global__ void k_fill(long long n, float* y, float val) {
    pdl_entry();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = val;
}

void launch_fill(reg_ctx* ctx, long long n, float* y, float val) {
    ktimer_begin(ctx, KC_POINT, 4.0 * n);
    launch_k(ctx, k_fill, NBLK_RED, NTHREADS, 0, n, y, val);
    ktimer_end(ctx);
}

// counts for the label overlap measures (App. F): nodes with f > thr (transported template
// labels), with L > 0.5 (reference labels) and with both
__global__ void k_overlap_counts(int N, const float* __restrict__ f, const float* __restrict__ L, float thr,
                                 double* part) {
    pdl_entry();
    double nT = 0.0, nR = 0.0, nB = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const bool t = f[i] > thr, r = L[i] > 0.5f;
        nT += t ? 1.0 : 0.0;
        nR += r ? 1.0 : 0.0;
        nB += (t && r) ? 1.0 : 0.0;
    }
    double c;
    c = block_reduce<0>(nT);
    if (threadIdx.x == 0) part[0 * gridDim.x + blockIdx.x] = c;
    c = block_reduce<0>(nR);
    if (threadIdx.x == 0) part[1 * gridDim.x + blockIdx.x] = c;
    c = block_reduce<0>(nB);
    if (threadIdx.x == 0) part[2 * gridDim.x + blockIdx.x] = c;
}

int launch_overlap_counts(reg_ctx* ctx, const float* f, const float* L, float thr, double* part) {
    ktimer_begin(ctx, KC_POINT, 8.0 * ctx->N);
    launch_k(ctx, k_overlap_counts, NBLK_RED, NTHREADS, 0, ctx->N, f, L, thr, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

// deformation gradient stage (Eq. (e:def-grad)); F planes (F11, F12, F21, F22),
// gF planes (d1 F11, d2 F11, d1 F12, d2 F12, ...), gv planes (d1 v1, d2 v1, d1 v2, d2 v2)
__global__ void k_defgrad_stage(int N, int stage, const float* __restrict__ F, const float* __restrict__ Fs,
                                const float* __restrict__ gF, const float* __restrict__ gv,
                                const float* __restrict__ v, float h, float* out) {
    pdl_entry();
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
    launch_k(ctx, k_defgrad_stage, NBLK_RED, NTHREADS, 0, ctx->N, stage, F, Fs, gF, gv, v, h, out);
    ktimer_end(ctx);
}

__global__ void k_det_stats(int N, const float* __restrict__ F, float* detF, double* part) {
    pdl_entry();
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
    launch_k(ctx, k_det_stats, NBLK_RED, NTHREADS, 0, ctx->N, F, detF, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

// shear control: strain rate, viscosity, stress (Eqs. (e:shear-control-reg-v), (e:1st-var-reg-v-nls))
#define SHEAR_EPS2 1.0e-6f
__global__ void k_shear_strain(int N, const float* __restrict__ gv, float nu, float* E, float* eta, float* T,
                               double* part) {
    pdl_entry();
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
    launch_k(ctx, k_shear_strain, NBLK_RED, NTHREADS, 0, ctx->N, gv, nu, E, eta, T, part);
    ktimer_end(ctx);
    return NBLK_RED;
}

__global__ void k_shear_second(int N, const float* __restrict__ gvt, const float* __restrict__ E,
                               const float* __restrict__ eta, float nu, float* T) {
    pdl_entry();
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
    launch_k(ctx, k_shear_second, NBLK_RED, NTHREADS, 0, ctx->N, gvt, E, eta, nu, T);
    ktimer_end(ctx);
}
