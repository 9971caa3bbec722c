// Transport solves resident in one thread-block cluster (sm_103a): the state
// solve (Eq. (e:state-eq-elim)), the adjoint solve with the body force
// (Eq. (e:adj-eq-elim), Sec. 3.1), and the Gauss-Newton matvec's incremental
// state and incremental adjoint solves (Eqs. (e:inc-state-eq-elim),
// (e:inc-adj-eq-elim) without the lambda terms, Sec. 4), each over all nt
// Heun steps in ONE launch.
//
// Data split.  An n x n grid (n = 2^LG, 16 <= n <= 512) is owned by a cluster
// of CS = max(1, n^2 / 16384) CTAs.  CTA r owns the R = n / CS consecutive
// grid rows r R .. r R + R - 1 and keeps their packed half spectra along x^2
// (R x n/2 complex = 64 KB at n >= 128) in shared memory for the whole solve;
// in the column phase it owns the C = (n/2) / CS spectrum columns
// r C .. r C + C - 1.  One RK2 stage is
//   column phase: gather the owned columns from every CTA of the cluster
//                 (distributed shared memory), FFT along x^1, multiply by
//                 i k1~ / n^2, inverse FFT, scatter back to the owners;
//   cluster barrier;
//   row phase:    per owned row, form the x^1 and x^2 derivatives (the x^2
//                 one is diagonal in the row spectrum), inverse FFT along x^2,
//                 the pointwise Heun stage with operands from global memory
//                 (v, v~, grad m, u_j), forward FFT of the result into the
//                 CTA's spectra;
//   cluster barrier.
// Spectra never leave the SMs; global memory carries the per-node operands
// and the solution history only.  The FFTs are the register-resident radix-8
// Stockham transforms of fft_reg.cuh, run in place in one shared-memory
// buffer per transform (an extra barrier per pass instead of a second
// buffer), with the twiddle table staged in shared memory.
//
// Synchronization: only __syncthreads and hardware cluster barriers
// (barrier.cluster arrive/wait through cooperative_groups); every CTA of a
// cluster executes the same sequence of barriers.  No spin loops.
#include <cooperative_groups.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "fft.cuh"
#include "fft_reg.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

constexpr int TC_THREADS = 512;


// ---------------------------------------------------------------------------
// in-place register FFT: the algorithm of reg_fft (fft_reg.cuh) with one
// exchange buffer of L + L/8 entries (padded indices, fft_pad).  On entry
// thread t holds x[k] = in[t + k T]; on exit x[k] = out[t + k T].  Every thread of the CTA calls it (it contains
// __syncthreads).  The caller must __syncthreads before the first call if buf
// still holds data other threads are reading, and after it before writing buf.
// ---------------------------------------------------------------------------
// The per-pass twiddle table of the transform length (fft.cuh layout: the threads of a warp
// read consecutive entries) is staged in shared memory once per launch.
template <int LOGL>
__device__ void tw_stage(float2* twp, const float2* __restrict__ tw_global) {
    for (int idx = threadIdx.x; idx < tw_entries(LOGL); idx += TC_THREADS) twp[idx] = tw_global[twp_base(LOGL) + idx];
}

template <int LOGL, bool INV>
__device__ __forceinline__ float2 tw_s(const float2* twp, int i, int k, int p) {
    float2 w = twp[tw_off(LOGL, i) + (k - 1) * tw_groups(LOGL, i) + p];
    if (INV) w.y = -w.y;
    return w;
}

template <int LG>
struct TcGeom {
    static constexpr int n = 1 << LG;         // grid points per direction
    static constexpr int W = n / 2;           // packed half-spectrum entries per row
    static constexpr int N = n * n;
    static constexpr int LOGCS = (2 * LG > 14) ? 2 * LG - 14 : 0;
    static constexpr int CS = 1 << LOGCS;     // CTAs per cluster
    static constexpr int R = n / CS;          // grid rows per CTA
    static constexpr int C = W / CS;          // spectrum columns per CTA
    static constexpr int T = n / 8;           // threads per length-n transform
    static constexpr int Q = TC_THREADS / T;  // transforms per CTA at once
    static constexpr int QR = Q < R ? Q : R;  // rows per row-phase round
    static constexpr int QC = Q < C ? Q : C;  // columns per column-phase round
    static constexpr int RW = R * W;          // complex entries of one spectra buffer
    static constexpr int SLOT = fft_buf(n);   // one transform's exchange buffer (padded, see fft_pad)
    static constexpr int GCOL = SLOT + 1;     // column stride of the column buffer
    static constexpr int OROW = QR * SLOT;    // row phase: offset of the real-valued staging rows
    static constexpr int ROWX = OROW + QR * n / 2;
    static constexpr int GX = (C * GCOL > ROWX) ? C * GCOL : ROWX;
    static constexpr int TWE = (tw_entries(LG) + 1) & ~1;  // per-pass twiddle table (even: 16-byte alignment)
    static constexpr size_t SMEM = (size_t)(TWE + 2 * RW + GX) * sizeof(float2);
    static_assert(CS <= 16, "a cluster has at most 16 CTAs");
    static_assert(R % QR == 0 && C % QC == 0 && QR % 2 == 0 && C % 2 == 0, "tiling");
    static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
};

template <int LOGL, bool INV>
__device__ __forceinline__ void fft_ip(float2 (&x)[8], int t, bool active, float2* buf, const float2* tws) {
    constexpr int L = 1 << LOGL;
    constexpr int T = L >> 3;
    constexpr int NP8 = LOGL / 3;
    constexpr int REM = LOGL - 3 * NP8;
#pragma unroll
    for (int i = 0; i < NP8; ++i) {
        const int ls = 3 * i;
        const int s = 1 << ls;
        const int q = t & (s - 1);
        const int p = t >> ls;
        const int m = L >> (ls + 3);
        const bool last = (i == NP8 - 1) && (REM == 0);
        if (i > 0) {
            if (active) {
#pragma unroll
                for (int k = 0; k < 8; ++k) x[k] = buf[fft_pad(q + s * (p + k * m))];
            }
            __syncthreads();
        }
        if (active) dft8<INV>(x);
        if (!last) {
            if (active) {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    buf[fft_pad(q + s * (8 * p + k))] = (k == 0) ? x[k] : cmul(x[k], tw_s<LOGL, INV>(tws, i, k, p));
            }
            __syncthreads();
        }
    }
    if (REM == 1) {
        if (active) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 a = buf[fft_pad(t + j * T)], b = buf[fft_pad(t + j * T + 4 * T)];
                x[j] = cadd(a, b);
                x[j + 4] = csub(a, b);
            }
        }
    } else if (REM == 2) {
        if (active) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int q = t + j * T;
                const float2 a0 = buf[fft_pad(q)], a1 = buf[fft_pad(q + 2 * T)], a2 = buf[fft_pad(q + 4 * T)],
                             a3 = buf[fft_pad(q + 6 * T)];
                const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3),
                             t3 = mul_mi<INV>(csub(a1, a3));
                x[j] = cadd(t0, t2);
                x[j + 2] = cadd(t1, t3);
                x[j + 4] = csub(t0, t2);
                x[j + 6] = csub(t1, t3);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// packed half spectra in row-major order: row r, entry e at r * W + e; entry 0
// holds (X_0, X_{L/2}) of the real row (both real).
// ---------------------------------------------------------------------------
// Z[e] of z = a + i b for real rows a, b given by their packed half spectra.
template <int LOGL>
__device__ __forceinline__ float2 zmerge(float2 A0, float2 Ae, float2 B0, float2 Be, int e) {
    constexpr int L = 1 << LOGL, H = L >> 1;
    if (e == 0) return make_float2(A0.x, B0.x);
    if (e == H) return make_float2(A0.y, B0.y);
    return (e < H) ? make_float2(Ae.x - Be.y, Ae.y + Be.x) : make_float2(Ae.x + Be.y, -Ae.y + Be.x);
}

// grad u from D (x^1-derivative spectrum row) and S (row spectrum of u):
// Z = D + i (i k2~ / n) S, whose inverse transform is (d1 u, d2 u).
template <int LOGL>
__device__ __forceinline__ float2 zgrad(const float2* D, const float2* S, int e, float c) {
    constexpr int L = 1 << LOGL, H = L >> 1;
    const int ee = (e < H) ? e : ((e == H) ? 0 : L - e);  // e = H reads nothing beyond entry 0
    const float2 s = S[ee];
    const float ce = (e == 0 || e == H) ? 0.f : c * (float)ee;
    return zmerge<LOGL>(D[0], D[ee], make_float2(0.f, 0.f), make_float2(-ce * s.y, ce * s.x), e);
}

// div of a flux for two rows a, b: per row Dx = D1x + (i k2~ / n) F2x (the x^1 part
// transformed in the column phase, the x^2 part diagonal), merged as Da + i Db.
template <int LOGL>
__device__ __forceinline__ float2 zdiv(const float2* D1a, const float2* F2a, const float2* D1b, const float2* F2b,
                                       int e, float c) {
    constexpr int L = 1 << LOGL, H = L >> 1;
    const int ee = (e < H) ? e : ((e == H) ? 0 : L - e);  // e = H reads nothing beyond entry 0
    const float ce = (e == 0 || e == H) ? 0.f : c * (float)ee;
    const float2 fa = F2a[ee], fb = F2b[ee];
    const float2 da = make_float2(D1a[ee].x - ce * fa.y, D1a[ee].y + ce * fa.x);
    const float2 db = make_float2(D1b[ee].x - ce * fb.y, D1b[ee].y + ce * fb.x);
    return zmerge<LOGL>(D1a[0], da, D1b[0], db, e);
}

// packed entry e of the real part (part 0) or imaginary part (part 1) of z from Z (natural order)
template <int LOGL>
__device__ __forceinline__ float2 zsplit(const float2* Z, int part, int e) {
    constexpr int L = 1 << LOGL, H = L >> 1;
    if (e == 0) {
        const float2 z0 = Z[0], zh = Z[H];
        return part == 0 ? make_float2(z0.x, zh.x) : make_float2(z0.y, zh.y);
    }
    const float2 zk = Z[e], zm = Z[L - e];
    return part == 0 ? make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y))
                     : make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
}

// ---------------------------------------------------------------------------
// column phase
// ---------------------------------------------------------------------------
// The CTA of rank `rank` gathers spectrum columns e0 .. e0 + C - 1 (all n rows)
// from buffer `src` of every CTA of the cluster, transforms them along x^1,
// multiplies by i k1~ / n^2 (k1~: Nyquist set to 0), transforms back and
// scatters the result into buffer `dst` of the row owners.  With ALIAS
// (dst == src) a cluster barrier separates the gather from the scatter.  Ends
// with a cluster barrier: on return every CTA's dst holds the x^1-derivative
// spectra of its rows.  The multiplier is the same complex number for both
// real fields packed in column 0, so that column needs no unpacking.
template <int LG, bool ALIAS>
__device__ void col_phase(cg::cluster_group& cl, int rank, float2* src, float2* dst, float2* X, const float2* tws,
                          float scale) {
    using G = TcGeom<LG>;
    constexpr int n = G::n, W = G::W, R = G::R, C = G::C, T = G::T, CP = C / 2;
    constexpr int ITER = (n * CP + TC_THREADS - 1) / TC_THREADS;
    const int e0 = rank * C;
    constexpr int GB = ITER < 4 ? ITER : 4;  // remote loads in flight per thread
#pragma unroll
    for (int i0 = 0; i0 < ITER; i0 += GB) {
        float4 val[GB];
#pragma unroll
        for (int it = 0; it < GB; ++it) {
            const int idx = threadIdx.x + (i0 + it) * TC_THREADS;
            if (i0 + it < ITER && idx < n * CP) {
                const int row = idx / CP, cp = idx - row * CP;
                const int p = row / R, r = row - p * R;
                const float2* srcp = cl.map_shared_rank(src, p);
                val[it] = *reinterpret_cast<const float4*>(srcp + r * W + e0 + 2 * cp);
            }
        }
#pragma unroll
        for (int it = 0; it < GB; ++it) {
            const int idx = threadIdx.x + (i0 + it) * TC_THREADS;
            if (i0 + it < ITER && idx < n * CP) {
                const int row = idx / CP, cp = idx - row * CP;
                X[(2 * cp) * G::GCOL + row] = make_float2(val[it].x, val[it].y);
                X[(2 * cp + 1) * G::GCOL + row] = make_float2(val[it].z, val[it].w);
            }
        }
    }
    __syncthreads();
    const int q = threadIdx.x / T, t = threadIdx.x - q * T;
    const bool active = q < G::QC;
#pragma unroll 1
    for (int c0 = 0; c0 < C; c0 += G::QC) {
        float2* col = X + (c0 + (active ? q : 0)) * G::GCOL;
        float2 x[8];
        if (active) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = col[t + k * T];
        }
        __syncthreads();
        fft_ip<LG, false>(x, t, active, col, tws);
        if (active) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int pk = t + k * T;
                const float k1 = (pk == n / 2) ? 0.f : (float)(pk < n / 2 ? pk : pk - n);
                x[k] = cscale(cmuli(x[k]), k1 * scale);
            }
        }
        __syncthreads();
        fft_ip<LG, true>(x, t, active, col, tws);
        __syncthreads();
        if (active) {
#pragma unroll
            for (int k = 0; k < 8; ++k) col[t + k * T] = x[k];
        }
    }
    __syncthreads();
    if (ALIAS) cl.sync();  // every CTA has gathered from src before it is overwritten
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int idx = threadIdx.x + it * TC_THREADS;
        if (idx < n * CP) {
            const int row = idx / CP, cp = idx - row * CP;
            const int p = row / R, r = row - p * R;
            float2* dstp = cl.map_shared_rank(dst, p);
            const float2 lo = X[(2 * cp) * G::GCOL + row], hi = X[(2 * cp + 1) * G::GCOL + row];
            *reinterpret_cast<float4*>(dstp + r * W + e0 + 2 * cp) = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
    }
    cl.sync();
}

// ---------------------------------------------------------------------------
// row phase, advection (state / incremental state), Heun stage:
//   k = -v . grad u_s - v~ . grad m(t)   (source only with gm)
//   stage 1: u* = u_j + h k ; stage 2: u_{j+1} = (u_j + u* + h k) / 2
// U: row spectra of u_s (in) and of the stage result (out, if want_spec);
// V: x^1-derivative spectra of u_s.
// ---------------------------------------------------------------------------
enum { ADV_STAGE = 0, ADV_INIT = 1, ADV_GRAD_ONLY = 2 };

struct AdvRow {
    int kind;             // ADV_STAGE, ADV_INIT (result = init, no derivative), ADV_GRAD_ONLY (grad_out only)
    int stage;            // 1 or 2
    bool zero_grad;       // u_s = 0 (incremental state at t = 0): no transform
    bool want_spec;       // write the result's row spectrum into U
    const float* init;    // ADV_INIT: the field whose spectrum starts the solve
    const float* uj;      // nullptr: u_j = 0
    const float* us;      // stage 2: u*
    float* out;           // nullable: stage result (global)
    float* grad_out;      // nullable: grad u_s (2 planes)
    const float* gm;      // nullable: grad m at the source time (incremental state)
};

template <int LG>
__device__ void adv_rows(int rank, const TcArgs& a, const AdvRow& s, float2* U, const float2* V, float2* X,
                         const float2* tws) {
    using G = TcGeom<LG>;
    constexpr int n = G::n, W = G::W, R = G::R, T = G::T, QR = G::QR, N = G::N;
    const int q = threadIdx.x / T, t = threadIdx.x - q * T;
    const bool act = q < QR;
    const float cd2 = 1.0f / (float)n;
#pragma unroll 1
    for (int r0 = 0; r0 < R; r0 += QR) {
        const int r = r0 + (act ? q : 0);
        const size_t rowbase = (size_t)(rank * R + r) * n;
        float2 x[8];
        // the stage results of the round's rows go to the staging rows O (real values) for the
        // forward transforms; O is last read before the previous round's closing barriers
        float* O = reinterpret_cast<float*>(X + G::OROW);
        if (s.kind == ADV_INIT) {
            if (act) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const size_t idx = rowbase + t + k * T;
                    const float o = s.init[idx];
                    if (s.out) s.out[idx] = o;
                    O[q * n + t + k * T] = o;
                }
            }
        } else {
            if (!s.zero_grad) {
                if (act) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) x[k] = zgrad<LG>(V + r * W, U + r * W, t + k * T, cd2);
                }
                fft_ip<LG, true>(x, t, act, X + (act ? q : 0) * G::SLOT, tws);
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) x[k] = make_float2(0.f, 0.f);
            }
            // operands loaded four elements at a time after the transform (keeps the register
            // count within the 128 of a 512-thread CTA)
            if (act) {
#pragma unroll
                for (int k0 = 0; k0 < 8; k0 += 4) {
                    float pv1[4], pv2[4], puj[4], pus[4], psrc[4];
                    if (s.kind == ADV_STAGE) {
#pragma unroll
                        for (int k = k0; k < k0 + 4; ++k) {
                            const size_t idx = rowbase + t + k * T;
                            pv1[k - k0] = a.v[idx];
                            pv2[k - k0] = a.v[N + idx];
                            puj[k - k0] = s.uj ? s.uj[idx] : 0.f;
                            pus[k - k0] = (s.stage == 2) ? s.us[idx] : 0.f;
                            psrc[k - k0] = s.gm ? -(a.vt[idx] * s.gm[idx] + a.vt[N + idx] * s.gm[N + idx]) : 0.f;
                        }
                    }
#pragma unroll
                    for (int k = k0; k < k0 + 4; ++k) {
                        const size_t idx = rowbase + t + k * T;
                        const float d1 = x[k].x, d2 = x[k].y;
                        if (s.grad_out) {
                            s.grad_out[idx] = d1;
                            s.grad_out[N + idx] = d2;
                        }
                        if (s.kind == ADV_STAGE) {
                            const float kk = psrc[k - k0] - (pv1[k - k0] * d1 + pv2[k - k0] * d2);
                            const float o = (s.stage == 1) ? fmaf(a.h, kk, puj[k - k0])
                                                           : 0.5f * (puj[k - k0] + pus[k - k0] + a.h * kk);
                            s.out[idx] = o;
                            O[q * n + t + k * T] = o;
                        }
                    }
                }
            }
        }
        __syncthreads();  // the inverse transform's last reads of X are done
        if (!s.want_spec) continue;
        // forward real transforms of the round's rows, two rows per complex transform
        const bool act2 = q < QR / 2;
        float2* slot = X + (act2 ? q : 0) * G::SLOT;
        if (act2) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int e = t + k * T;
                x[k] = make_float2(O[2 * q * n + e], O[(2 * q + 1) * n + e]);
            }
        }
        fft_ip<LG, false>(x, t, act2, slot, tws);
        __syncthreads();
        if (act2) {
#pragma unroll
            for (int k = 0; k < 8; ++k) slot[t + k * T] = x[k];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < QR * W; idx += TC_THREADS) {
            const int rr = idx / W, e = idx - rr * W;
            U[(r0 + rr) * W + e] = zsplit<LG>(X + (rr >> 1) * G::SLOT, rr & 1, e);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// row phase, adjoint (backward in time), Heun stage:
//   k = div(lam_s v); stage 1: lam* = lam_j + h k; stage 2: lam_{j-1} = (lam_j + lam* + h k) / 2,
//   b += w lam_{j-1} grad m_{j-1} (trapezoid weight w)
// or, with init, lam = ca a + cb c and b = w lam grad m (the final-time condition).
// On entry U holds the x^1-derivative spectra of the flux lam_s v1 and V the row
// spectra of lam_s v2; on exit (want_spec) U, V hold the row spectra of the new
// flux lam v1, lam v2.
// ---------------------------------------------------------------------------
struct AdjRow {
    bool init;
    int stage;
    bool want_spec;
    const float* a;  // init: lam = ca a + cb c (a nullable)
    float ca;
    const float* c;
    float cb;
    const float* lj;
    const float* ls;
    float* out;
    float* b;        // nullable: body force (init: written; stage 2: accumulated)
    const float* gm; // grad m at the output time
    float w;
};

template <int LG>
__device__ void adj_rows(int rank, const TcArgs& a, const AdjRow& s, float2* U, float2* V, float2* X,
                         const float2* tws) {
    using G = TcGeom<LG>;
    constexpr int n = G::n, W = G::W, R = G::R, T = G::T, QR = G::QR, N = G::N;
    const int q = threadIdx.x / T, t = threadIdx.x - q * T;
    const bool act = q < QR;
    const bool act2 = q < QR / 2;
    const float cd2 = 1.0f / (float)n;
    float* O = reinterpret_cast<float*>(X + G::OROW);
#pragma unroll 1
    for (int r0 = 0; r0 < R; r0 += QR) {
        const int r = r0 + (act ? q : 0);
        const size_t rowbase = (size_t)(rank * R + r) * n;
        float2 x[8];
        if (!s.init) {
            // divergence of rows r0 + 2q, r0 + 2q + 1, packed as one complex inverse transform
            const int ra = r0 + 2 * (act2 ? q : 0);
            if (act2) {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    x[k] = zdiv<LG>(U + ra * W, V + ra * W, U + (ra + 1) * W, V + (ra + 1) * W, t + k * T, cd2);
            }
            float2* slot = X + (act2 ? q : 0) * G::SLOT;
            fft_ip<LG, true>(x, t, act2, slot, tws);
            if (act2) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    O[2 * q * n + t + k * T] = x[k].x;
                    O[(2 * q + 1) * n + t + k * T] = x[k].y;
                }
            }
            __syncthreads();
        }
        if (act) {
#pragma unroll
            for (int k0 = 0; k0 < 8; k0 += 4) {
                float lv[4], v1[4], v2[4];
#pragma unroll
                for (int k = k0; k < k0 + 4; ++k) {
                    const size_t idx = rowbase + t + k * T;
                    v1[k - k0] = a.v[idx];
                    v2[k - k0] = a.v[N + idx];
                    if (s.init) {
                        float l = s.cb * s.c[idx];
                        if (s.a) l = fmaf(s.ca, s.a[idx], l);
                        lv[k - k0] = l;
                    } else {
                        const float lj = s.lj[idx];
                        const float ls = (s.stage == 2) ? s.ls[idx] : 0.f;
                        const float dv = O[q * n + t + k * T];
                        lv[k - k0] = (s.stage == 1) ? fmaf(a.h, dv, lj) : 0.5f * (lj + ls + a.h * dv);
                    }
                }
#pragma unroll
                for (int k = k0; k < k0 + 4; ++k) {
                    const size_t idx = rowbase + t + k * T;
                    const float l = lv[k - k0];
                    s.out[idx] = l;
                    if (s.b) {
                        const float wl = s.w * l;
                        if (s.init) {
                            s.b[idx] = wl * s.gm[idx];
                            s.b[N + idx] = wl * s.gm[N + idx];
                        } else {
                            s.b[idx] = fmaf(wl, s.gm[idx], s.b[idx]);
                            s.b[N + idx] = fmaf(wl, s.gm[N + idx], s.b[N + idx]);
                        }
                    }
                    x[k] = make_float2(l * v1[k - k0], l * v2[k - k0]);
                }
            }
        }
        if (!s.want_spec) {
            __syncthreads();
            continue;
        }
        __syncthreads();  // the inverse transforms' last reads of their slots are done
        float2* slot = X + (act ? q : 0) * G::SLOT;
        fft_ip<LG, false>(x, t, act, slot, tws);
        __syncthreads();
        if (act) {
#pragma unroll
            for (int k = 0; k < 8; ++k) slot[t + k * T] = x[k];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < QR * W; idx += TC_THREADS) {
            const int rr = idx / W, e = idx - rr * W;
            const float2* Z = X + rr * G::SLOT;
            U[(r0 + rr) * W + e] = zsplit<LG>(Z, 0, e);
            V[(r0 + rr) * W + e] = zsplit<LG>(Z, 1, e);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// the kernel: one cluster = one transport solve (or both solves of a matvec)
// ---------------------------------------------------------------------------
template <int LG, int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_transport_cluster(TcArgs a) {
    using G = TcGeom<LG>;
    extern __shared__ __align__(16) float2 sm[];
    float2* tws = sm;
    float2* U = sm + G::TWE;
    float2* V = U + G::RW;
    float2* X = V + G::RW;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    tw_stage<LG>(tws, a.tw);
    __syncthreads();
    const float scale = 1.0f / (float)G::N;
    const int nt = a.nt;

    if (MODE == TC_STATE) {
        // m_0 = m_T; Heun steps; grad m_j stored at stage 1 of step j, grad m_nt at the end
        AdvRow s{};
        s.kind = ADV_INIT; s.init = a.mT; s.out = a.m_hist; s.want_spec = true;
        adv_rows<LG>(rank, a, s, U, V, X, tws);
        cl.sync();
#pragma unroll 1
        for (int j = 0; j < nt; ++j) {
            float* mj = a.m_hist + (size_t)j * G::N;
            col_phase<LG, false>(cl, rank, U, V, X, tws, scale);
            AdvRow s1{};
            s1.kind = ADV_STAGE; s1.stage = 1; s1.want_spec = true;
            s1.uj = mj; s1.out = a.us; s1.grad_out = a.gm_hist + (size_t)j * 2 * G::N;
            adv_rows<LG>(rank, a, s1, U, V, X, tws);
            cl.sync();
            col_phase<LG, false>(cl, rank, U, V, X, tws, scale);
            AdvRow s2{};
            s2.kind = ADV_STAGE; s2.stage = 2; s2.want_spec = true;
            s2.uj = mj; s2.us = a.us; s2.out = mj + G::N;
            adv_rows<LG>(rank, a, s2, U, V, X, tws);
            cl.sync();
        }
        col_phase<LG, false>(cl, rank, U, V, X, tws, scale);
        AdvRow sg{};
        sg.kind = ADV_GRAD_ONLY; sg.grad_out = a.gm_hist + (size_t)nt * 2 * G::N;
        adv_rows<LG>(rank, a, sg, U, V, X, tws);
        return;
    }

    if (MODE == TC_MATVEC) {
        // incremental state from m~_0 = 0 (Eq. (e:inc-state-eq-elim)); m~_j in a.uj, m~* in a.us
#pragma unroll 1
        for (int j = 0; j < nt; ++j) {
            if (j > 0) col_phase<LG, false>(cl, rank, U, V, X, tws, scale);
            AdvRow s1{};
            s1.kind = ADV_STAGE; s1.stage = 1; s1.want_spec = true; s1.zero_grad = (j == 0);
            s1.uj = (j > 0) ? a.uj : nullptr; s1.out = a.us; s1.gm = a.gm_hist + (size_t)j * 2 * G::N;
            adv_rows<LG>(rank, a, s1, U, V, X, tws);
            cl.sync();
            col_phase<LG, false>(cl, rank, U, V, X, tws, scale);
            AdvRow s2{};
            s2.kind = ADV_STAGE; s2.stage = 2; s2.want_spec = (j + 1 < nt);
            s2.uj = (j > 0) ? a.uj : nullptr; s2.us = a.us; s2.out = a.uj;
            s2.gm = a.gm_hist + (size_t)(j + 1) * 2 * G::N;
            adv_rows<LG>(rank, a, s2, U, V, X, tws);
            cl.sync();
        }
    }

    // adjoint backward in time (Eq. (e:adj-eq-elim); Gauss-Newton incremental adjoint
    // Eq. (e:inc-adj-eq-elim)): lam_nt = ca a + cb c, body force with trapezoid weights
    {
        AdjRow s0{};
        s0.init = true; s0.want_spec = true;
        s0.a = a.adj_a; s0.ca = a.adj_ca; s0.c = (MODE == TC_MATVEC) ? a.uj : a.adj_c; s0.cb = a.adj_cb;
        s0.out = a.lj; s0.b = a.b; s0.gm = a.gm_hist + (size_t)nt * 2 * G::N; s0.w = 0.5f * a.h;
        adj_rows<LG>(rank, a, s0, U, V, X, tws);
        cl.sync();
#pragma unroll 1
        for (int j = nt; j >= 1; --j) {
            col_phase<LG, true>(cl, rank, U, U, X, tws, scale);
            AdjRow s1{};
            s1.stage = 1; s1.want_spec = true; s1.lj = a.lj; s1.out = a.ls;
            adj_rows<LG>(rank, a, s1, U, V, X, tws);
            cl.sync();
            col_phase<LG, true>(cl, rank, U, U, X, tws, scale);
            AdjRow s2{};
            s2.stage = 2; s2.want_spec = (j > 1); s2.lj = a.lj; s2.ls = a.ls; s2.out = a.lj;
            s2.b = a.b; s2.gm = a.gm_hist + (size_t)(j - 1) * 2 * G::N; s2.w = (j - 1 == 0) ? 0.5f * a.h : a.h;
            adj_rows<LG>(rank, a, s2, U, V, X, tws);
            cl.sync();
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
#define TC_DISPATCH(LOG, ...)                                     \
    switch (LOG) {                                                \
        case 4: { constexpr int LG = 4; __VA_ARGS__; } break;     \
        case 5: { constexpr int LG = 5; __VA_ARGS__; } break;     \
        case 6: { constexpr int LG = 6; __VA_ARGS__; } break;     \
        case 7: { constexpr int LG = 7; __VA_ARGS__; } break;     \
        case 8: { constexpr int LG = 8; __VA_ARGS__; } break;     \
        case 9: { constexpr int LG = 9; __VA_ARGS__; } break;     \
        default: break;                                           \
    }

template <int LG, int MODE>
static cudaLaunchConfig_t tc_config(cudaStream_t stream, cudaLaunchAttribute* attr) {
    using G = TcGeom<LG>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G::CS, 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G::CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Per (device, kernel): opt in to the shared memory and the cluster size (the attributes
// apply to the current device only).
template <int LG, int MODE>
static cudaError_t tc_prepare() {
    using G = TcGeom<LG>;
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    auto kern = k_transport_cluster<LG, MODE>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    if (G::CS > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    done[dev] = true;
    return cudaSuccess;
}

template <int LG, int MODE>
static int tc_max_clusters() {
    if (tc_prepare<LG, MODE>() != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tc_config<LG, MODE>(0, attr);
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, k_transport_cluster<LG, MODE>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return num;
}

int tc_max_active_clusters(int n1, int n2) {
    if (n1 != n2 || n1 < 16 || n1 > 512 || (n1 & (n1 - 1))) return 0;
    int lg = 0;
    while ((1 << lg) < n1) ++lg;
    int m = 0;
    TC_DISPATCH(lg, {
        const int a = tc_max_clusters<LG, TC_STATE>();
        const int b = tc_max_clusters<LG, TC_ADJOINT>();
        const int c = tc_max_clusters<LG, TC_MATVEC>();
        m = a < b ? a : b;
        m = m < c ? m : c;
    });
    return m;
}

int tc_cluster_size(int n) {
    int lg = 0;
    while ((1 << lg) < n) ++lg;
    int cs = 0;
    TC_DISPATCH(lg, { cs = TcGeom<LG>::CS; });
    return cs;
}

void launch_transport_cluster(reg_ctx* ctx, int mode, const TcArgs& args) {
    TcArgs a = args;
    a.tw = ctx->tw;
    const double N = (double)ctx->N;
    const int nt = a.nt;
    // algorithmic bytes of the launch (each input and output field once per time level it is
    // used at): state: m_T, v, m_1..m_nt, grad m_0..nt; adjoint: m_R, m_nt, v, grad m_0..nt, b;
    // matvec: v, v~, grad m_0..nt (both sweeps), b~
    double fields = 0;
    if (mode == TC_STATE) fields = 1 + 2 + nt + 2.0 * (nt + 1);
    else if (mode == TC_ADJOINT) fields = 2 + 2 + 2.0 * (nt + 1) + 2;
    else fields = 2 + 2 + 4.0 * (nt + 1) + 2;
    ktimer_begin(ctx, KC_TRANSPORT, 4.0 * fields * N);
    TC_DISPATCH(ctx->log1, {
        cudaLaunchAttribute attr[1];
        if (mode == TC_STATE) {
            tc_prepare<LG, TC_STATE>();
            cudaLaunchConfig_t cfg = tc_config<LG, TC_STATE>(ctx->stream, attr);
            cudaLaunchKernelEx(&cfg, k_transport_cluster<LG, TC_STATE>, a);
        } else if (mode == TC_ADJOINT) {
            tc_prepare<LG, TC_ADJOINT>();
            cudaLaunchConfig_t cfg = tc_config<LG, TC_ADJOINT>(ctx->stream, attr);
            cudaLaunchKernelEx(&cfg, k_transport_cluster<LG, TC_ADJOINT>, a);
        } else {
            tc_prepare<LG, TC_MATVEC>();
            cudaLaunchConfig_t cfg = tc_config<LG, TC_MATVEC>(ctx->stream, attr);
            cudaLaunchKernelEx(&cfg, k_transport_cluster<LG, TC_MATVEC>, a);
        }
    });
    ktimer_end(ctx);
}
