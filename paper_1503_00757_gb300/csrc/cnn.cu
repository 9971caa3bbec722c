// Learned warm start: an 8-layer 3x3 convolutional network with
// circular padding (channel widths 2 -> 32 x 7 -> 2, ReLU between layers)
// that predicts the velocity of a registration from the image pair
// (m_T, m_R).  The middle layers are dilated (layer l samples its taps
// d_l = min(DIL[l], H / TH, W / TW) pixels apart), so the receptive field
// covers the large-scale motion.  The raw output is low-pass filtered by a
// Gaussian (symbol exp(-sigma^2 |k|^2 / 2), sigma = 2 h, h = 2 pi / max(H, W))
// and Leray-projected (Eq. (e:project-body-force) with w = 0), so that a warm
// start carries no grid-scale noise and satisfies div v = 0.  The paper has no
// learned component; the network only seeds reg_solve, whose tolerance test
// is unchanged.
//
// A convolution of dilation d on an H x W periodic grid is an ordinary 3x3
// circular convolution on each of the d^2 interleaved sub-grids
// {(Y d + ry, X d + rx)} of size (H/d) x (W/d); each CTA tile lives in one
// sub-grid, so the halo staging and the tensor-core loop are those of d = 1.
//
// Arithmetic: BF16 activations and weights, FP32 accumulation on the tensor
// cores (mma.sync m16n8k16), FP32 master weights, Adam.  Layouts:
// activations NHWC BF16 with C in {16, 32} (channels beyond the real width
// are zero); forward weights [Cout][tap][Cin] BF16; transposed-flipped
// weights [Cin][8 - tap][Cout] for the input gradient (the adjoint of a
// circular correlation is the correlation with the flipped kernel).
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"

typedef __nv_bfloat16 bf16;

namespace {

constexpr int TH = 8;    // output rows per CTA tile
constexpr int TW = 32;   // output columns per CTA tile
constexpr int NLAYER = 8;
constexpr int CH[NLAYER + 1] = {2, 32, 32, 32, 32, 32, 32, 32, 2};
constexpr int DIL[NLAYER] = {1, 2, 4, 8, 8, 4, 2, 1};

// dilation of layer l on an H x W grid (every sub-grid at least TH x TW)
int layer_dil(int l, int H, int W) {
    int d = DIL[l];
    while (d > 1 && (H / d < TH || W / d < TW)) d >>= 1;
    return d;
}

// CTA tile -> sub-grid (ry, rx) of dilation d and tile origin (Y0, X0) in
// sub-grid coordinates; grid point of sub-grid point (Y, X): (Y d + ry, X d + rx).
struct TileMap {
    int d, Hs, Ws, ry, rx, Y0, X0;
    __device__ __forceinline__ int gy(int Y) const { return (Y & (Hs - 1)) * d + ry; }
    __device__ __forceinline__ int gx(int X) const { return (X & (Ws - 1)) * d + rx; }
};
__device__ __forceinline__ TileMap tile_map(int tile, int H, int W, int d) {
    TileMap m;
    m.d = d;
    m.Hs = H / d;
    m.Ws = W / d;
    const int tx = m.Ws / TW, per = (m.Hs / TH) * tx;
    const int r = tile / per, tt = tile - r * per;
    m.ry = r / d;
    m.rx = r - m.ry * d;
    m.Y0 = (tt / tx) * TH;
    m.X0 = (tt - (tt / tx) * tx) * TW;
    return m;
}

__host__ __device__ constexpr int padc(int c) { return c <= 16 ? 16 : 32; }

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack_h(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ---------------------------------------------------------------------------
// conv3x3 (circular), implicit GEMM: M = pixels of a TH x TW tile, N = COUT,
// K = 9 * CIN.  Warp w computes output row w of the tile (2 m16 tiles).
// MODE 0: out = bf16 NHWC relu(z + bias)
// MODE 1: out = fp32 planar [B][2][H][W] z + bias (channels 0, 1 only)
// MODE 2: out = bf16 NHWC z * (mask > 0)       (input gradient through a ReLU)
// MODE 3: out = bf16 NHWC z                      (input gradient, no ReLU)
// ---------------------------------------------------------------------------
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(256) k_conv3x3(const bf16* __restrict__ in, const bf16* __restrict__ w,
                                                 const float* __restrict__ bias, void* out,
                                                 const bf16* __restrict__ mask, int H, int W, int dil) {
    constexpr int SP = CIN + 8;            // smem pixel stride (halves), conflict-free fragment loads
    constexpr int KW = 9 * CIN + 8;        // smem weight row stride (halves)
    constexpr int HP = (TH + 2) * (TW + 2);
    extern __shared__ __align__(16) unsigned char smraw[];
    bf16* s_in = reinterpret_cast<bf16*>(smraw);
    bf16* s_w = s_in + HP * SP;
    const TileMap tm = tile_map(blockIdx.x, H, W, dil);
    const int b = blockIdx.y;
    // stage the input tile with a one-point circular halo of its sub-grid (16-byte pieces)
    constexpr int V = CIN / 8;  // uint4 per pixel
    for (int i = threadIdx.x; i < HP * V; i += blockDim.x) {
        const int hp = i / V, part = i - hp * V;
        const int hy = hp / (TW + 2), hx = hp - hy * (TW + 2);
        const int gy = tm.gy(tm.Y0 + hy - 1 + tm.Hs), gx = tm.gx(tm.X0 + hx - 1 + tm.Ws);
        const uint4 val = reinterpret_cast<const uint4*>(in + (((size_t)b * H + gy) * W + gx) * CIN)[part];
        *reinterpret_cast<uint4*>(s_in + hp * SP + part * 8) = val;
    }
    for (int i = threadIdx.x; i < COUT * 9 * CIN / 8; i += blockDim.x) {
        const int row = i / (9 * CIN / 8), part = i - row * (9 * CIN / 8);
        *reinterpret_cast<uint4*>(s_w + row * KW + part * 8) = reinterpret_cast<const uint4*>(w + row * 9 * CIN)[part];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    constexpr int NT = COUT / 8;
    float acc[2][NT][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
    const uint32_t* s_in32 = reinterpret_cast<const uint32_t*>(s_in);
    const uint32_t* s_w32 = reinterpret_cast<const uint32_t*>(s_w);
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap - 3 * dy;  // halo offsets 0..2 (= -1..1 + 1)
#pragma unroll
        for (int kc = 0; kc < CIN / 16; ++kc) {
            uint32_t a[2][4];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int px = m * 16 + g;
                const int p0 = (warp + dy) * (TW + 2) + px + dx;
                const int p1 = p0 + 8;
                const int c0 = kc * 16 + 2 * t;
                a[m][0] = s_in32[(p0 * SP + c0) >> 1];
                a[m][1] = s_in32[(p1 * SP + c0) >> 1];
                a[m][2] = s_in32[(p0 * SP + c0 + 8) >> 1];
                a[m][3] = s_in32[(p1 * SP + c0 + 8) >> 1];
            }
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int k0 = tap * CIN + kc * 16 + 2 * t;
                uint32_t bb[2];
                bb[0] = s_w32[((n * 8 + g) * KW + k0) >> 1];
                bb[1] = s_w32[((n * 8 + g) * KW + k0 + 8) >> 1];
#pragma unroll
                for (int m = 0; m < 2; ++m) mma16816(acc[m][n], a[m], bb);
            }
        }
    }
    const int y = tm.gy(tm.Y0 + warp);
#pragma unroll
    for (int m = 0; m < 2; ++m) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int x = tm.gx(tm.X0 + m * 16 + g + 8 * h);
            const size_t pix = ((size_t)b * H + y) * W + x;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int co = n * 8 + 2 * t;
                float v0 = acc[m][n][2 * h], v1 = acc[m][n][2 * h + 1];
                if (MODE == 0) {
                    v0 = fmaxf(v0 + bias[co], 0.f);
                    v1 = fmaxf(v1 + bias[co + 1], 0.f);
                    reinterpret_cast<uint32_t*>(out)[(pix * COUT + co) >> 1] = pack2(v0, v1);
                } else if (MODE == 1) {
                    if (co == 0) {
                        float* o = reinterpret_cast<float*>(out);
                        const size_t plane = (size_t)H * W;
                        o[((size_t)b * 2 + 0) * plane + (size_t)y * W + x] = v0 + bias[0];
                        o[((size_t)b * 2 + 1) * plane + (size_t)y * W + x] = v1 + bias[1];
                    }
                } else {
                    if (MODE == 2) {
                        const __nv_bfloat162 mk = reinterpret_cast<const __nv_bfloat162*>(mask)[(pix * COUT + co) >> 1];
                        if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                        if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
                    }
                    reinterpret_cast<uint32_t*>(out)[(pix * COUT + co) >> 1] = pack2(v0, v1);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// weight gradient: dW[co][tap][ci] = sum_pixels dz[p][co] a[p + tap][ci], as a
// GEMM with M = COUT, N = 9 * CIN (warp w = tap w), K = pixels; each CTA
// accumulates a strided set of TH x TW tiles and writes its partial sums
// (deterministic reduction in k_wgrad_reduce).  Also the bias partials.
// ---------------------------------------------------------------------------
template <int CIN, int COUT>
__global__ void __launch_bounds__(288) k_wgrad(const bf16* __restrict__ a, const bf16* __restrict__ dz,
                                               float* partial, float* bpartial, int H, int W, int B, int dil) {
    constexpr int HP = (TH + 2) * (TW + 2);
    constexpr int PT = TH * TW;        // pixels per tile
    constexpr int DZS = PT + 8;        // smem stride of dz^T rows (halves)
    constexpr int AS = HP + 8;         // smem stride of a^T rows (halves)
    extern __shared__ __align__(16) unsigned char smraw[];
    bf16* s_dz = reinterpret_cast<bf16*>(smraw);   // [COUT][PT]
    bf16* s_a = s_dz + COUT * DZS;                  // [CIN][HP]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int tap = warp;  // 9 warps
    const int dy = tap / 3, dx = tap - 3 * dy;
    constexpr int NT = CIN / 8;
    float acc[COUT / 16][NT][4];
#pragma unroll
    for (int m = 0; m < COUT / 16; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
    float bacc = 0.f;
    const int per_img = (H / TH) * (W / TW), tiles = per_img * B;
    const uint32_t* s_dz32 = reinterpret_cast<const uint32_t*>(s_dz);
    for (int ti = blockIdx.x; ti < tiles; ti += gridDim.x) {
        const int b = ti / per_img;
        const TileMap tm = tile_map(ti - b * per_img, H, W, dil);
        __syncthreads();
        for (int i = threadIdx.x; i < PT * COUT; i += blockDim.x) {
            const int p = i / COUT, co = i - p * COUT;
            const size_t pix = ((size_t)b * H + tm.gy(tm.Y0 + p / TW)) * W + tm.gx(tm.X0 + (p % TW));
            s_dz[co * DZS + p] = dz[pix * COUT + co];
        }
        for (int i = threadIdx.x; i < HP * CIN; i += blockDim.x) {
            const int hp = i / CIN, ci = i - hp * CIN;
            const int hy = hp / (TW + 2), hx = hp - hy * (TW + 2);
            const int gy = tm.gy(tm.Y0 + hy - 1 + tm.Hs), gx = tm.gx(tm.X0 + hx - 1 + tm.Ws);
            s_a[ci * AS + hp] = a[(((size_t)b * H + gy) * W + gx) * CIN + ci];
        }
        __syncthreads();
        if (threadIdx.x < COUT) {
            float s = 0.f;
            for (int p = 0; p < PT; ++p) s += __bfloat162float(s_dz[threadIdx.x * DZS + p]);
            bacc += s;
        }
#pragma unroll 1
        for (int k0 = 0; k0 < PT; k0 += 16) {
            const int row = k0 / TW, col0 = k0 % TW;  // 16 pixels of one tile row
            uint32_t af[COUT / 16][4];
#pragma unroll
            for (int m = 0; m < COUT / 16; ++m) {
                const int co = m * 16 + g;
                af[m][0] = s_dz32[(co * DZS + k0 + 2 * t) >> 1];
                af[m][1] = s_dz32[((co + 8) * DZS + k0 + 2 * t) >> 1];
                af[m][2] = s_dz32[(co * DZS + k0 + 2 * t + 8) >> 1];
                af[m][3] = s_dz32[((co + 8) * DZS + k0 + 2 * t + 8) >> 1];
            }
            const int hbase = (row + dy) * (TW + 2) + col0 + dx;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const bf16* arow = s_a + (n * 8 + g) * AS + hbase;
                uint32_t bf[2];
                bf[0] = pack_h(arow[2 * t], arow[2 * t + 1]);
                bf[1] = pack_h(arow[2 * t + 8], arow[2 * t + 9]);
#pragma unroll
                for (int m = 0; m < COUT / 16; ++m) mma16816(acc[m][n], af[m], bf);
            }
        }
    }
    float* P = partial + (size_t)blockIdx.x * COUT * 9 * CIN;
#pragma unroll
    for (int m = 0; m < COUT / 16; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int co = m * 16 + g + (q >= 2 ? 8 : 0);
                const int ci = n * 8 + 2 * t + (q & 1);
                P[(co * 9 + tap) * CIN + ci] = acc[m][n][q];
            }
    if (threadIdx.x < COUT) bpartial[(size_t)blockIdx.x * COUT + threadIdx.x] = bacc;
}

__global__ void k_wgrad_reduce(const float* __restrict__ partial, const float* __restrict__ bpartial, int nparts,
                               int nw, int nb, float* dW, float* db) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nw) {
        float s = 0.f;
        for (int p = 0; p < nparts; ++p) s += partial[(size_t)p * nw + i];
        dW[i] = s;
    } else if (i < nw + nb) {
        const int j = i - nw;
        float s = 0.f;
        for (int p = 0; p < nparts; ++p) s += bpartial[(size_t)p * nb + j];
        db[j] = s;
    }
}

// images (fp32 planar [B][2][H][W]) -> NHWC bf16 with 16 channels (2 real)
__global__ void k_pack_input(const float* __restrict__ img, bf16* x, int B, int H, int W) {
    const size_t n = (size_t)B * H * W;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const size_t b = p / ((size_t)H * W), r = p - b * H * W;
        const float c0 = img[(b * 2 + 0) * H * W + r], c1 = img[(b * 2 + 1) * H * W + r];
        uint4 v0, v1;
        v0.x = pack2(c0, c1);
        v0.y = v0.z = v0.w = 0u;
        v1.x = v1.y = v1.z = v1.w = 0u;
        reinterpret_cast<uint4*>(x + p * 16)[0] = v0;
        reinterpret_cast<uint4*>(x + p * 16)[1] = v1;
    }
}

// dL/d out (fp32 planar) -> NHWC bf16 with 16 channels (2 real)
__global__ void k_pack_grad(const float* __restrict__ d, bf16* dz, int B, int H, int W) {
    const size_t n = (size_t)B * H * W;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const size_t b = p / ((size_t)H * W), r = p - b * H * W;
        uint4 v0, v1;
        v0.x = pack2(d[(b * 2 + 0) * H * W + r], d[(b * 2 + 1) * H * W + r]);
        v0.y = v0.z = v0.w = 0u;
        v1.x = v1.y = v1.z = v1.w = 0u;
        reinterpret_cast<uint4*>(dz + p * 16)[0] = v0;
        reinterpret_cast<uint4*>(dz + p * 16)[1] = v1;
    }
}

// residual r = pred - target, FP64 partials of sum(r^2)
__global__ void k_residual(const float* __restrict__ pred, const float* __restrict__ tgt, float* r, long long n,
                           double* part) {
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = pred[i] - tgt[i];
        r[i] = d;
        acc += (double)d * d;
    }
    __shared__ double sm[256];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

struct LayerDesc {
    int cin, cout, cinp, coutp;
    long long woff, boff;  // offsets into the flat FP32 parameter array (oracle layout)
};

// Adam on the flat FP32 parameters (W (Cout, Cin, 3, 3) then b (Cout) per
// layer); gradients come in the padded [Cout_p][tap][Cin_p] layout.  Also
// rewrites the BF16 forward and transposed-flipped weights.
__global__ void k_adam_pack(float* params, const float* __restrict__ gW, const float* __restrict__ gb, float* m1,
                            float* m2, int nparams, const LayerDesc* __restrict__ layers, int nlayers,
                            const long long* __restrict__ gwoff, const long long* __restrict__ gboff, float lr,
                            float c1, float c2, int update, bf16* wf, bf16* wt, const long long* __restrict__ wfoff) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nparams; i += gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < nlayers && i >= layers[l + 1].woff) ++l;
        const LayerDesc L = layers[l];
        float grad;
        int co, ci = -1, tap = -1;
        if (i < L.boff) {
            const int j = (int)(i - L.woff);
            co = j / (L.cin * 9);
            const int rem = j - co * L.cin * 9;
            ci = rem / 9;
            tap = rem - ci * 9;
            grad = gW[gwoff[l] + ((long long)co * 9 + tap) * L.cinp + ci];
        } else {
            co = (int)(i - L.boff);
            grad = gb[gboff[l] + co];
        }
        float p = params[i];
        if (update) {
            const float a = 0.9f * m1[i] + 0.1f * grad;
            const float v = 0.999f * m2[i] + 0.001f * grad * grad;
            m1[i] = a;
            m2[i] = v;
            p -= lr * (a / c1) / (sqrtf(v / c2) + 1e-8f);
            params[i] = p;
        }
        if (tap >= 0) {
            wf[wfoff[l] + ((long long)co * 9 + tap) * L.cinp + ci] = __float2bfloat16_rn(p);
            wt[wfoff[l] + ((long long)ci * 9 + (8 - tap)) * L.coutp + co] = __float2bfloat16_rn(p);
        }
    }
}

__global__ void k_bias_pad(const float* __restrict__ params, const LayerDesc* __restrict__ layers, int nlayers,
                           float* bpad) {
    for (int l = 0; l < nlayers; ++l)
        for (int c = threadIdx.x; c < 32; c += blockDim.x)
            bpad[l * 32 + c] = (c < layers[l].cout) ? params[layers[l].boff + c] : 0.f;
}

}  // namespace

// ---------------------------------------------------------------------------
// network object
// ---------------------------------------------------------------------------
struct reg_net {
    int H, W, maxB;
    cudaStream_t stream;
    reg_ctx* proj;             // Leray projection on the H x W grid
    std::vector<LayerDesc> layers;
    LayerDesc* d_layers;
    long long nparams;
    float *params, *m1, *m2;   // FP32 master weights and Adam moments (flat, oracle layout)
    float *gW, *gb;            // padded gradients
    long long *d_gwoff, *d_gboff, *d_wfoff;
    std::vector<long long> gwoff, gboff, wfoff;
    bf16 *wf, *wt;             // BF16 weights (forward, transposed-flipped)
    float* bpad;               // biases padded to 32 per layer
    bf16* act[NLAYER];         // layer inputs: act[0] = packed images (16 ch), act[l] = relu output of layer l
    bf16 *dzA, *dzB;           // gradient ping-pong (NHWC, 32 ch)
    float *out, *pred, *res, *dout;
    float *partial, *bpartial;
    int nwg;                   // wgrad CTAs
    double *d_part, *h_part;
    int adam_t;
    float out_scale;           // reg_net_forward multiplies its prediction by this
};

static size_t conv_smem(int cin, int cout) {
    return (size_t)((TH + 2) * (TW + 2) * (cin + 8) + cout * (9 * cin + 8)) * sizeof(bf16);
}
static size_t wgrad_smem(int cin, int cout) {
    return (size_t)(cout * (TH * TW + 8) + cin * ((TH + 2) * (TW + 2) + 8)) * sizeof(bf16);
}

template <typename K>
static void opt_in(K k, size_t bytes) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

extern "C" void reg_net_destroy(reg_net* n) {
    if (!n) return;
    if (n->proj) reg_destroy(n->proj);
    void* ptrs[] = {n->d_layers, n->params, n->m1, n->m2, n->gW, n->gb, n->d_gwoff, n->d_gboff, n->d_wfoff,
                    n->wf, n->wt, n->bpad, n->dzA, n->dzB, n->out, n->pred, n->res, n->dout, n->partial,
                    n->bpartial, n->d_part};
    for (void* p : ptrs) cudaFree(p);
    for (int l = 0; l < NLAYER; ++l) cudaFree(n->act[l]);
    cudaFreeHost(n->h_part);
    delete n;
}

extern "C" long long reg_net_num_params(reg_net* n) { return n ? n->nparams : 0; }

extern "C" int reg_net_create(int H, int W, int max_batch, reg_net** out) {
    if (!out) return reg_fail(REG_ERR_ARG, "out is NULL");
    *out = nullptr;
    auto p2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    if (!p2(H) || !p2(W) || H < 32 || W < 32 || H > 1024 || W > 1024)
        return reg_fail(REG_ERR_ARG, "H and W must be powers of two in [32, 1024]");
    if (max_batch < 1 || max_batch > 256) return reg_fail(REG_ERR_ARG, "max_batch must be in [1, 256]");
    reg_net* n = new reg_net();
    n->H = H; n->W = W; n->maxB = max_batch; n->stream = 0; n->adam_t = 0; n->out_scale = 1.f;
    long long off = 0, gwo = 0, gbo = 0, wfo = 0;
    for (int l = 0; l < NLAYER; ++l) {
        LayerDesc d;
        d.cin = CH[l]; d.cout = CH[l + 1]; d.cinp = padc(d.cin); d.coutp = padc(d.cout);
        d.woff = off; off += (long long)d.cout * d.cin * 9;
        d.boff = off; off += d.cout;
        n->layers.push_back(d);
        n->gwoff.push_back(gwo); gwo += (long long)d.coutp * 9 * d.cinp;
        n->gboff.push_back(gbo); gbo += d.coutp;
        n->wfoff.push_back(wfo); wfo += (long long)d.coutp * 9 * d.cinp;
    }
    n->nparams = off;
    const size_t pix = (size_t)max_batch * H * W;
    n->nwg = 2 * 152;
    bool ok = reg_create(reg_grid{H, W}, 1, REG_H1, 1.0, INFINITY, 0.0, &n->proj) == REG_OK;
    auto M = [&](void** p, size_t bytes) { if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false; };
    M((void**)&n->d_layers, sizeof(LayerDesc) * NLAYER);
    M((void**)&n->params, sizeof(float) * off);
    M((void**)&n->m1, sizeof(float) * off);
    M((void**)&n->m2, sizeof(float) * off);
    M((void**)&n->gW, sizeof(float) * gwo);
    M((void**)&n->gb, sizeof(float) * gbo);
    M((void**)&n->d_gwoff, sizeof(long long) * NLAYER);
    M((void**)&n->d_gboff, sizeof(long long) * NLAYER);
    M((void**)&n->d_wfoff, sizeof(long long) * NLAYER);
    M((void**)&n->wf, sizeof(bf16) * wfo);
    M((void**)&n->wt, sizeof(bf16) * wfo);
    M((void**)&n->bpad, sizeof(float) * 32 * NLAYER);
    for (int l = 0; l < NLAYER; ++l) M((void**)&n->act[l], sizeof(bf16) * pix * (l == 0 ? 16 : 32));
    M((void**)&n->dzA, sizeof(bf16) * pix * 32);
    M((void**)&n->dzB, sizeof(bf16) * pix * 32);
    M((void**)&n->out, sizeof(float) * pix * 2);
    M((void**)&n->pred, sizeof(float) * pix * 2);
    M((void**)&n->res, sizeof(float) * pix * 2);
    M((void**)&n->dout, sizeof(float) * pix * 2);
    M((void**)&n->partial, sizeof(float) * n->nwg * 32 * 9 * 32);
    M((void**)&n->bpartial, sizeof(float) * n->nwg * 32);
    M((void**)&n->d_part, sizeof(double) * 1024);
    if (ok && cudaMallocHost((void**)&n->h_part, sizeof(double) * 1024) != cudaSuccess) ok = false;
    if (!ok) {
        cudaGetLastError();
        reg_net_destroy(n);
        return reg_fail(REG_ERR_NOMEM, "network allocation failed");
    }
    cudaMemcpy(n->d_layers, n->layers.data(), sizeof(LayerDesc) * NLAYER, cudaMemcpyHostToDevice);
    cudaMemcpy(n->d_gwoff, n->gwoff.data(), sizeof(long long) * NLAYER, cudaMemcpyHostToDevice);
    cudaMemcpy(n->d_gboff, n->gboff.data(), sizeof(long long) * NLAYER, cudaMemcpyHostToDevice);
    cudaMemcpy(n->d_wfoff, n->wfoff.data(), sizeof(long long) * NLAYER, cudaMemcpyHostToDevice);
    cudaMemset(n->params, 0, sizeof(float) * off);
    cudaMemset(n->m1, 0, sizeof(float) * off);
    cudaMemset(n->m2, 0, sizeof(float) * off);
    cudaMemset(n->wf, 0, sizeof(bf16) * wfo);
    cudaMemset(n->wt, 0, sizeof(bf16) * wfo);
    cudaMemset(n->gW, 0, sizeof(float) * gwo);
    cudaMemset(n->gb, 0, sizeof(float) * gbo);
    opt_in(k_conv3x3<16, 32, 0>, conv_smem(16, 32));
    opt_in(k_conv3x3<32, 32, 0>, conv_smem(32, 32));
    opt_in(k_conv3x3<32, 16, 1>, conv_smem(32, 16));
    opt_in(k_conv3x3<16, 32, 2>, conv_smem(16, 32));
    opt_in(k_conv3x3<32, 32, 2>, conv_smem(32, 32));
    opt_in(k_wgrad<16, 32>, wgrad_smem(16, 32));
    opt_in(k_wgrad<32, 32>, wgrad_smem(32, 32));
    opt_in(k_wgrad<32, 16>, wgrad_smem(32, 16));
    if (cudaDeviceSynchronize() != cudaSuccess) {
        reg_net_destroy(n);
        return reg_fail(REG_ERR_CUDA, "network initialisation failed");
    }
    *out = n;
    return REG_OK;
}

extern "C" int reg_net_set_stream(reg_net* n, void* stream) {
    if (!n) return reg_fail(REG_ERR_ARG, "net is NULL");
    n->stream = (cudaStream_t)stream;
    return reg_set_stream(n->proj, stream);
}

static void repack(reg_net* n, int update, float lr) {
    float c1 = 1.f, c2 = 1.f;
    if (update) {
        n->adam_t += 1;
        c1 = 1.f - powf(0.9f, (float)n->adam_t);
        c2 = 1.f - powf(0.999f, (float)n->adam_t);
    }
    k_adam_pack<<<304, 256, 0, n->stream>>>(n->params, n->gW, n->gb, n->m1, n->m2, (int)n->nparams, n->d_layers,
                                            NLAYER, n->d_gwoff, n->d_gboff, lr, c1, c2, update, n->wf, n->wt,
                                            n->d_wfoff);
    k_bias_pad<<<1, 32, 0, n->stream>>>(n->params, n->d_layers, NLAYER, n->bpad);
}

extern "C" int reg_net_set_params(reg_net* n, const float* params) {
    if (!n || !params) return reg_fail(REG_ERR_ARG, "net or params is NULL");
    cudaMemcpyAsync(n->params, params, sizeof(float) * n->nparams, cudaMemcpyDeviceToDevice, n->stream);
    cudaMemsetAsync(n->m1, 0, sizeof(float) * n->nparams, n->stream);
    cudaMemsetAsync(n->m2, 0, sizeof(float) * n->nparams, n->stream);
    n->adam_t = 0;
    repack(n, 0, 0.f);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? REG_OK : reg_fail(REG_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" int reg_net_get_params(reg_net* n, float* params) {
    if (!n || !params) return reg_fail(REG_ERR_ARG, "net or params is NULL");
    const cudaError_t e = cudaMemcpyAsync(params, n->params, sizeof(float) * n->nparams, cudaMemcpyDeviceToDevice, n->stream);
    return e == cudaSuccess ? REG_OK : reg_fail(REG_ERR_CUDA, cudaGetErrorString(e));
}

// out = P G in per velocity (the output map; also its adjoint G P, since P and G
// are commuting symmetric Fourier multipliers)
static int leray_batch(reg_net* n, const float* in, float* out, int B) {
    const size_t f = (size_t)2 * n->H * n->W;
    const double sigma = 2.0 * (2.0 * M_PI / (double)(n->H > n->W ? n->H : n->W));
    for (int b = 0; b < B; ++b) {
        const int st = apply_smooth_proj(n->proj, (float)(0.5 * sigma * sigma), in + b * f, out + b * f);
        if (st != REG_OK) return st;
    }
    return REG_OK;
}

static int net_forward(reg_net* n, const float* images, int B) {
    const int H = n->H, W = n->W;
    k_pack_input<<<304, 256, 0, n->stream>>>(images, n->act[0], B, H, W);
    const dim3 grid((H / TH) * (W / TW), B);
    for (int l = 0; l < NLAYER; ++l) {
        const float* bias = n->bpad + 32 * l;
        const bf16* wl = n->wf + n->wfoff[l];
        const int d = layer_dil(l, H, W);
        if (l == 0)
            k_conv3x3<16, 32, 0><<<grid, 256, conv_smem(16, 32), n->stream>>>(n->act[0], wl, bias, n->act[1], nullptr, H, W, d);
        else if (l < NLAYER - 1)
            k_conv3x3<32, 32, 0><<<grid, 256, conv_smem(32, 32), n->stream>>>(n->act[l], wl, bias, n->act[l + 1], nullptr, H, W, d);
        else
            k_conv3x3<32, 16, 1><<<grid, 256, conv_smem(32, 16), n->stream>>>(n->act[l], wl, bias, n->out, nullptr, H, W, d);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("net forward: ") + cudaGetErrorString(e));
    return leray_batch(n, n->out, n->pred, B);
}

extern "C" int reg_net_forward(reg_net* n, const float* images, int B, float* v_out) {
    if (!n || !images || !v_out) return reg_fail(REG_ERR_ARG, "NULL argument");
    if (B < 1 || B > n->maxB) return reg_fail(REG_ERR_ARG, "batch out of range");
    const int st = net_forward(n, images, B);
    if (st != REG_OK) return st;
    cudaError_t e;
    if (n->out_scale != 1.f) {
        launch_axpby(n->proj, 2LL * B * n->H * n->W, n->out_scale, n->pred, 0.f, n->pred, -1, -1, v_out);
        e = cudaGetLastError();
    } else {
        e = cudaMemcpyAsync(v_out, n->pred, sizeof(float) * 2 * B * n->H * n->W, cudaMemcpyDeviceToDevice,
                            n->stream);
    }
    return e == cudaSuccess ? REG_OK : reg_fail(REG_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" int reg_net_set_output_scale(reg_net* n, float scale) {
    if (!n) return reg_fail(REG_ERR_ARG, "net is NULL");
    if (!(scale > 0.f && scale <= 4.f)) return reg_fail(REG_ERR_ARG, "output scale must be in (0, 4]");
    n->out_scale = scale;
    return REG_OK;
}

// forward, loss, backward into n->gW / n->gb
static int net_loss_grad(reg_net* n, const float* images, const float* targets, int B, double* loss) {
    const int H = n->H, W = n->W;
    int st = net_forward(n, images, B);
    if (st != REG_OK) return st;
    const long long M = 2LL * B * H * W;
    k_residual<<<256, 256, 0, n->stream>>>(n->pred, targets, n->res, M, n->d_part);
    cudaMemcpyAsync(n->h_part, n->d_part, sizeof(double) * 256, cudaMemcpyDeviceToHost, n->stream);
    st = leray_batch(n, n->res, n->dout, B);  // dL/d out = G P r / M (scaled below)
    if (st != REG_OK) return st;
    k_pack_grad<<<304, 256, 0, n->stream>>>(n->dout, n->dzA, B, H, W);
    const dim3 grid((H / TH) * (W / TW), B);
    const float invM = 1.0f / (float)M;
    bf16* dz = n->dzA;
    bf16* dnext = n->dzB;
    for (int l = NLAYER - 1; l >= 0; --l) {
        const LayerDesc& L = n->layers[l];
        float* gWl = n->gW + n->gwoff[l];
        float* gbl = n->gb + n->gboff[l];
        const int d = layer_dil(l, H, W);
        if (l == NLAYER - 1)
            k_wgrad<32, 16><<<n->nwg, 288, wgrad_smem(32, 16), n->stream>>>(n->act[l], dz, n->partial, n->bpartial, H, W, B, d);
        else if (l > 0)
            k_wgrad<32, 32><<<n->nwg, 288, wgrad_smem(32, 32), n->stream>>>(n->act[l], dz, n->partial, n->bpartial, H, W, B, d);
        else
            k_wgrad<16, 32><<<n->nwg, 288, wgrad_smem(16, 32), n->stream>>>(n->act[0], dz, n->partial, n->bpartial, H, W, B, d);
        const int nw = L.coutp * 9 * L.cinp, nb = L.coutp;
        k_wgrad_reduce<<<(nw + nb + 255) / 256, 256, 0, n->stream>>>(n->partial, n->bpartial, n->nwg, nw, nb, gWl, gbl);
        if (l > 0) {
            // input gradient through the ReLU of layer l-1: correlation with the flipped, transposed kernel
            const bf16* wtl = n->wt + n->wfoff[l];
            if (l == NLAYER - 1)
                k_conv3x3<16, 32, 2><<<grid, 256, conv_smem(16, 32), n->stream>>>(dz, wtl, nullptr, dnext, n->act[l], H, W, d);
            else
                k_conv3x3<32, 32, 2><<<grid, 256, conv_smem(32, 32), n->stream>>>(dz, wtl, nullptr, dnext, n->act[l], H, W, d);
            bf16* tmp = dz; dz = dnext; dnext = tmp;
        }
    }
    // the 1/M factor of the loss is applied to the FP32 gradients
    const long long ngw = n->gwoff.back() + (long long)n->layers.back().coutp * 9 * n->layers.back().cinp;
    const long long ngb = n->gboff.back() + n->layers.back().coutp;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("net backward: ") + cudaGetErrorString(e));
    // scale gradients in place
    launch_axpby(n->proj, ngw, invM, n->gW, 0.f, n->gW, -1, -1, n->gW);
    launch_axpby(n->proj, ngb, invM, n->gb, 0.f, n->gb, -1, -1, n->gb);
    e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("net backward: ") + cudaGetErrorString(e));
    double s = 0.0;
    for (int i = 0; i < 256; ++i) s += n->h_part[i];
    if (loss) *loss = 0.5 * s / (double)M;
    return REG_OK;
}

extern "C" int reg_net_loss_grad(reg_net* n, const float* images, const float* targets, int B, double* loss,
                                 float* grads) {
    if (!n || !images || !targets) return reg_fail(REG_ERR_ARG, "NULL argument");
    if (B < 1 || B > n->maxB) return reg_fail(REG_ERR_ARG, "batch out of range");
    int st = net_loss_grad(n, images, targets, B, loss);
    if (st != REG_OK) return st;
    if (grads) {
        // unpack padded gradients into the flat oracle layout
        std::vector<float> hw(n->gwoff.back() + (size_t)n->layers.back().coutp * 9 * n->layers.back().cinp);
        std::vector<float> hb(n->gboff.back() + n->layers.back().coutp);
        cudaMemcpy(hw.data(), n->gW, sizeof(float) * hw.size(), cudaMemcpyDeviceToHost);
        cudaMemcpy(hb.data(), n->gb, sizeof(float) * hb.size(), cudaMemcpyDeviceToHost);
        std::vector<float> flat(n->nparams);
        for (int l = 0; l < NLAYER; ++l) {
            const LayerDesc& L = n->layers[l];
            for (int co = 0; co < L.cout; ++co)
                for (int ci = 0; ci < L.cin; ++ci)
                    for (int tap = 0; tap < 9; ++tap)
                        flat[L.woff + ((long long)co * L.cin + ci) * 9 + tap] =
                            hw[n->gwoff[l] + ((long long)co * 9 + tap) * L.cinp + ci];
            for (int co = 0; co < L.cout; ++co) flat[L.boff + co] = hb[n->gboff[l] + co];
        }
        const cudaError_t e = cudaMemcpy(grads, flat.data(), sizeof(float) * n->nparams, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, cudaGetErrorString(e));
    }
    return REG_OK;
}

extern "C" int reg_net_train_step(reg_net* n, const float* images, const float* targets, int B, float lr,
                                  double* loss) {
    if (!n || !images || !targets) return reg_fail(REG_ERR_ARG, "NULL argument");
    if (B < 1 || B > n->maxB) return reg_fail(REG_ERR_ARG, "batch out of range");
    const int st = net_loss_grad(n, images, targets, B, loss);
    if (st != REG_OK) return st;
    repack(n, 1, lr);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? REG_OK : reg_fail(REG_ERR_CUDA, cudaGetErrorString(e));
}
