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
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"
#include "tc.cuh"

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
// conv3x3 on the 5th-generation tensor cores (tcgen05, accumulator in TMEM),
// operands staged by TMA: the same implicit GEMM and the same MODEs as
// k_conv3x3.  A CTA owns one TH x TW tile at a time (persistent loop over
// tiles); its 256 pixels form two M = 128 blocks (tile rows 0-3 and 4-7),
// N = COUT, and each of the 9 taps adds CIN / 16 MMAs of K = 16 per block,
// issued by one thread; TMEM columns 0 and 32 hold the two FP32 accumulators.
//
// Shared-memory operands, canonical K-major without swizzle (16-byte rows of
// 8 channels, 8-row core matrices of 128 contiguous bytes):
//   B (weights, staged once per CTA): row (tap, c, co) at ((tap NC + c) COUT + co) 16,
//     so an MMA's K = 16 slice (chunks c, c + 1) has LBO = 16 COUT, SBO = 128;
//   A (input tile, two buffers): three column-shifted copies s = 0, 1, 2 of the
//     halo tile; block (s, c) holds channels 8c..8c+7 of halo pixel (hr, x + s)
//     at row hr TW + x, blocks ABS = (TH + 2) TW 16 bytes apart.  Tap (dy, dx) of
//     M block mt starts at block (dx, c), row (4 mt + dy) TW: 128 consecutive
//     rows with the uniform stride the descriptor needs (LBO = ABS, SBO = 128).
// Each block (s, c) is one TMA box (8 channels x TW columns x TH + 2 rows) of
// a 5-D view of the NHWC activations, dims (C, rx, X, ry, Y + (H/d) b), in
// which the sub-grid (ry, rx) of dilation d is a plain 3-D box.  TMA cannot
// wrap around the periodic boundary (it zero-fills outside the view and reads
// across image boundaries), so halo rows 0 / TH+1 and columns 0 / TW+1 of
// tiles at a sub-grid edge are rewritten from global memory by the threads.
// Pipeline over a CTA's tiles i = 0, 1, ...: three A buffers and two TMEM
// accumulator sets.  In iteration i thread 0 issues the MMAs of tile i, then,
// once the MMAs of tile i - 1 have completed, the TMA of tile i + 2 into the
// buffer tile i - 1 used, while all threads load tile i + 1's wrap-around
// pieces into registers and drain tile i - 1's accumulators (epilogue), so
// TMA, tensor cores and epilogue overlap.
// ---------------------------------------------------------------------------
// A-buffer layouts of a staged halo tile (three column-shifted copies s, halo rows hr,
// columns x, channel chunks c of 8):
//   SW = false: blocks (s, c) of (TH + 2) TW 16-byte rows, ABS bytes apart (canonical layout
//     without swizzle; also the MN-major layout of the weight gradient);
//   SW = true (CIN = 32): copies of (TH + 2) TW 64-byte rows (a whole pixel), 16-byte chunks
//     permuted by the 64-byte swizzle (chunk c of row r at chunk c ^ ((r >> 1) & 3)), the
//     layout a TMA box with the 64-byte swizzle writes: one box per copy instead of NC.
template <int CIN, bool SW>
struct HaloLayout {
    static constexpr int NC = CIN / 8;
    static constexpr int ABS = (TH + 2) * TW * 16;        // one block (SW = false)
    static constexpr int CPY = NC * ABS;                  // one shifted copy
    static constexpr int ABYTES = 3 * CPY;
    static_assert(!SW || CIN == 32, "64-byte rows hold 32 channels");
    __device__ __forceinline__ static int off(int s, int c, int hr, int x) {
        const int row = hr * TW + x;
        if constexpr (SW) return s * CPY + row * 64 + ((c ^ ((row >> 1) & 3)) << 4);
        else return (s * NC + c) * ABS + row * 16;
    }
};

template <int CIN, int COUT>
struct TcConv {
    static constexpr int NC = CIN / 8;
    static constexpr bool SW = CIN == 32;
    using L = HaloLayout<CIN, SW>;
    static constexpr int ABS = L::ABS;
    static constexpr int CPY = L::CPY;
    static constexpr int ALIGN = SW ? 1024 : 128;                  // swizzle atoms / TMA destinations
    static constexpr int BBYTES = 9 * NC * COUT * 16;
    static constexpr int ABYTES = L::ABYTES;                       // one A buffer
    static constexpr int NBUF = 3;                                 // A buffers (TMA two tiles ahead)
    static constexpr int SMEM = ALIGN + BBYTES + NBUF * ABYTES + 96 + COUT * 4;
    static constexpr int TMEM_COLS = 128;                          // two accumulator sets of 2 x 32 columns
    static constexpr int THREADS = 288;                            // 8 worker warps + 1 control warp
    // wrap-around pieces of a tile: halo rows 0 and TH + 1 (TW + 2 columns each), then halo
    // columns 0 and TW + 1 (all TH + 2 rows: a corner is wrong whenever its row or its
    // column lies outside the sub-grid), each NC 16-byte chunks
    static constexpr int NROWP = 2 * (TW + 2) * NC;
    static constexpr int NFIX = NROWP + 2 * (TH + 2) * NC;
    static constexpr int NFIXK = (NFIX + 255) / 256;              // per worker thread (256 workers)
    static_assert(CPY % ALIGN == 0 && BBYTES % ALIGN == 0 && ABS % 128 == 0, "aligned TMA destinations");
    static_assert(TW == 32 && TH == 8, "two M = 128 blocks of four 32-pixel rows");
    static_assert(COUT == 16 || COUT == 32, "N = 16 or 32");
};

constexpr uint64_t TC_WAIT_NS = 1000000000ull;  // 1 s bound on any TMA or MMA completion wait

// wrap-around piece j of a tile at a sub-grid edge: its halo position (packed hr | hx << 8 |
// c << 16, or -1 when the tile does not need it) and its 16 bytes of input
template <int CIN>
__device__ __forceinline__ int tc_fix_piece(const bf16* __restrict__ in, const TileMap& tm, int b, int H, int W,
                                            int j, uint4& val) {
    constexpr int NC = CIN / 8;
    constexpr int NROWP = 2 * (TW + 2) * NC;
    int hr, hx, c;
    bool need;
    if (j < NROWP) {
        const int r = j / ((TW + 2) * NC), rem = j - r * ((TW + 2) * NC);
        hx = rem / NC;
        c = rem - hx * NC;
        hr = r ? TH + 1 : 0;
        need = r ? (tm.Y0 + TH == tm.Hs) : (tm.Y0 == 0);
    } else {
        const int jj = j - NROWP;
        const int e = jj / ((TH + 2) * NC), rem = jj - e * ((TH + 2) * NC);
        hr = rem / NC;
        c = rem - hr * NC;
        hx = e ? TW + 1 : 0;
        need = e ? (tm.X0 + TW == tm.Ws) : (tm.X0 == 0);
    }
    if (!need) return -1;
    const int gy = tm.gy(tm.Y0 + hr - 1 + tm.Hs), gx = tm.gx(tm.X0 + hx - 1 + tm.Ws);
    val = __ldg(reinterpret_cast<const uint4*>(in + (((size_t)b * H + gy) * W + gx) * CIN) + c);
    return hr | (hx << 8) | (c << 16);
}

// TMA of a tile's halo into an A buffer (completion on *bar, whose expected byte count the
// caller has raised): one box per shifted copy s and channel chunk c, or with the 64-byte
// swizzle one box of all 32 channels per copy
template <int CIN, bool SW>
__device__ __forceinline__ void tc_issue_halo(const CUtensorMap* map, unsigned char* dst, uint64_t* bar,
                                              const TileMap& tm, int b) {
    using L = HaloLayout<CIN, SW>;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        if constexpr (SW) {
            tc::tma_load_5d(dst + s * L::CPY, map, bar, 0, tm.rx, tm.X0 - 1 + s, tm.ry, b * tm.Hs + tm.Y0 - 1);
        } else {
#pragma unroll
            for (int c = 0; c < L::NC; ++c)
                tc::tma_load_5d(dst + (s * L::NC + c) * L::ABS, map, bar, 8 * c, tm.rx, tm.X0 - 1 + s, tm.ry,
                                b * tm.Hs + tm.Y0 - 1);
        }
    }
}

// this thread's wrap-around pieces of tile t (none for an interior tile); pieces are dealt to
// the 256 threads 0..255 round-robin
template <int CIN, int K>
__device__ __forceinline__ void tc_load_fix(const bf16* __restrict__ in, int t, int tiles_per_img, int H, int W,
                                            int dil, uint4 (&fixv)[K], int (&fixp)[K]) {
    constexpr int NFIX = TcConv<CIN, 16>::NFIX;
    const int b = t / tiles_per_img;
    const TileMap tm = tile_map(t - b * tiles_per_img, H, W, dil);
    const bool edge = tm.Y0 == 0 || tm.Y0 + TH == tm.Hs || tm.X0 == 0 || tm.X0 + TW == tm.Ws;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = threadIdx.x + 256 * k;
        fixp[k] = (edge && j < NFIX) ? tc_fix_piece<CIN>(in, tm, b, H, W, j, fixv[k]) : -1;
    }
}

// the pieces into every shifted copy that holds them
template <int CIN, bool SW, int K>
__device__ __forceinline__ void tc_store_fix(unsigned char* sA, const uint4 (&fixv)[K], const int (&fixp)[K]) {
    using L = HaloLayout<CIN, SW>;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (fixp[k] < 0) continue;
        const int hr = fixp[k] & 255, hx = (fixp[k] >> 8) & 255, c = fixp[k] >> 16;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int x = hx - s;
            if (x >= 0 && x < TW) *reinterpret_cast<uint4*>(sA + L::off(s, c, hr, x)) = fixv[k];
        }
    }
}

// bounded mbarrier wait shared by the warp-specialized kernels: false (and the CTA's abort
// flag and the error word set) once TC_WAIT_NS has passed or another thread has aborted
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* err) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = tc::globaltimer();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (tc::globaltimer() - t0 > TC_WAIT_NS) {
            *abort = 1;
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

// Warp roles: warps 0-7 (workers) patch the wrap-around pieces of each staged tile and drain
// the accumulators (warp w reads TMEM lanes 32 (w % 4).. of M block w / 4); warp 8 (control,
// one lane) issues the TMA loads and the MMAs.  Hand-offs, per tile i of the CTA (buffer
// i % 3, accumulator set i % 2), all through mbarriers:
//   full[b]    TMA bytes landed (expect-tx)         control -> workers
//   fixed[b]   pieces patched (8 warp arrivals)     workers -> control
//   done[s]    MMAs of the set completed (commit)   control -> workers, and buffer b reusable
//   drained[s] accumulators read (8 warp arrivals)  workers -> control
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(288) k_conv3x3_tc(const __grid_constant__ CUtensorMap tmap,
                                                    const bf16* __restrict__ in, const bf16* __restrict__ w,
                                                    const float* __restrict__ bias, void* out,
                                                    const bf16* __restrict__ mask, int H, int W, int dil,
                                                    int tiles_per_img, int B, int* err) {
    using G = TcConv<CIN, COUT>;
    constexpr int NC = G::NC;
    constexpr bool SW = G::SW;
    extern __shared__ unsigned char smraw[];
    unsigned char* sB = smraw + ((G::ALIGN - (tc::smem_u32(smraw) & (G::ALIGN - 1))) & (G::ALIGN - 1));
    unsigned char* sA0 = sB + G::BBYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sA0 + G::NBUF * G::ABYTES);
    uint64_t* fixed = full + 3;
    uint64_t* done = full + 6;
    uint64_t* drained = full + 8;
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(full + 10);
    volatile int* abort = reinterpret_cast<volatile int*>(full + 10) + 1;
    float* s_bias = reinterpret_cast<float*>(full + 12);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = tiles_per_img * B;
    const int G0 = gridDim.x;
    auto issue = [&](int t, int buf) {
        const int b = t / tiles_per_img;
        const TileMap tm = tile_map(t - b * tiles_per_img, H, W, dil);
        tc::mbar_arrive_expect_tx(&full[buf], G::ABYTES);
        tc_issue_halo<CIN, SW>(&tmap, sA0 + buf * G::ABYTES, &full[buf], tm, b);
    };
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) {
            tc::mbar_init(&full[k], 1);
            tc::mbar_init(&fixed[k], 8);
        }
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(&done[k], 1);
            tc::mbar_init(&drained[k], 8);
        }
        *abort = 0;
    }
    if (warp == 8) {
        tc::alloc(s_tmem, G::TMEM_COLS);
        tc::relinquish();
    }
    // weights w[co][tap][ci] -> B: rows (tap, c, co) of 16 bytes, or with the swizzle rows
    // (tap, co) of 64 bytes (chunk c at c ^ ((row >> 1) & 3)); the bias
    for (int i = threadIdx.x; i < COUT * 9 * NC; i += blockDim.x) {
        const int co = i / (9 * NC), r = i - co * (9 * NC);
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(w) + i);
        if constexpr (SW) {
            const int tap = r / NC, c = r - tap * NC, row = tap * COUT + co;
            *reinterpret_cast<uint4*>(sB + row * 64 + ((c ^ ((row >> 1) & 3)) << 4)) = v;
        } else {
            *reinterpret_cast<uint4*>(sB + (r * COUT + co) * 16) = v;
        }
    }
    if (MODE != 2 && threadIdx.x < COUT) s_bias[threadIdx.x] = __ldg(bias + threadIdx.x);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp == 8) {
        // ---------------- control: TMA and MMA issue (lane 0) ----------------
        if (lane == 0) {
            const uint64_t a_desc0 =
                SW ? tc::desc_sw64(tc::smem_u32(sA0)) : tc::desc_noswz(tc::smem_u32(sA0), G::ABS, 128);
            const uint64_t b_desc0 =
                SW ? tc::desc_sw64(tc::smem_u32(sB)) : tc::desc_noswz(tc::smem_u32(sB), COUT * 16, 128);
            constexpr uint32_t IDESC = tc::idesc_bf16(128, COUT);
            int n_tma = 0, n_mma = 0;  // issued
            if ((int)blockIdx.x < total) { issue(blockIdx.x, 0); ++n_tma; }
            if ((int)blockIdx.x + G0 < total) { issue(blockIdx.x + G0, 1); ++n_tma; }
            int i = 0;
            for (int t = blockIdx.x; t < total; t += G0, ++i) {
                const int buf = i % 3, set = i & 1;
                if (!tc_wait(&fixed[buf], (i / 3) & 1, abort, err)) break;
                if (i >= 2 && !tc_wait(&drained[set], ((i - 2) >> 1) & 1, abort, err)) break;
                tc::fence_after();
                const uint64_t a_buf = a_desc0 + (uint64_t)((buf * G::ABYTES) >> 4);
                const uint32_t d_set = tmem + 64 * set;
#pragma unroll 1
                for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int dy = tap / 3, dx = tap - 3 * dy;
#pragma unroll
                        for (int kk = 0; kk < NC / 2; ++kk) {
                            // start addresses advance in 16-byte units in the descriptor's low bits; with
                            // the swizzle, row offsets are whole 8-row atoms and K half kk starts 32 bytes in
                            const int a_off = SW ? dx * G::CPY + (4 * mt + dy) * TW * 64 + 32 * kk
                                                 : (dx * NC + 2 * kk) * G::ABS + (4 * mt + dy) * TW * 16;
                            const int b_off = SW ? tap * COUT * 64 + 32 * kk : (tap * NC + 2 * kk) * COUT * 16;
                            tc::mma_bf16(d_set + 32 * mt, a_buf + (uint64_t)(a_off >> 4),
                                         b_desc0 + (uint64_t)(b_off >> 4), IDESC, (tap | kk) != 0);
                        }
                    }
                }
                tc::commit(&done[set]);
                ++n_mma;
                // the buffer of tile i - 1 takes the TMA of tile i + 2 once that tile's MMAs completed
                if (t + 2 * G0 < total) {
                    if (i >= 1 && !tc_wait(&done[(i - 1) & 1], ((i - 1) >> 1) & 1, abort, err)) break;
                    issue(t + 2 * G0, (i + 2) % 3);
                    ++n_tma;
                }
            }
            if (*abort) {
                // one more bounded wait for everything issued: the last MMA batch and the last two TMAs
                if (n_mma > 0) tc::mbar_wait(&done[(n_mma - 1) & 1], ((n_mma - 1) >> 1) & 1, TC_WAIT_NS);
                for (int k = n_tma - 2 < 0 ? 0 : n_tma - 2; k < n_tma; ++k)
                    tc::mbar_wait(&full[k % 3], (k / 3) & 1, TC_WAIT_NS);
            }
        }
        __syncwarp();
    } else {
        // ---------------- workers: wrap-around pieces and epilogue ----------------
        uint4 fixv[G::NFIXK];
        int fixp[G::NFIXK];
        const int q = warp & 3, mt = warp >> 2;
        // this thread's pixel of tile t and, for the input gradient, its ReLU mask (loaded one patch
        // step before the epilogue that uses it)
        auto pixel_of = [&](int t) {
            const int b = t / tiles_per_img;
            const TileMap tm = tile_map(t - b * tiles_per_img, H, W, dil);
            return ((size_t)b * H + tm.gy(tm.Y0 + 4 * mt + q)) * W + tm.gx(tm.X0 + lane);
        };
        uint4 mpre[COUT / 8];
        auto load_mask = [&](int t) {
            if constexpr (MODE == 2) {
                const uint4* mk = reinterpret_cast<const uint4*>(mask + pixel_of(t) * COUT);
#pragma unroll
                for (int j = 0; j < COUT / 8; ++j) mpre[j] = __ldg(mk + j);
            }
        };
        auto epilogue = [&](int t, int set) {
            const int b = t / tiles_per_img;
            const TileMap tm = tile_map(t - b * tiles_per_img, H, W, dil);
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + 64 * set + 32 * mt;
            float v[COUT];
            if constexpr (COUT == 32) {
                uint32_t r[32];
                tc::ld_32x32b_x32(taddr, r);
                tc::wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
            } else {
                uint32_t r[16];
                tc::ld_32x32b_x16(taddr, r);
                tc::wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
            }
            const int y = tm.gy(tm.Y0 + 4 * mt + q), x = tm.gx(tm.X0 + lane);
            const size_t pix = ((size_t)b * H + y) * W + x;
            if (MODE == 1) {
                float* o = reinterpret_cast<float*>(out);
                const size_t plane = (size_t)H * W;
                o[((size_t)b * 2 + 0) * plane + (size_t)y * W + x] = v[0] + s_bias[0];
                o[((size_t)b * 2 + 1) * plane + (size_t)y * W + x] = v[1] + s_bias[1];
            } else {
                uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(out) + pix * COUT);
    #pragma unroll
                for (int j = 0; j < COUT / 8; ++j) {
                    float e[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) e[k] = v[8 * j + k];
                    if (MODE == 0) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) e[k] = fmaxf(e[k] + s_bias[8 * j + k], 0.f);
                    } else if (MODE == 2) {
                        const uint4 m4 = mpre[j];
                        const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const unsigned short h = (unsigned short)(mw[k >> 1] >> (16 * (k & 1)));
                            if (!(__bfloat162float(__ushort_as_bfloat16(h)) > 0.f)) e[k] = 0.f;
                        }
                    }
                    o[j] = make_uint4(pack2(e[0], e[1]), pack2(e[2], e[3]), pack2(e[4], e[5]), pack2(e[6], e[7]));
                }
            }
        };
        if ((int)blockIdx.x < total) tc_load_fix<CIN>(in, blockIdx.x, tiles_per_img, H, W, dil, fixv, fixp);
        int i = 0;
        for (int t = blockIdx.x; t < total; t += G0, ++i) {
            const int buf = i % 3;
            if (!tc_wait(&full[buf], (i / 3) & 1, abort, err)) break;
            tc_store_fix<CIN, SW>(sA0 + buf * G::ABYTES, fixv, fixp);
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&fixed[buf]);
            if (t + G0 < total) tc_load_fix<CIN>(in, t + G0, tiles_per_img, H, W, dil, fixv, fixp);
            if (i >= 1) {
                load_mask(t - G0);
                // tile i - 1: its MMAs have had the whole patch step of tile i to complete
                if (!tc_wait(&done[(i - 1) & 1], ((i - 1) >> 1) & 1, abort, err)) break;
                tc::fence_after();
                epilogue(t - G0, (i - 1) & 1);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&drained[(i - 1) & 1]);
            }
        }
        if (!*abort && i >= 1) {
            load_mask(blockIdx.x + (i - 1) * G0);
            if (tc_wait(&done[(i - 1) & 1], ((i - 1) >> 1) & 1, abort, err)) {
                tc::fence_after();
                epilogue(blockIdx.x + (i - 1) * G0, (i - 1) & 1);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 8) tc::dealloc(tmem, G::TMEM_COLS);
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

// sum of the CTAs' partials in a fixed order: a 256-thread block owns 32 consecutive outputs;
// thread (g, j) adds partials g, g + 8, ... of output j, then the 8 group sums are added in order
__global__ void __launch_bounds__(256) k_wgrad_reduce(const float* __restrict__ partial,
                                                      const float* __restrict__ bpartial, int nparts, int nw, int nb,
                                                      float* dW, float* db) {
    __shared__ float part[8][33];
    const int j = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + j;
    float s = 0.f;
    if (i < nw) {
        for (int p = g; p < nparts; p += 8) s += __ldg(partial + (size_t)p * nw + i);
    } else if (i < nw + nb) {
        for (int p = g; p < nparts; p += 8) s += __ldg(bpartial + (size_t)p * nb + (i - nw));
    }
    part[g][j] = s;
    __syncthreads();
    if (g == 0 && i < nw + nb) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += part[k][j];
        if (i < nw) dW[i] = t;
        else db[i - nw] = t;
    }
}

// ---------------------------------------------------------------------------
// weight gradient on the tcgen05 tensor cores (CIN = 32), operands staged by TMA:
// D[m][co] = sum_p A[m][p] dz[p][co] with M rows m = (dx, ci) of one dy, i.e.
// the taps (dy, 0..2) times 32 input channels, and K = the pixels of the CTA's
// tiles.  Both operands are MN-major (one row per pixel holding consecutive M or
// N elements), which is the NHWC layout itself.  A is the forward kernel's three
// column-shifted halo copies in the 64-byte-swizzled layout: a copy's 64-byte
// rows hold the 32 channels, so the four 32-element M groups of an M block are
// copies s = 0..3 (LBO = the copy size) and 8-pixel K groups are 512 bytes apart
// (SBO); the row offset dy selects the tap row.  Copy s = 3 is a constant block
// of ones, so M rows 96..127 of the dy = 0 block accumulate sum_p dz[p][co], the
// bias gradient.  dz of a tile is one TMA box of (TH x TW pixels x 32 channels)
// with the same swizzle (COUT = 32) or two 8-channel boxes without swizzle
// (COUT = 16; LBO = 128 along K, SBO = TH TW 16 between the 8-channel groups).
// Three accumulators (dy = 0, 1, 2) of N = COUT columns stay in TMEM over all of
// the CTA's tiles and are written once as the CTA's partial sums (reduced by
// k_wgrad_reduce).  Warp roles and hand-offs as in k_conv3x3_tc, two stages:
// full[b] (TMA landed), fixed[b] (pieces patched), done[b] (MMAs of the tile in
// buffer b completed, so the buffer takes the TMA two tiles ahead).
// ---------------------------------------------------------------------------
template <int COUT>
struct TcWgrad {
    static constexpr int CIN = 32, NC = 4;
    using L = HaloLayout<32, true>;
    static constexpr bool DSW = COUT == 32;                       // dz swizzled
    static constexpr int DBS = TH * TW * 16;                      // one 8-channel dz block (COUT = 16)
    static constexpr int ABLK = 4 * L::CPY;                       // three shifted copies + the ones copy
    static constexpr int DZB = TH * TW * COUT * 2;
    static constexpr int STAGE = ABLK + DZB;                      // one buffer: A then dz
    static constexpr int TXBYTES = 3 * L::CPY + DZB;
    static constexpr int NBUF = 2;
    static constexpr int SMEM = 1024 + NBUF * STAGE + 96;
    static constexpr int TMEM_COLS = 128;
    static constexpr int THREADS = 288;
    static constexpr int NFIXK = (TcConv<32, 16>::NFIX + 255) / 256;
    static_assert(STAGE % 1024 == 0 && L::CPY % 1024 == 0, "swizzle atoms aligned");
};

template <int COUT>
__global__ void __launch_bounds__(288) k_wgrad_tc(const __grid_constant__ CUtensorMap amap,
                                                  const __grid_constant__ CUtensorMap dzmap,
                                                  const bf16* __restrict__ a, float* partial, float* bpartial,
                                                  int H, int W, int B, int dil, int* err) {
    using G = TcWgrad<COUT>;
    using L = typename G::L;
    constexpr int CIN = 32;
    extern __shared__ unsigned char smraw[];
    unsigned char* s0 = smraw + ((1024u - (tc::smem_u32(smraw) & 1023u)) & 1023u);
    uint64_t* full = reinterpret_cast<uint64_t*>(s0 + G::NBUF * G::STAGE);
    uint64_t* fixed = full + 2;
    uint64_t* done = full + 4;
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(full + 6);
    volatile int* abort = reinterpret_cast<volatile int*>(full + 6) + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_per_img = (H / TH) * (W / TW), total = tiles_per_img * B;
    const int G0 = gridDim.x;
    auto issue = [&](int t, int buf) {
        const int b = t / tiles_per_img;
        const TileMap tm = tile_map(t - b * tiles_per_img, H, W, dil);
        unsigned char* st = s0 + buf * G::STAGE;
        tc::mbar_arrive_expect_tx(&full[buf], G::TXBYTES);
        tc_issue_halo<CIN, true>(&amap, st, &full[buf], tm, b);
        if constexpr (G::DSW) {
            tc::tma_load_5d(st + G::ABLK, &dzmap, &full[buf], 0, tm.rx, tm.X0, tm.ry, b * tm.Hs + tm.Y0);
        } else {
#pragma unroll
            for (int c = 0; c < COUT / 8; ++c)
                tc::tma_load_5d(st + G::ABLK + c * G::DBS, &dzmap, &full[buf], 8 * c, tm.rx, tm.X0, tm.ry,
                                b * tm.Hs + tm.Y0);
        }
    };
    if (threadIdx.x == 0) {
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(&full[k], 1);
            tc::mbar_init(&fixed[k], 8);
            tc::mbar_init(&done[k], 1);
        }
        *abort = 0;
    }
    if (warp == 8) {
        tc::alloc(s_tmem, G::TMEM_COLS);
        tc::relinquish();
    }
    // the ones copies (s = 3) of both buffers: BF16 1.0 = 0x3F80 (constant, so the swizzle is moot)
    for (int i = threadIdx.x; i < G::NBUF * L::CPY / 16; i += blockDim.x) {
        const int buf = i / (L::CPY / 16), r = i - buf * (L::CPY / 16);
        *reinterpret_cast<uint4*>(s0 + buf * G::STAGE + 3 * L::CPY + r * 16) =
            make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *s_tmem;
    int n_tiles = 0;  // tiles of this CTA
    for (int t = blockIdx.x; t < total; t += G0) ++n_tiles;

    if (warp == 8) {
        // ---------------- control: TMA and MMA issue (lane 0) ----------------
        if (lane == 0) {
            // MN-major with the 64-byte swizzle: LBO = the step between 32-element M groups (copies),
            // SBO = 512 between 8-pixel K groups; without swizzle: LBO = 128 along K, SBO between
            // 8-element N groups
            auto desc_sw64_mn = [](uint32_t saddr, uint32_t lbo) {
                return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
                       ((uint64_t)(512 >> 4) << 32) | (1ull << 46) | (4ull << 61);
            };
            const uint64_t a_desc0 = desc_sw64_mn(tc::smem_u32(s0), L::CPY);
            const uint64_t d_desc0 = G::DSW ? desc_sw64_mn(tc::smem_u32(s0 + G::ABLK), G::DZB)
                                            : tc::desc_noswz(tc::smem_u32(s0 + G::ABLK), 128, G::DBS);
            constexpr uint32_t IDESC = tc::idesc_bf16(128, COUT) | (1u << 15) | (1u << 16);
            int n_tma = 0, n_mma = 0;
            if (n_tiles > 0) { issue(blockIdx.x, 0); ++n_tma; }
            if (n_tiles > 1) { issue(blockIdx.x + G0, 1); ++n_tma; }
            for (int i = 0; i < n_tiles; ++i) {
                const int buf = i & 1;
                if (!tc_wait(&fixed[buf], (i >> 1) & 1, abort, err)) break;
                tc::fence_after();
                const uint64_t a_st = a_desc0 + (uint64_t)((buf * G::STAGE) >> 4);
                const uint64_t d_st = d_desc0 + (uint64_t)((buf * G::STAGE) >> 4);
#pragma unroll 1
                for (int dy = 0; dy < 3; ++dy) {
#pragma unroll 4
                    for (int ks = 0; ks < TH * TW / 16; ++ks) {
                        // K slice ks: 16 pixels of tile row r = ks / 2 from column x0 = 16 (ks & 1)
                        const int r = ks >> 1, x0 = (ks & 1) * 16;
                        const int a_off = ((r + dy) * TW + x0) * 64;
                        const int d_off = (r * TW + x0) * (G::DSW ? 64 : 16);
                        tc::mma_bf16(tmem + 32 * dy, a_st + (uint64_t)(a_off >> 4), d_st + (uint64_t)(d_off >> 4),
                                     IDESC, (i | ks) != 0);
                    }
                }
                tc::commit(&done[buf]);
                ++n_mma;
                if (i + 2 < n_tiles) {
                    if (!tc_wait(&done[buf], (i >> 1) & 1, abort, err)) break;
                    issue(blockIdx.x + (i + 2) * G0, buf);
                    ++n_tma;
                }
            }
            if (*abort) {
                if (n_mma > 0) tc::mbar_wait(&done[(n_mma - 1) & 1], ((n_mma - 1) >> 1) & 1, TC_WAIT_NS);
                for (int k = n_tma - 2 < 0 ? 0 : n_tma - 2; k < n_tma; ++k)
                    tc::mbar_wait(&full[k & 1], (k >> 1) & 1, TC_WAIT_NS);
            }
        }
        __syncwarp();
    } else {
        // ---------------- workers: wrap-around pieces, then the partial sums ----------------
        uint4 fixv[G::NFIXK];
        int fixp[G::NFIXK];
        if (n_tiles > 0) tc_load_fix<CIN>(a, blockIdx.x, tiles_per_img, H, W, dil, fixv, fixp);
        for (int i = 0; i < n_tiles; ++i) {
            const int buf = i & 1;
            if (!tc_wait(&full[buf], (i >> 1) & 1, abort, err)) break;
            tc_store_fix<CIN, true>(s0 + buf * G::STAGE, fixv, fixp);
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&fixed[buf]);
            if (i + 1 < n_tiles) tc_load_fix<CIN>(a, blockIdx.x + (i + 1) * G0, tiles_per_img, H, W, dil, fixv, fixp);
        }
        // the last batch's commit completes after every earlier MMA of this thread
        if (!*abort && n_tiles > 0 && tc_wait(&done[(n_tiles - 1) & 1], ((n_tiles - 1) >> 1) & 1, abort, err)) {
            tc::fence_after();
            // warp w: lane quarter q = w % 4 holds M rows 32 q + lane = (dx = q, ci = lane); warps 0-3
            // drain the dy = 0 and dy = 2 accumulators, warps 4-7 the dy = 1 one
            const int q = warp & 3;
            float* P = partial + (size_t)blockIdx.x * COUT * 9 * CIN;
            for (int dy = warp >> 2; dy < 3; dy += 2) {
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + 32 * dy;
                float v[COUT];
                if constexpr (COUT == 32) {
                    uint32_t r[32];
                    tc::ld_32x32b_x32(taddr, r);
                    tc::wait_ld();
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
                } else {
                    uint32_t r[16];
                    tc::ld_32x32b_x16(taddr, r);
                    tc::wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
                }
                if (q < 3) {
                    const int tap = 3 * dy + q;
#pragma unroll
                    for (int co = 0; co < COUT; ++co) P[(co * 9 + tap) * CIN + lane] = v[co];
                } else if (dy == 0 && lane == 0) {
#pragma unroll
                    for (int co = 0; co < COUT; ++co) bpartial[(size_t)blockIdx.x * COUT + co] = v[co];
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 8) tc::dealloc(tmem, G::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// weight and bias gradient of layer 0 (2 real input channels, stored padded to 16):
// 18 products per pixel and output channel, far from a dense contraction, so CUDA
// cores.  Thread (co, r) of a 32 x TH block keeps dW[co][tap][0..1] for all 9 taps
// in registers and walks the TW pixels of tile row r: one dz load, nine broadcast
// float2 halo loads and 18 FMAs per pixel.  Partials per CTA are summed over the
// rows in a fixed order and written as [co][tap][2] and [co] (k_wgrad_reduce_l0).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_wgrad_l0(const bf16* __restrict__ a, const bf16* __restrict__ dz,
                                                  float* partial, float* bpartial, int H, int W, int B, int dil) {
    constexpr int COUT = 32, CS = 16;  // output channels; stored input channels per pixel
    __shared__ float2 s_a[(TH + 2) * (TW + 2)];
    // dz of the tile, then (after the tile loop) the per-row partial sums
    __shared__ float s_buf[TH * TW * (COUT + 1)];
    float(*s_dz)[COUT + 1] = reinterpret_cast<float(*)[COUT + 1]>(s_buf);
    float(*s_red)[COUT][19] = reinterpret_cast<float(*)[COUT][19]>(s_buf);
    static_assert(TH * COUT * 19 <= TH * TW * (COUT + 1), "reduction fits the dz tile");
    const int co = threadIdx.x & 31, r = threadIdx.x >> 5;
    float acc[9][2], bacc = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t][0] = acc[t][1] = 0.f;
    const int per_img = (H / TH) * (W / TW), tiles = per_img * B;
    for (int ti = blockIdx.x; ti < tiles; ti += gridDim.x) {
        const int b = ti / per_img;
        const TileMap tm = tile_map(ti - b * per_img, H, W, dil);
        __syncthreads();
        for (int i = threadIdx.x; i < (TH + 2) * (TW + 2); i += blockDim.x) {
            const int hy = i / (TW + 2), hx = i - hy * (TW + 2);
            const int gy = tm.gy(tm.Y0 + hy - 1 + tm.Hs), gx = tm.gx(tm.X0 + hx - 1 + tm.Ws);
            const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(a + (((size_t)b * H + gy) * W + gx) * CS);
            s_a[i] = make_float2(__bfloat162float(v.x), __bfloat162float(v.y));
        }
        for (int i = threadIdx.x; i < TH * TW * COUT / 8; i += blockDim.x) {
            const int p = i / (COUT / 8), c8 = i - p * (COUT / 8);
            const size_t pix = ((size_t)b * H + tm.gy(tm.Y0 + p / TW)) * W + tm.gx(tm.X0 + (p % TW));
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(dz + pix * COUT) + c8);
            const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                s_dz[p][8 * c8 + 2 * k] = __uint_as_float(w4[k] << 16);
                s_dz[p][8 * c8 + 2 * k + 1] = __uint_as_float(w4[k] & 0xFFFF0000u);
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int x = 0; x < TW; ++x) {
            const float d = s_dz[r * TW + x][co];
            bacc += d;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const float2 av = s_a[(r + dy) * (TW + 2) + x + dx];
                    acc[3 * dy + dx][0] = fmaf(d, av.x, acc[3 * dy + dx][0]);
                    acc[3 * dy + dx][1] = fmaf(d, av.y, acc[3 * dy + dx][1]);
                }
        }
    }
    __syncthreads();  // every thread is done with the last dz tile
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        s_red[r][co][2 * t] = acc[t][0];
        s_red[r][co][2 * t + 1] = acc[t][1];
    }
    s_red[r][co][18] = bacc;
    __syncthreads();
    for (int i = threadIdx.x; i < COUT * 19; i += blockDim.x) {
        const int c = i / 19, k = i - c * 19;
        float v = 0.f;
        for (int rr = 0; rr < TH; ++rr) v += s_red[rr][c][k];
        if (k < 18) partial[(size_t)blockIdx.x * COUT * 18 + c * 18 + k] = v;
        else bpartial[(size_t)blockIdx.x * COUT + c] = v;
    }
}

// layer 0's partials [part][co][tap][2] -> gW [co][tap][16] (channels 2..15 stay zero), gb [co]
__global__ void k_wgrad_reduce_l0(const float* __restrict__ partial, const float* __restrict__ bpartial, int nparts,
                                  float* gW, float* gb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 32 * 18) {
        float v = 0.f;
        for (int p = 0; p < nparts; ++p) v += partial[(size_t)p * 32 * 18 + i];
        const int co = i / 18, k = i - co * 18, tap = k >> 1, ci = k & 1;
        gW[(co * 9 + tap) * 16 + ci] = v;
    } else if (i < 32 * 18 + 32) {
        const int c = i - 32 * 18;
        float v = 0.f;
        for (int p = 0; p < nparts; ++p) v += bpartial[(size_t)p * 32 + c];
        gb[c] = v;
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
    int conv_kind;             // REG_CONV_TCGEN05 or REG_CONV_MMA_SYNC
    int tc_grid[2][2][3];      // persistent grid of k_conv3x3_tc<CIN 16/32, COUT 16/32, MODE>
    int tc_wgrad_grid[2];      // grid of k_wgrad_tc<COUT 16/32>
    int* d_err;                // set by a tensor-core conv whose MMAs did not complete in time
    int* h_err;                // pinned copy, refreshed at the end of every forward / backward
    bool record;               // keep every layer's output gradient (reg_net_layer_tensor)
    bf16* dz_rec[NLAYER];
    reg_ctx* proj_fine;        // output map on the (2H, 2W) grid of reg_net_forward_fine (created on first use)
    float *coarse_img, *fine_v;  // restricted images (maxB x 2 x H x W), prolonged prediction (maxB x 2 x 2H x 2W)
};

static size_t conv_smem(int cin, int cout) {
    return (size_t)((TH + 2) * (TW + 2) * (cin + 8) + cout * (9 * cin + 8)) * sizeof(bf16);
}
// cuTensorMapEncodeTiled from the driver (resolved once through the runtime)
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

// 5-D view (C, rx, X, ry, Y + (H/d) b) of B NHWC images with C channels: the sub-grid
// (ry, rx) of dilation d is the 3-D box (C, X, Y) at fixed (rx, ry); boxes of 8 channels x TW x rows
static bool halo_tensor_map(CUtensorMap* m, const bf16* act, int C, int d, int H, int W, int B, int rows = TH + 2,
                            bool sw64 = false) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    const cuuint64_t e = sizeof(bf16);
    cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)d, (cuuint64_t)(W / d), (cuuint64_t)d, (cuuint64_t)(H / d) * B};
    cuuint64_t strides[4] = {C * e, (cuuint64_t)d * C * e, (cuuint64_t)W * C * e, (cuuint64_t)d * W * C * e};
    // boxes of 8 channels (16-byte rows), or of all 32 channels with the 64-byte swizzle
    cuuint32_t box[5] = {sw64 ? 32u : 8u, 1, TW, 1, (cuuint32_t)rows};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    if (sw64 && C != 32) return false;
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(act), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, sw64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int CIN, int COUT, int MODE>
static bool conv_launch(reg_net* n, const bf16* in, const bf16* w, const float* bias, void* out, const bf16* mask,
                        int B, int d) {
    const int tiles = (n->H / TH) * (n->W / TW);
    if (n->conv_kind == REG_CONV_TCGEN05) {
        CUtensorMap map;
        if (!halo_tensor_map(&map, in, CIN, d, n->H, n->W, B, TH + 2, TcConv<CIN, COUT>::SW)) return false;
        const int total = tiles * B;
        int grid = n->tc_grid[CIN == 32][COUT == 32][MODE];
        if (grid > total) grid = total;
        k_conv3x3_tc<CIN, COUT, MODE><<<grid, TcConv<CIN, COUT>::THREADS, TcConv<CIN, COUT>::SMEM, n->stream>>>(
            map, in, w, bias, out, mask, n->H, n->W, d, tiles, B, n->d_err);
    } else {
        k_conv3x3<CIN, COUT, MODE><<<dim3(tiles, B), 256, conv_smem(CIN, COUT), n->stream>>>(in, w, bias, out, mask,
                                                                                           n->H, n->W, d);
    }
    return true;
}

// weight and bias gradient partials of a CIN = 32 layer on the tensor cores; returns the
// number of partials (CTAs), 0 if the tensor maps could not be encoded
template <int COUT>
static int wgrad_tc_launch(reg_net* n, const bf16* a, const bf16* dz, int B, int d) {
    CUtensorMap am, dm;
    if (!halo_tensor_map(&am, a, 32, d, n->H, n->W, B, TH + 2, true) ||
        !halo_tensor_map(&dm, dz, COUT, d, n->H, n->W, B, TH, TcWgrad<COUT>::DSW))
        return 0;
    const int total = (n->H / TH) * (n->W / TW) * B;
    const int grid = std::min(total, n->tc_wgrad_grid[COUT == 32]);
    k_wgrad_tc<COUT><<<grid, TcWgrad<COUT>::THREADS, TcWgrad<COUT>::SMEM, n->stream>>>(
        am, dm, a, n->partial, n->bpartial, n->H, n->W, B, d, n->d_err);
    return grid;
}

template <int COUT>
static int tc_wgrad_prepare(reg_net* n, int dev) {
    using G = TcWgrad<COUT>;
    auto k = k_wgrad_tc<COUT>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM) != cudaSuccess) return 0;
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return 0;
    // one CTA per SM (the shared memory of two stages); never more CTAs than partial slots
    n->tc_wgrad_grid[COUT == 32] = std::min(pr.multiProcessorCount, n->nwg);
    return 1;
}

// resident CTAs per SM of k_conv3x3_tc<CIN, COUT, MODE> from its registers and shared memory
// and the device limits (at most 512 / TMEM_COLS, the TMEM columns of an SM)
template <int CIN, int COUT, int MODE>
static int tc_prepare(reg_net* n, int dev) {
    using G = TcConv<CIN, COUT>;
    auto k = k_conv3x3_tc<CIN, COUT, MODE>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess)
        return 0;
    cudaFuncAttributes fa;
    cudaDeviceProp pr;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess || cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return 0;
    const int warps = G::THREADS / 32;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    int occ = pr.regsPerMultiprocessor / (regs_warp * warps);
    occ = std::min(occ, (int)(pr.sharedMemPerMultiprocessor / (G::SMEM + fa.sharedSizeBytes + pr.reservedSharedMemPerBlock)));
    occ = std::min(occ, pr.maxThreadsPerMultiProcessor / G::THREADS);
    occ = std::min(occ, 512 / G::TMEM_COLS);
    if (occ < 1) return 0;
    n->tc_grid[CIN == 32][COUT == 32][MODE] = occ * pr.multiProcessorCount;
    return occ;
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
    if (n->proj_fine) reg_destroy(n->proj_fine);
    cudaFree(n->coarse_img);
    cudaFree(n->fine_v);
    void* ptrs[] = {n->d_layers, n->params, n->m1, n->m2, n->gW, n->gb, n->d_gwoff, n->d_gboff, n->d_wfoff,
                    n->wf, n->wt, n->bpad, n->dzA, n->dzB, n->out, n->pred, n->res, n->dout, n->partial,
                    n->bpartial, n->d_part, n->d_err};
    for (void* p : ptrs) cudaFree(p);
    for (int l = 0; l < NLAYER; ++l) {
        cudaFree(n->act[l]);
        cudaFree(n->dz_rec[l]);
    }
    cudaFreeHost(n->h_part);
    cudaFreeHost(n->h_err);
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
    M((void**)&n->d_err, sizeof(int));
    if (ok && cudaMallocHost((void**)&n->h_part, sizeof(double) * 1024) != cudaSuccess) ok = false;
    if (ok && cudaMallocHost((void**)&n->h_err, sizeof(int)) != cudaSuccess) ok = false;
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
    cudaMemset(n->d_err, 0, sizeof(int));
    *n->h_err = 0;
    n->conv_kind = REG_CONV_TCGEN05;
    int dev = 0;
    cudaGetDevice(&dev);
    const bool tc_ok = tc_prepare<16, 32, 0>(n, dev) && tc_prepare<32, 32, 0>(n, dev) &&
                       tc_prepare<32, 16, 1>(n, dev) && tc_prepare<16, 32, 2>(n, dev) &&
                       tc_prepare<32, 32, 2>(n, dev) && tc_wgrad_prepare<16>(n, dev) &&
                       tc_wgrad_prepare<32>(n, dev) && tmap_encoder() != nullptr;
    if (!tc_ok || cudaDeviceSynchronize() != cudaSuccess) {
        reg_net_destroy(n);
        return reg_fail(REG_ERR_CUDA, "network initialisation failed");
    }
    *out = n;
    return REG_OK;
}

extern "C" int reg_net_set_stream(reg_net* n, void* stream) {
    if (!n) return reg_fail(REG_ERR_ARG, "net is NULL");
    n->stream = (cudaStream_t)stream;
    if (n->proj_fine) {
        const int st = reg_set_stream(n->proj_fine, stream);
        if (st != REG_OK) return st;
    }
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

// a tensor-core conv of an earlier call that reported an MMA timeout (sticky; read from
// the pinned copy, refreshed at the end of every forward pass)
static int conv_status(reg_net* n) {
    return *n->h_err ? reg_fail(REG_ERR_TIMEOUT, "tensor-core convolution: MMA completion timed out") : REG_OK;
}

static int net_forward(reg_net* n, const float* images, int B) {
    const int H = n->H, W = n->W;
    int st = conv_status(n);
    if (st != REG_OK) return st;
    k_pack_input<<<304, 256, 0, n->stream>>>(images, n->act[0], B, H, W);
    for (int l = 0; l < NLAYER; ++l) {
        const float* bias = n->bpad + 32 * l;
        const bf16* wl = n->wf + n->wfoff[l];
        const int d = layer_dil(l, H, W);
        bool ok;
        if (l == 0)
            ok = conv_launch<16, 32, 0>(n, n->act[0], wl, bias, n->act[1], nullptr, B, d);
        else if (l < NLAYER - 1)
            ok = conv_launch<32, 32, 0>(n, n->act[l], wl, bias, n->act[l + 1], nullptr, B, d);
        else
            ok = conv_launch<32, 16, 1>(n, n->act[l], wl, bias, n->out, nullptr, B, d);
        if (!ok) return reg_fail(REG_ERR_CUDA, "net forward: tensor map encoding failed");
    }
    cudaMemcpyAsync(n->h_err, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream);
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
    const float invM = 1.0f / (float)M;
    bf16* dz = n->dzA;
    bf16* dnext = n->dzB;
    for (int l = NLAYER - 1; l >= 0; --l) {
        const LayerDesc& L = n->layers[l];
        float* gWl = n->gW + n->gwoff[l];
        float* gbl = n->gb + n->gboff[l];
        const int d = layer_dil(l, H, W);
        if (n->record)
            cudaMemcpyAsync(n->dz_rec[l], dz, sizeof(bf16) * (size_t)B * H * W * L.coutp, cudaMemcpyDeviceToDevice,
                            n->stream);
        int nparts = n->nwg;
        if (l > 0 && n->conv_kind == REG_CONV_TCGEN05) {
            nparts = l == NLAYER - 1 ? wgrad_tc_launch<16>(n, n->act[l], dz, B, d) : wgrad_tc_launch<32>(n, n->act[l], dz, B, d);
            if (nparts == 0) return reg_fail(REG_ERR_CUDA, "net backward: tensor map encoding failed");
        } else if (l == NLAYER - 1) {
            k_wgrad<32, 16><<<n->nwg, 288, wgrad_smem(32, 16), n->stream>>>(n->act[l], dz, n->partial, n->bpartial, H, W, B, d);
        } else if (l > 0) {
            k_wgrad<32, 32><<<n->nwg, 288, wgrad_smem(32, 32), n->stream>>>(n->act[l], dz, n->partial, n->bpartial, H, W, B, d);
        } else if (n->conv_kind == REG_CONV_TCGEN05) {
            // layer 0 (2 real input channels): CUDA-core kernel, its own partial layout
            k_wgrad_l0<<<n->nwg, 256, 0, n->stream>>>(n->act[0], dz, n->partial, n->bpartial, H, W, B, d);
            k_wgrad_reduce_l0<<<3, 256, 0, n->stream>>>(n->partial, n->bpartial, n->nwg, gWl, gbl);
            nparts = 0;
        } else {
            k_wgrad<16, 32><<<n->nwg, 288, wgrad_smem(16, 32), n->stream>>>(n->act[0], dz, n->partial, n->bpartial, H, W, B, d);
        }
        const int nw = L.coutp * 9 * L.cinp, nb = L.coutp;
        if (nparts > 0)
            k_wgrad_reduce<<<(nw + nb + 31) / 32, 256, 0, n->stream>>>(n->partial, n->bpartial, nparts, nw, nb, gWl, gbl);
        if (l > 0) {
            // input gradient through the ReLU of layer l-1: correlation with the flipped, transposed kernel
            const bf16* wtl = n->wt + n->wfoff[l];
            const bool ok = l == NLAYER - 1 ? conv_launch<16, 32, 2>(n, dz, wtl, nullptr, dnext, n->act[l], B, d)
                                            : conv_launch<32, 32, 2>(n, dz, wtl, nullptr, dnext, n->act[l], B, d);
            if (!ok) return reg_fail(REG_ERR_CUDA, "net backward: tensor map encoding failed");
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
    cudaMemcpyAsync(n->h_err, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream);
    e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("net backward: ") + cudaGetErrorString(e));
    st = conv_status(n);
    if (st != REG_OK) return st;
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

extern "C" int reg_net_set_conv_kernel(reg_net* n, int kind) {
    if (!n) return reg_fail(REG_ERR_ARG, "net is NULL");
    if (kind != REG_CONV_TCGEN05 && kind != REG_CONV_MMA_SYNC) return reg_fail(REG_ERR_ARG, "unknown conv kernel");
    n->conv_kind = kind;
    return REG_OK;
}

extern "C" int reg_net_set_record(reg_net* n, int on) {
    if (!n) return reg_fail(REG_ERR_ARG, "net is NULL");
    if (on && !n->record) {
        const size_t pix = (size_t)n->maxB * n->H * n->W;
        for (int l = 0; l < NLAYER; ++l)
            if (!n->dz_rec[l] && cudaMalloc((void**)&n->dz_rec[l], sizeof(bf16) * pix * n->layers[l].coutp) != cudaSuccess) {
                cudaGetLastError();
                return reg_fail(REG_ERR_NOMEM, "record buffers");
            }
    }
    n->record = on != 0;
    return REG_OK;
}

namespace {
// NHWC BF16 with cs channels per pixel -> planar FP32 [B][c][H][W], first c channels
__global__ void k_unpack_nhwc(const bf16* __restrict__ a, float* __restrict__ out, int cs, int c, long long npix,
                              long long plane) {
    const long long total = npix * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / c;
        const int ch = (int)(i - p * c);
        const long long b = p / plane, r = p - b * plane;
        out[(b * c + ch) * plane + r] = __bfloat162float(a[p * cs + ch]);
    }
}
}  // namespace

extern "C" int reg_net_layer_tensor(reg_net* n, int kind, int layer, int B, float* out) {
    if (!n || !out) return reg_fail(REG_ERR_ARG, "net or out is NULL");
    if (layer < 0 || layer >= NLAYER || B < 1 || B > n->maxB) return reg_fail(REG_ERR_ARG, "layer or batch out of range");
    const LayerDesc& L = n->layers[layer];
    const long long plane = (long long)n->H * n->W, npix = plane * B;
    const bf16* src = nullptr;
    int cs = 0, c = 0;
    if (kind == REG_NET_INPUT) {
        src = n->act[layer]; cs = L.cinp; c = L.cin;
    } else if (kind == REG_NET_OUTPUT) {
        if (layer == NLAYER - 1) {
            const cudaError_t e = cudaMemcpyAsync(out, n->out, sizeof(float) * 2 * npix, cudaMemcpyDeviceToDevice, n->stream);
            return e == cudaSuccess ? REG_OK : reg_fail(REG_ERR_CUDA, cudaGetErrorString(e));
        }
        src = n->act[layer + 1]; cs = L.coutp; c = L.cout;
    } else if (kind == REG_NET_OUTPUT_GRAD) {
        if (!n->record) return reg_fail(REG_ERR_ARG, "output gradients are kept only after reg_net_set_record(net, 1)");
        src = n->dz_rec[layer]; cs = L.coutp; c = L.cout;
    } else {
        return reg_fail(REG_ERR_ARG, "unknown tensor kind");
    }
    k_unpack_nhwc<<<304, 256, 0, n->stream>>>(src, out, cs, c, npix, plane);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? REG_OK : reg_fail(REG_ERR_CUDA, cudaGetErrorString(e));
}

namespace {
// (B, 2, 2H, 2W) -> (B, 2, H, W): full weighting, weights 1/4, 1/2, 1/4 along each axis around
// fine node (2i, 2j), periodic
__global__ void k_restrict2(const float* __restrict__ f, float* __restrict__ c, int planes, int H, int W) {
    const int Hf = 2 * H, Wf = 2 * W;
    const long long total = (long long)planes * H * W;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long pl = idx / ((long long)H * W);
        const int r = (int)(idx - pl * H * W), i = r / W, j = r - i * W;
        const float* fp = f + pl * (long long)Hf * Wf;
        const float wgt[3] = {0.25f, 0.5f, 0.25f};
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int y = (2 * i + a - 1 + Hf) & (Hf - 1);
            float row = 0.f;
#pragma unroll
            for (int b = 0; b < 3; ++b) row += wgt[b] * fp[(long long)y * Wf + ((2 * j + b - 1 + Wf) & (Wf - 1))];
            acc += wgt[a] * row;
        }
        c[idx] = acc;
    }
}

// (B, 2, H, W) -> (B, 2, 2H, 2W): bilinear, periodic; fine node (y, x) sits at coarse (y / 2, x / 2)
__global__ void k_prolong2(const float* __restrict__ c, float* __restrict__ f, int planes, int H, int W) {
    const int Hf = 2 * H, Wf = 2 * W;
    const long long total = (long long)planes * Hf * Wf;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long pl = idx / ((long long)Hf * Wf);
        const int r = (int)(idx - pl * Hf * Wf), y = r / Wf, x = r - y * Wf;
        const float* cp = c + pl * (long long)H * W;
        const int i0 = y >> 1, j0 = x >> 1, i1 = (i0 + 1) & (H - 1), j1 = (j0 + 1) & (W - 1);
        const float ty = 0.5f * (y & 1), tx = 0.5f * (x & 1);
        f[idx] = (1.f - ty) * ((1.f - tx) * cp[i0 * W + j0] + tx * cp[i0 * W + j1]) +
                 ty * ((1.f - tx) * cp[i1 * W + j0] + tx * cp[i1 * W + j1]);
    }
}
}  // namespace

extern "C" int reg_net_forward_fine(reg_net* n, const float* images, int B, float* v_out) {
    if (!n || !images || !v_out) return reg_fail(REG_ERR_ARG, "NULL argument");
    if (B < 1 || B > n->maxB) return reg_fail(REG_ERR_ARG, "batch out of range");
    const int H = n->H, W = n->W, Hf = 2 * H, Wf = 2 * W;
    if (Hf > 1024 || Wf > 1024) return reg_fail(REG_ERR_ARG, "the fine grid (2H, 2W) must fit [16, 1024]");
    if (!n->proj_fine) {
        reg_ctx* pf = nullptr;
        int st = reg_create(reg_grid{Hf, Wf}, 1, REG_H1, 1.0, INFINITY, 0.0, &pf);
        if (st != REG_OK) return st;
        st = reg_set_stream(pf, n->stream);
        if (st != REG_OK) {
            reg_destroy(pf);
            return st;
        }
        const size_t pix = (size_t)n->maxB * H * W;
        if (cudaMalloc((void**)&n->coarse_img, sizeof(float) * 2 * pix) != cudaSuccess ||
            cudaMalloc((void**)&n->fine_v, sizeof(float) * 8 * pix) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(n->coarse_img);
            n->coarse_img = nullptr;
            reg_destroy(pf);
            return reg_fail(REG_ERR_NOMEM, "fine-grid warm-start buffers");
        }
        n->proj_fine = pf;
    }
    k_restrict2<<<304, 256, 0, n->stream>>>(images, n->coarse_img, 2 * B, H, W);
    int st = net_forward(n, n->coarse_img, B);  // n->pred = P G net(x) on the H x W grid
    if (st != REG_OK) return st;
    k_prolong2<<<304, 256, 0, n->stream>>>(n->pred, n->fine_v, 2 * B, H, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, cudaGetErrorString(e));
    // the fine grid's own output map P G (sigma = 2 h of that grid), then the output scale
    const size_t ff = (size_t)2 * Hf * Wf;
    const double sigma = 2.0 * (2.0 * M_PI / (double)(Hf > Wf ? Hf : Wf));
    for (int b = 0; b < B; ++b) {
        st = apply_smooth_proj(n->proj_fine, (float)(0.5 * sigma * sigma), n->fine_v + b * ff, v_out + b * ff);
        if (st != REG_OK) return st;
    }
    if (n->out_scale != 1.f) launch_axpby(n->proj_fine, (long long)B * ff, n->out_scale, v_out, 0.f, v_out, -1, -1, v_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? REG_OK : reg_fail(REG_ERR_CUDA, cudaGetErrorString(e));
}
