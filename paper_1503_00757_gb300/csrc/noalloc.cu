// Allocation-free spectral gradient (see reg_spectral_grad_static in
// include/reg.h).
//
// Some callers cannot allocate device memory: their device memory is owned
// by another allocator that reserves it up front, or they run where a
// synchronizing cudaMalloc / cudaFree is not acceptable.  This entry point
// needs no context: its scratch (three packed half spectra) and the FFT
// twiddle table live in file-scope __device__ arrays that every GPU which
// loads the library holds until the process exits.  The caller passes the
// input field and the output buffer only.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "fft.cuh"
#include "internal.h"

// Largest grid (n1 * n2 nodes) the static scratch serves: 512 x 512.
#define REG_STATIC_MAX_NODES (512 * 512)

// Scratch of the three packed half spectra (f^, d1 f^, d2 f^): 3 MiB.
static __device__ __align__(256) float2 g_static_scratch[3 * (REG_STATIC_MAX_NODES / 2)];
// Twiddle tables (the layout of fft.cuh), filled at set-up.
static __device__ __align__(256) float2 g_static_twiddles[REG_TW_TOTAL];

namespace {
struct StaticDevice {
    bool ready;
    float2* scratch;  // device address of g_static_scratch on this device
    float2* tw;       // device address of g_static_twiddles on this device
};
constexpr int kMaxDevices = 64;
StaticDevice g_static[kMaxDevices];
std::mutex g_static_mu;

// Once per device, with that device current: resolve the device addresses of
// the file-scope arrays (host code must not use their names as pointers),
// upload the twiddle table and wait for the upload to complete.
int static_setup(int dev) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticDevice& s = g_static[dev];
    if (s.ready) return REG_OK;
    cudaError_t e = cudaGetSymbolAddress((void**)&s.scratch, g_static_scratch);
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress((void**)&s.tw, g_static_twiddles);
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("cudaGetSymbolAddress(twiddles): ") + cudaGetErrorString(e));
    static float2 h[REG_TW_TOTAL];  // under g_static_mu
    fill_twiddles(h);
    e = cudaMemcpyToSymbol(g_static_twiddles, h, sizeof(h));
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("twiddle upload: ") + cudaGetErrorString(e));
    // A copy from pageable host memory may return once the data is staged; the first
    // call's kernels then run on the caller's stream, which need not be ordered after the
    // legacy stream (cudaStreamNonBlocking).  Wait until the table is on the device.
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("twiddle upload (sync): ") + cudaGetErrorString(e));
    s.ready = true;
    return REG_OK;
}

bool pow2_in_range(int n) { return n >= 16 && n <= 1024 && (n & (n - 1)) == 0; }
int ilog2i(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
}  // namespace

extern "C" int reg_spectral_grad_static(reg_grid grid, const float* f, float* grad_f, void* stream) {
    if (!pow2_in_range(grid.n1) || !pow2_in_range(grid.n2))
        return reg_fail(REG_ERR_ARG, "n1 and n2 must be powers of two in [16, 1024]");
    if ((long long)grid.n1 * grid.n2 > REG_STATIC_MAX_NODES)
        return reg_fail(REG_ERR_ARG, "grid exceeds the static scratch of reg_spectral_grad_static (at most 512 x 512 nodes)");
    if (!f || !grad_f) return reg_fail(REG_ERR_ARG, "f and grad_f must not be NULL");
    if ((((uintptr_t)f) & 15) || (((uintptr_t)grad_f) & 15))
        return reg_fail(REG_ERR_ARG, "f and grad_f must be 16-byte aligned");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return reg_fail(REG_ERR_ARG, "device ordinal out of range");
    const int st = static_setup(dev);
    if (st != REG_OK) return st;

    // A context on the stack that points at the static arrays; nothing is allocated.
    reg_ctx c{};
    c.n1 = grid.n1;
    c.n2 = grid.n2;
    c.N = grid.n1 * grid.n2;
    c.log1 = ilog2i(grid.n1);
    c.log2 = ilog2i(grid.n2);
    c.stream = (cudaStream_t)stream;
    c.pdl = true;
    c.tw = g_static[dev].tw;
    const size_t half = (size_t)c.N / 2;
    float2* S0 = g_static[dev].scratch;
    float2* S1 = S0 + half;
    float2* S2 = S1 + half;

    SpecParams P{};
    P.scale = 1.0f / (float)c.N;
    launch_r2c_scalar(&c, f, S0);
    const float2* in[1] = {S0};
    float2* out[2] = {S1, S2};
    launch_col(&c, OP_GRAD, in, out, P, nullptr);
    launch_c2r_vec(&c, S1, S2, grad_f, grad_f + c.N);
    e = cudaGetLastError();
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return REG_OK;
}
