// Autotuner of the FFT tile choices (row a15).  The row kernels process R
// grid rows per CTA and the column kernels C spectrum columns per CTA; the
// best pair depends on the grid (CTA count against the 152 SMs, threads per
// CTA, shared memory per CTA) and is found by timing the Gauss-Newton Hessian
// matvec (the incremental state and adjoint transports, Algorithm 2) for every
// valid pair.  Results live in a process-wide table per (device, n1, n2);
// contexts created afterwards on that device and grid use them.
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tune;

bool pow2_grid(int n) { return n >= 16 && n <= 1024 && (n & (n - 1)) == 0; }

// Mean milliseconds of one Hessian matvec with tiles (R, C); < 0 on failure.
double time_matvec(reg_grid grid, int nt, int R, int C, float* mT, float* mR, float* v, float* out,
                   cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
    reg_ctx* c = nullptr;
    if (reg_create(grid, nt, REG_H1, 1e-3, INFINITY, 0.0, &c) != REG_OK) return -1.0;
    c->tileR = R;
    c->tileC = C;
    double ms = -1.0;
    bool ok = reg_set_stream(c, st) == REG_OK && reg_set_images(c, mT, mR) == REG_OK &&
              reg_gradient(c, v, out, nullptr) == REG_OK;
    for (int i = 0; ok && i < 2; ++i) ok = reg_hessian_matvec(c, v, out) == REG_OK;
    const int reps = 3;
    if (ok && cudaEventRecord(e0, st) == cudaSuccess) {
        for (int i = 0; ok && i < reps; ++i) ok = reg_hessian_matvec(c, v, out) == REG_OK;
        float t = 0.f;
        if (ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
            ms = t / reps;
    }
    cudaStreamSynchronize(st);
    reg_destroy(c);
    return ms;
}
}  // namespace

bool tuned_tiles(int dev, int n1, int n2, int* R, int* C) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(dev, n1, n2));
    if (it == g_tune.end()) return false;
    *R = it->second.first;
    *C = it->second.second;
    return true;
}

extern "C" int reg_autotune(reg_grid grid, int nt, int force, int* rows_per_cta, int* cols_per_cta,
                            double* ms_per_matvec) {
    if (!pow2_grid(grid.n1) || !pow2_grid(grid.n2))
        return reg_fail(REG_ERR_ARG, "n1 and n2 must be powers of two in [16, 1024]");
    if (nt < 1 || nt > 4096) return reg_fail(REG_ERR_ARG, "nt must be in [1, 4096]");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    int R = 0, C = 0;
    if (!force && tuned_tiles(dev, grid.n1, grid.n2, &R, &C)) {
        if (rows_per_cta) *rows_per_cta = R;
        if (cols_per_cta) *cols_per_cta = C;
        if (ms_per_matvec) *ms_per_matvec = -1.0;
        return REG_OK;
    }
    std::vector<std::pair<int, int>> cands;
    for (int r = 4; r <= grid.n1; r *= 2)
        for (int c = 2; c <= grid.n2 / 2; c *= 2)
            if (tiles_valid(grid.n1, grid.n2, r, c)) cands.emplace_back(r, c);
    int R0, C0;
    default_tiles(grid.n1, grid.n2, &R0, &C0);
    if (cands.empty()) cands.emplace_back(R0, C0);

    const size_t N = (size_t)grid.n1 * grid.n2;
    float *buf = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&buf, sizeof(float) * 6 * N) != cudaSuccess) {
        cudaGetLastError();
        return reg_fail(REG_ERR_NOMEM, "autotune buffers");
    }
    int status = REG_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemsetAsync(buf, 0, sizeof(float) * 6 * N, st) != cudaSuccess) {
        status = reg_fail(REG_ERR_CUDA, "autotune stream / events");
    }
    // zero images and velocity: every kernel runs its full work, no value can overflow
    float *mT = buf, *mR = buf + N, *v = buf + 2 * N, *out = buf + 4 * N;
    double best = -1.0;
    int bR = R0, bC = C0;
    for (size_t i = 0; status == REG_OK && i < cands.size(); ++i) {
        const double ms = time_matvec(grid, nt, cands[i].first, cands[i].second, mT, mR, v, out, st, e0, e1);
        if (ms < 0.0) {
            status = reg_fail(REG_ERR_CUDA, std::string("autotune candidate failed: ") + reg_last_error());
            break;
        }
        if (best < 0.0 || ms < best) {
            best = ms;
            bR = cands[i].first;
            bC = cands[i].second;
        }
    }
    if (st) cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(buf);
    if (status != REG_OK) return status;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[std::make_tuple(dev, grid.n1, grid.n2)] = std::make_pair(bR, bC);
    }
    if (rows_per_cta) *rows_per_cta = bR;
    if (cols_per_cta) *cols_per_cta = bC;
    if (ms_per_matvec) *ms_per_matvec = best;
    return REG_OK;
}

extern "C" int reg_tile_config(reg_ctx* ctx, int* rows_per_cta, int* cols_per_cta) {
    if (!ctx) return reg_fail(REG_ERR_ARG, "ctx is NULL");
    int R, C;
    default_tiles(ctx->n1, ctx->n2, &R, &C);
    if (rows_per_cta) *rows_per_cta = ctx->tileR > 0 ? ctx->tileR : R;
    if (cols_per_cta) *cols_per_cta = ctx->tileC > 0 ? ctx->tileC : C;
    return REG_OK;
}
