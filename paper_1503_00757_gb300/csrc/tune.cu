// Autotuner of the FFT tile choices.  The row kernels process R
// grid rows per CTA and the column kernels C spectrum columns per CTA, and the
// RK2 row kernels either prefetch their operands before waiting on the
// preceding kernel (P = 1, more registers) or load them after the FFT (P = 0,
// two 512-thread CTAs per SM).  The best choice depends on the grid (CTA count
// against the 152 SMs, threads and shared memory per CTA) and on how many
// solves share the GPU, so it is found by timing the Gauss-Newton Hessian
// matvec (the incremental state and adjoint transports, Algorithm 2) for
// every valid (R, C, P) with a given number of solves running concurrently on
// their own streams, each with and without programmatic dependent launch
// (D): early launch hides one solve's launch latency but lets waiting CTAs
// hold SM resources, and which wins depends on the concurrency.  The
// cluster-resident transport kernel (T = 1) is not a candidate: measured on a
// GB300 it is slower than the row / column kernel pairs at every grid size,
// nt and concurrency tried (reg_set_transport selects it by hand).  Results
// live in a process-wide table per (device, n1, n2); contexts created
// afterwards on that device and grid use them.
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::tuple<int, int, int, int, int>> g_tune;

bool pow2_grid(int n) { return n >= 16 && n <= 1024 && (n & (n - 1)) == 0; }

struct Lane {
    reg_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
};

// Milliseconds per Hessian matvec (throughput over `lanes.size()` concurrent
// solves) with tiles (R, C, P), launch mode D and transport path T; < 0 on failure.
double time_matvec(reg_grid grid, int nt, int R, int C, int P, int D, int T, std::vector<Lane>& lanes, float* mT,
                   float* mR, float* v, float* out, cudaStream_t root, cudaEvent_t e0, cudaEvent_t e1) {
    const size_t N2 = 2 * (size_t)grid.n1 * grid.n2;
    bool ok = true;
    for (size_t i = 0; ok && i < lanes.size(); ++i) {
        Lane& L = lanes[i];
        ok = reg_create(grid, nt, REG_H1, 1e-3, INFINITY, 0.0, &L.ctx) == REG_OK;
        if (!ok) break;
        L.ctx->tileR = R;
        L.ctx->tileC = C;
        L.ctx->tileP = P;
        L.ctx->pdl = D != 0;
        L.ctx->use_tc = T != 0 && L.ctx->tc_ok;
        float* o = out + i * N2;
        ok = reg_set_stream(L.ctx, L.st) == REG_OK && reg_set_images(L.ctx, mT, mR) == REG_OK &&
             reg_gradient(L.ctx, v, o, nullptr) == REG_OK;
        for (int k = 0; ok && k < 2; ++k) ok = reg_hessian_matvec(L.ctx, v, o) == REG_OK;
    }
    const int reps = 4;
    double ms = -1.0;
    for (size_t i = 0; ok && i < lanes.size(); ++i) ok = cudaStreamSynchronize(lanes[i].st) == cudaSuccess;
    if (ok) ok = cudaEventRecord(e0, root) == cudaSuccess;
    for (size_t i = 0; ok && i < lanes.size(); ++i) {
        Lane& L = lanes[i];
        ok = cudaStreamWaitEvent(L.st, e0, 0) == cudaSuccess;
        for (int k = 0; ok && k < reps; ++k) ok = reg_hessian_matvec(L.ctx, v, out + i * N2) == REG_OK;
        if (ok) ok = cudaEventRecord(L.done, L.st) == cudaSuccess && cudaStreamWaitEvent(root, L.done, 0) == cudaSuccess;
    }
    float t = 0.f;
    if (ok && cudaEventRecord(e1, root) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
        ms = t / (reps * (double)lanes.size());
    for (Lane& L : lanes) {
        if (L.st) cudaStreamSynchronize(L.st);
        if (L.ctx) reg_destroy(L.ctx);
        L.ctx = nullptr;
    }
    return ms;
}
}  // namespace

bool tuned_tiles(int dev, int n1, int n2, int* R, int* C, int* P, int* D, int* T) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(dev, n1, n2));
    if (it == g_tune.end()) return false;
    *R = std::get<0>(it->second);
    *C = std::get<1>(it->second);
    *P = std::get<2>(it->second);
    *D = std::get<3>(it->second);
    if (T) *T = std::get<4>(it->second);
    return true;
}

extern "C" int reg_autotune(reg_grid grid, int nt, int concurrency, int force, int* rows_per_cta, int* cols_per_cta,
                            int* prefetch, int* pdl, double* ms_per_matvec) {
    if (!pow2_grid(grid.n1) || !pow2_grid(grid.n2))
        return reg_fail(REG_ERR_ARG, "n1 and n2 must be powers of two in [16, 1024]");
    if (nt < 1 || nt > 4096) return reg_fail(REG_ERR_ARG, "nt must be in [1, 4096]");
    if (concurrency < 1 || concurrency > 16) return reg_fail(REG_ERR_ARG, "concurrency must be in [1, 16]");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    int R = 0, C = 0, P = 0, D = 1;
    if (!force && tuned_tiles(dev, grid.n1, grid.n2, &R, &C, &P, &D, nullptr)) {
        if (rows_per_cta) *rows_per_cta = R;
        if (cols_per_cta) *cols_per_cta = C;
        if (prefetch) *prefetch = P;
        if (pdl) *pdl = D;
        if (ms_per_matvec) *ms_per_matvec = -1.0;
        return REG_OK;
    }
    std::vector<std::tuple<int, int, int, int, int>> cands;
    for (int r = 4; r <= grid.n1; r *= 2)
        for (int c = 2; c <= grid.n2 / 2; c *= 2)
            for (int p = 0; p <= 1; ++p)
                for (int d = 0; d <= 1; ++d)
                    if (tiles_valid(grid.n1, grid.n2, r, c, p)) cands.emplace_back(r, c, p, d, 0);
    int R0, C0, P0;
    default_tiles(grid.n1, grid.n2, &R0, &C0, &P0);
    if (cands.empty()) cands.emplace_back(R0, C0, P0, 1, 0);


    const size_t N = (size_t)grid.n1 * grid.n2;
    const int K = concurrency;
    float* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(float) * (4 + 2 * (size_t)K) * N) != cudaSuccess) {
        cudaGetLastError();
        return reg_fail(REG_ERR_NOMEM, "autotune buffers");
    }
    std::vector<Lane> lanes(K);
    cudaStream_t root = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = REG_OK;
    bool ok = cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    for (Lane& L : lanes)
        ok = ok && cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) == cudaSuccess;
    // zero images and velocity: every kernel runs its full work, no value can overflow
    ok = ok && cudaMemsetAsync(buf, 0, sizeof(float) * (4 + 2 * (size_t)K) * N, root) == cudaSuccess &&
         cudaStreamSynchronize(root) == cudaSuccess;
    if (!ok) status = reg_fail(REG_ERR_CUDA, "autotune streams / events");
    float *mT = buf, *mR = buf + N, *v = buf + 2 * N, *out = buf + 4 * N;
    // two passes over all candidates, each candidate's faster time kept: neighbouring choices
    // differ by a few percent, about the run-to-run spread of one short measurement
    std::vector<double> tbest(cands.size(), -1.0);
    for (int pass = 0; pass < 2 && status == REG_OK; ++pass) {
        for (size_t i = 0; status == REG_OK && i < cands.size(); ++i) {
            const int r = std::get<0>(cands[i]), c = std::get<1>(cands[i]), p = std::get<2>(cands[i]);
            const int d = std::get<3>(cands[i]), tc = std::get<4>(cands[i]);
            const double ms = time_matvec(grid, nt, r, c, p, d, tc, lanes, mT, mR, v, out, root, e0, e1);
            if (ms < 0.0) {
                status = reg_fail(REG_ERR_CUDA, std::string("autotune candidate failed: ") + reg_last_error());
                break;
            }
            if (tbest[i] < 0.0 || ms < tbest[i]) tbest[i] = ms;
        }
    }
    double best = -1.0;
    int bR = R0, bC = C0, bP = P0, bD = 1, bT = 0;
    for (size_t i = 0; status == REG_OK && i < cands.size(); ++i) {
        const int r = std::get<0>(cands[i]), c = std::get<1>(cands[i]), p = std::get<2>(cands[i]);
        const int d = std::get<3>(cands[i]), tc = std::get<4>(cands[i]);
        const double ms = tbest[i];
        if (best < 0.0 || ms < best) {
            best = ms;
            bR = r;
            bC = c;
            bP = p;
            bD = d;
            bT = tc;
        }
    }
    if (root) cudaStreamSynchronize(root);
    for (Lane& L : lanes) {
        if (L.st) cudaStreamSynchronize(L.st);
        if (L.done) cudaEventDestroy(L.done);
        if (L.st) cudaStreamDestroy(L.st);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (root) cudaStreamDestroy(root);
    cudaFree(buf);
    if (status != REG_OK) return status;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[std::make_tuple(dev, grid.n1, grid.n2)] = std::make_tuple(bR, bC, bP, bD, bT);
    }
    if (rows_per_cta) *rows_per_cta = bR;
    if (cols_per_cta) *cols_per_cta = bC;
    if (prefetch) *prefetch = bP;
    if (pdl) *pdl = bD;
    if (ms_per_matvec) *ms_per_matvec = best;
    return REG_OK;
}

extern "C" int reg_tile_config(reg_ctx* ctx, int* rows_per_cta, int* cols_per_cta, int* prefetch, int* pdl) {
    if (!ctx) return reg_fail(REG_ERR_ARG, "ctx is NULL");
    int R, C, P;
    default_tiles(ctx->n1, ctx->n2, &R, &C, &P);
    const bool set = ctx->tileR > 0;
    if (rows_per_cta) *rows_per_cta = set ? ctx->tileR : R;
    if (cols_per_cta) *cols_per_cta = set ? ctx->tileC : C;
    if (prefetch) *prefetch = set ? ctx->tileP : P;
    if (pdl) *pdl = ctx->pdl ? 1 : 0;
    return REG_OK;
}
