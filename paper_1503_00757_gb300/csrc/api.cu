// C ABI (include/reg.h) and host orchestration of the reduced-space
// Gauss-Newton-Krylov registration solver (Algorithms 1 and 2 of Mang & Biros,
// arXiv 1503.00757).  Every arithmetic step runs in the kernels of kernels.cu;
// the host only sequences launches and reads back FP64 scalars for the
// decisions of the PCG stop test, the Armijo test and the Newton stop test.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <string>

#include "fft.cuh"
#include "internal.h"

static thread_local std::string g_err = "no error";

int reg_fail(int status, const std::string& msg) {
    g_err = msg;
    return status;
}

extern "C" const char* reg_last_error(void) { return g_err.c_str(); }

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return reg_fail(REG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKL()                                                                                       \
    do {                                                                                            \
        cudaError_t e_ = cudaGetLastError();                                                        \
        if (e_ != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)

#define RET(x)                  \
    do {                        \
        int s_ = (x);           \
        if (s_ != REG_OK) return s_; \
    } while (0)

int col_blocks(reg_ctx* ctx);

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
static int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

extern "C" void reg_default_opts(reg_solve_opts* o) {
    if (!o) return;
    o->tol = 1e-2;
    o->maxit_newton = 50;
    o->maxit_pcg = 100;
    o->armijo_c1 = 1e-4;
    o->armijo_rho = 0.5;
    o->max_ls = 20;
    o->nt_policy = REG_NT_FIXED;
    o->cfl_max = 0.25;
    o->warm_start = 0;
}

// ---------------------------------------------------------------------------
// allocation
// ---------------------------------------------------------------------------
static void clear_graphs(reg_ctx* c) {
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

static void free_hist(reg_ctx* c) {
    clear_graphs(c);  // captured sequences hold history pointers
    cudaFree(c->m_hist);
    cudaFree(c->gm_hist);
    cudaFree(c->lam_hist);
    cudaFree(c->gmt_hist);
    c->m_hist = c->gm_hist = c->lam_hist = c->gmt_hist = nullptr;
}

// full-Newton histories (adjoint lam_j, grad m~_j) at the current capacity
static int alloc_newton_hist(reg_ctx* c) {
    if (c->lam_hist) return REG_OK;
    const size_t N = c->N;
    if (cudaMalloc(&c->lam_hist, sizeof(float) * N * (c->nt_cap + 1)) != cudaSuccess ||
        cudaMalloc(&c->gmt_hist, sizeof(float) * 2 * N * (c->nt_cap + 1)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->lam_hist);
        cudaFree(c->gmt_hist);
        c->lam_hist = c->gmt_hist = nullptr;
        return reg_fail(REG_ERR_NOMEM, "cudaMalloc of the full-Newton histories failed");
    }
    return REG_OK;
}

static int alloc_hist(reg_ctx* c, int nt) {
    if (nt <= c->nt_cap && c->m_hist) return REG_OK;
    free_hist(c);
    const size_t N = c->N;
    if (cudaMalloc(&c->m_hist, sizeof(float) * N * (nt + 1)) != cudaSuccess ||
        cudaMalloc(&c->gm_hist, sizeof(float) * 2 * N * (nt + 1)) != cudaSuccess) {
        cudaGetLastError();
        free_hist(c);
        c->nt_cap = 0;
        return reg_fail(REG_ERR_NOMEM, "cudaMalloc of the state history failed");
    }
    c->nt_cap = nt;
    c->have_lin = false;
    if (c->full_newton) return alloc_newton_hist(c);
    return REG_OK;
}

extern "C" void reg_destroy(reg_ctx* c) {
    if (!c) return;
    float** fl[] = {&c->mT, &c->mR, &c->v_lin, &c->E_lin, &c->eta_lin, &c->w0, &c->w1, &c->w2, &c->w3,
                    &c->bvec, &c->vtmp, &c->vtmp2, &c->gtmp, &c->T3, &c->T3b, &c->vx, &c->g, &c->r, &c->z, &c->s, &c->Hs,
                    &c->vt, &c->vtrial, &c->F, &c->Fs, &c->gF, &c->gv, &c->ybuf, &c->ytrial, &c->vtil};
    for (auto p : fl) cudaFree(*p);
    for (int i = 0; i < 6; ++i) cudaFree(c->S[i]);
    free_hist(c);
    clear_graphs(c);
    for (auto g : c->timing_graphs) cudaGraphExecDestroy(g);
    cudaFree(c->d_scal);
    cudaFree(c->d_part);
    cudaFree(c->tw);
    cudaFreeHost(c->h_scal);
    for (auto e : c->event_pool) cudaEventDestroy(e);
    delete c;
}

static int check_params(int nt, int regnorm, double beta, double gamma, double shear) {
    if (nt < 1 || nt > 100000) return reg_fail(REG_ERR_ARG, "nt must be in [1, 100000]");
    if (regnorm != REG_H1 && regnorm != REG_H2 && regnorm != REG_H3)
        return reg_fail(REG_ERR_ARG, "regnorm must be REG_H1, REG_H2 or REG_H3");
    if (!(beta > 0.0) || !std::isfinite(beta)) return reg_fail(REG_ERR_ARG, "beta must be finite and > 0");
    if (!(gamma >= 0.0)) return reg_fail(REG_ERR_ARG, "gamma must be >= 0 or +INFINITY");
    if (!(shear > -1.0 && shear < 1.0)) return reg_fail(REG_ERR_ARG, "shear must be in (-1, 1)");
    if (shear != 0.0 && regnorm != REG_H1) return reg_fail(REG_ERR_ARG, "shear control requires REG_H1");
    return REG_OK;
}

static void set_params(reg_ctx* c, int nt, int regnorm, double beta, double gamma, double shear) {
    c->nt = nt;
    c->regnorm = regnorm;
    c->beta_v = beta;
    c->beta_w = gamma;
    c->shear = shear;
    c->shear_model = shear != 0.0;
    c->nu = (1.0 + shear) / (1.0 - shear);
    c->pmode = (gamma == 0.0) ? PROJ_IDENTITY : (std::isinf(gamma) ? PROJ_LERAY : PROJ_MASS);
    c->ypath = regnorm != REG_H1 && !c->shear_model;
    c->have_lin = false;
}

extern "C" int reg_create(reg_grid grid, int nt, int regnorm, double beta, double gamma, double shear, reg_ctx** out) {
    if (!out) return reg_fail(REG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!is_pow2(grid.n1) || !is_pow2(grid.n2) || grid.n1 < 16 || grid.n2 < 16 || grid.n1 > 1024 || grid.n2 > 1024)
        return reg_fail(REG_ERR_ARG, "n1 and n2 must be powers of two in [16, 1024]");
    RET(check_params(nt, regnorm, beta, gamma, shear));

    reg_ctx* c = new reg_ctx();
    memset(c->S, 0, sizeof(c->S));
    c->full_newton = false;
    c->lam_hist = c->gmt_hist = nullptr;
    c->n1 = grid.n1;
    c->n2 = grid.n2;
    c->N = grid.n1 * grid.n2;
    c->log1 = ilog2(grid.n1);
    c->log2 = ilog2(grid.n2);
    c->nt_cap = 0;
    set_params(c, nt, regnorm, beta, gamma, shear);
    c->stream = 0;
    c->launches = 0;
    c->tileR = c->tileC = c->tileP = 0;
    c->pdl = true;
    c->tc_ok = tc_max_active_clusters(c->n1, c->n2) > 0;
    c->use_tc = false;  // the row / column kernel pairs unless the autotuner measured the cluster kernel faster
    {
        int dev = 0, R, C, P, D, T;
        if (cudaGetDevice(&dev) == cudaSuccess && tuned_tiles(dev, c->n1, c->n2, &R, &C, &P, &D, &T)) {
            c->tileR = R;
            c->tileC = C;
            c->tileP = P;
            c->pdl = D != 0;
            c->use_tc = T != 0 && c->tc_ok;
        }
    }
    c->use_graphs = true;
    c->timing = false;
    for (int k = 0; k < KC_COUNT; ++k) { c->tcount[k] = 0; c->tms[k] = 0.0; c->tbytes[k] = 0.0; }

    const size_t N = c->N;
    bool ok = true;
    auto A = [&](float** p, size_t n) { if (ok && cudaMalloc(p, sizeof(float) * n) != cudaSuccess) ok = false; };
    A(&c->mT, N); A(&c->mR, N); A(&c->v_lin, 2 * N); A(&c->E_lin, 3 * N); A(&c->eta_lin, N);
    A(&c->w0, N); A(&c->w1, N); A(&c->w2, N); A(&c->w3, N);
    A(&c->bvec, 2 * N); A(&c->vtmp, 2 * N); A(&c->vtmp2, 2 * N); A(&c->gtmp, 4 * N); A(&c->T3, 3 * N);
    A(&c->T3b, 3 * N); A(&c->vx, 2 * N);
    A(&c->g, 2 * N); A(&c->r, 2 * N); A(&c->z, 2 * N); A(&c->s, 2 * N); A(&c->Hs, 2 * N);
    A(&c->vt, 2 * N); A(&c->vtrial, 2 * N);
    A(&c->ybuf, 2 * N); A(&c->ytrial, 2 * N); A(&c->vtil, 2 * N);
    A(&c->F, 4 * N); A(&c->Fs, 4 * N); A(&c->gF, 8 * N); A(&c->gv, 4 * N);
    for (int i = 0; i < 6 && ok; ++i)
        if (cudaMalloc(&c->S[i], sizeof(float2) * N / 2) != cudaSuccess) ok = false;
    c->npart = 5 * 304 + 4096;
    if (ok && cudaMalloc(&c->d_scal, sizeof(double) * SL_COUNT) != cudaSuccess) ok = false;
    if (ok && cudaMalloc(&c->d_part, sizeof(double) * c->npart) != cudaSuccess) ok = false;
    if (ok && cudaMalloc(&c->tw, sizeof(float2) * REG_TW_TOTAL) != cudaSuccess) ok = false;
    if (ok && cudaMallocHost(&c->h_scal, sizeof(double) * SL_COUNT) != cudaSuccess) ok = false;
    if (!ok) {
        cudaGetLastError();
        reg_destroy(c);
        return reg_fail(REG_ERR_NOMEM, "device allocation failed");
    }
    if (k_init_twiddles(c) != cudaSuccess) {
        reg_destroy(c);
        return reg_fail(REG_ERR_CUDA, "twiddle upload failed");
    }
    int st = alloc_hist(c, nt);
    if (st != REG_OK) {
        reg_destroy(c);
        return st;
    }
    cudaMemset(c->mT, 0, sizeof(float) * N);
    cudaMemset(c->mR, 0, sizeof(float) * N);
    {
        const double one = 1.0;  // the unit denominator of device-scalar-scaled updates
        if (cudaMemcpy(c->d_scal + SL_ONE, &one, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            reg_destroy(c);
            return reg_fail(REG_ERR_CUDA, "scalar upload failed");
        }
    }
    *out = c;
    return REG_OK;
}

extern "C" int reg_set_params(reg_ctx* c, int nt, int regnorm, double beta, double gamma, double shear) {
    if (!c) return reg_fail(REG_ERR_ARG, "ctx is NULL");
    RET(check_params(nt, regnorm, beta, gamma, shear));
    const bool same = nt == c->nt && regnorm == c->regnorm && beta == c->beta_v && gamma == c->beta_w &&
                      shear == c->shear;
    if (!same) clear_graphs(c);  // captured sequences bake in nt and the Fourier-multiplier parameters
    set_params(c, nt, regnorm, beta, gamma, shear);
    return alloc_hist(c, nt);
}

extern "C" int reg_set_tiles(reg_ctx* c, int rows_per_cta, int cols_per_cta, int prefetch) {
    if (!c) return reg_fail(REG_ERR_ARG, "ctx is NULL");
    if (rows_per_cta == 0 && cols_per_cta == 0) {
        if (c->tileR != 0 || c->tileC != 0) clear_graphs(c);
        c->tileR = c->tileC = c->tileP = 0;
        return REG_OK;
    }
    if (!tiles_valid(c->n1, c->n2, rows_per_cta, cols_per_cta, prefetch))
        return reg_fail(REG_ERR_ARG, "tiles outside the launch limits of this grid");
    if (rows_per_cta != c->tileR || cols_per_cta != c->tileC || prefetch != c->tileP)
        clear_graphs(c);  // captures bake in launch shapes and kernels
    c->tileR = rows_per_cta;
    c->tileC = cols_per_cta;
    c->tileP = prefetch;
    return REG_OK;
}

extern "C" int reg_set_transport(reg_ctx* c, int cluster) {
    if (!c) return reg_fail(REG_ERR_ARG, "ctx is NULL");
    if (cluster && !c->tc_ok)
        return reg_fail(REG_ERR_ARG, "the cluster-resident transport kernel does not run on this grid or device");
    const bool on = cluster != 0;
    if (on != c->use_tc) clear_graphs(c);  // captures bake in the kernels
    c->use_tc = on;
    return REG_OK;
}

extern "C" int reg_set_hessian(reg_ctx* c, int full) {
    if (!c) return reg_fail(REG_ERR_ARG, "ctx is NULL");
    const bool on = full != 0;
    if (on == c->full_newton) return REG_OK;
    clear_graphs(c);  // captures bake in the matvec's launch sequence
    c->have_lin = false;  // the adjoint history belongs to the next reg_gradient
    c->full_newton = on;
    if (on) return alloc_newton_hist(c);
    cudaFree(c->lam_hist);
    cudaFree(c->gmt_hist);
    c->lam_hist = c->gmt_hist = nullptr;
    return REG_OK;
}

extern "C" int reg_transport_config(reg_ctx* c, int* cluster, int* ctas_per_cluster, int* max_active_clusters) {
    if (!c) return reg_fail(REG_ERR_ARG, "ctx is NULL");
    if (cluster) *cluster = (c->use_tc && !c->full_newton) ? 1 : 0;
    if (ctas_per_cluster) *ctas_per_cluster = c->tc_ok ? tc_cluster_size(c->n1) : 0;
    if (max_active_clusters) *max_active_clusters = c->tc_ok ? tc_max_active_clusters(c->n1, c->n2) : 0;
    return REG_OK;
}

extern "C" int reg_set_pdl(reg_ctx* c, int enable) {
    if (!c) return reg_fail(REG_ERR_ARG, "ctx is NULL");
    const bool on = enable != 0;
    if (on != c->pdl) clear_graphs(c);  // captures bake in the launch attribute
    c->pdl = on;
    return REG_OK;
}

extern "C" int reg_set_stream(reg_ctx* c, void* stream) {
    if (!c) return reg_fail(REG_ERR_ARG, "ctx is NULL");
    if ((cudaStream_t)stream != c->stream) clear_graphs(c);
    c->stream = (cudaStream_t)stream;
    return REG_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs: each fixed launch sequence (objective, gradient tail, matvec,
// one PCG iteration) is captured once per (kind, pointers, nt) and replayed.
// Sequences run directly on the legacy default stream (it cannot be
// captured) and while per-kernel timing is on.
// ---------------------------------------------------------------------------
enum GraphKind {
    GK_OBJECTIVE = 1, GK_GRADIENT = 2, GK_MATVEC = 3, GK_PCG_ITER = 4, GK_PCG_INIT = 5, GK_DETGRAD = 6,
    GK_GRADIENT_Y = 7, GK_PCG_ITER_Y = 8, GK_PCG_INIT_Y = 9
};

template <typename F>
static int run_seq(reg_ctx* c, int kind, const void* p0, const void* p1, int nt, F&& body) {
    if (c->timing && c->stream != 0) {
        // per-kernel timing: capture the sequence with its event records as graph nodes, so
        // the events bracket the kernels on the device without host launch gaps in between
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
        body();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (e != cudaSuccess || graph == nullptr)
            return reg_fail(REG_ERR_CUDA, std::string("stream capture failed: ") + cudaGetErrorString(e));
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        c->timing_graphs.push_back(exec);
        CK(cudaGraphLaunch(exec, c->stream));
        return REG_OK;
    }
    if (!c->use_graphs || c->timing || c->stream == 0) {
        body();
        CKL();
        return REG_OK;
    }
    for (auto& g : c->graphs) {
        if (g.kind == kind && g.p0 == p0 && g.p1 == p1 && g.nt == nt) {
            CK(cudaGraphLaunch(g.exec, c->stream));
            c->launches += g.nkern;
            return REG_OK;
        }
    }
    const long long l0 = c->launches;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
    body();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    const long long nk = c->launches - l0;
    c->launches = l0;
    if (e != cudaSuccess || graph == nullptr) {
        cudaGetLastError();
        return reg_fail(REG_ERR_CUDA, std::string("stream capture failed: ") + cudaGetErrorString(e));
    }
    GraphEntry g;
    g.kind = kind; g.p0 = p0; g.p1 = p1; g.nt = nt; g.nkern = nk;
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    if (c->graphs.size() >= 64) {  // callers that pass many distinct pointers: drop the oldest capture
        cudaGraphExecDestroy(c->graphs.front().exec);
        c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back(g);
    CK(cudaGraphLaunch(g.exec, c->stream));
    c->launches += nk;
    return REG_OK;
}

static int check_ptr(const void* p, const char* what) {
    if (!p) return reg_fail(REG_ERR_ARG, std::string(what) + " is NULL");
    if (((uintptr_t)p) & 15) return reg_fail(REG_ERR_ARG, std::string(what) + " is not 16-byte aligned");
    return REG_OK;
}

extern "C" int reg_set_images(reg_ctx* c, const float* mT, const float* mR) {
    if (!c) return reg_fail(REG_ERR_ARG, "ctx is NULL");
    RET(check_ptr(mT, "mT"));
    RET(check_ptr(mR, "mR"));
    CK(cudaMemcpyAsync(c->mT, mT, sizeof(float) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->mR, mR, sizeof(float) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    c->have_lin = false;
    return REG_OK;
}

// ---------------------------------------------------------------------------
// spectral building blocks
// ---------------------------------------------------------------------------
static SpecParams spec_params(reg_ctx* c, float coefA) {
    SpecParams P;
    P.scale = 1.0f / (float)c->N;
    P.coefA = coefA;
    P.beta_v = (float)c->beta_v;
    P.beta_w = (c->pmode == PROJ_MASS) ? (float)c->beta_w : 0.f;
    P.regnorm = c->shear_model ? REG_H1 : c->regnorm;
    P.pmode = c->pmode;
    const double h1 = 2.0 * M_PI / c->n1, h2 = 2.0 * M_PI / c->n2;
    P.escale = h1 * h2 / (double)c->N;
    P.ebv = 0.5 * c->beta_v;
    P.ebw = (c->pmode == PROJ_MASS) ? 0.5 * c->beta_w : 0.0;
    P.eta_bar = c->d_scal + SL_ETABAR;
    return P;
}

static double hh(reg_ctx* c) { return (2.0 * M_PI / c->n1) * (2.0 * M_PI / c->n2); }

// grad of a scalar field into out (2N)
static void sp_grad(reg_ctx* c, const float* f, float* out) {
    launch_r2c_scalar(c, f, c->S[0]);
    const float2* in[1] = {c->S[0]};
    float2* o[2] = {c->S[1], c->S[2]};
    launch_col(c, OP_GRAD, in, o, spec_params(c, 0.f), nullptr);
    launch_c2r_vec(c, c->S[1], c->S[2], out, out + c->N);
}

static void sp_div(reg_ctx* c, const float* u, float* out) {
    launch_r2c_vec(c, u, u + c->N, c->S[0], c->S[1]);
    const float2* in[2] = {c->S[0], c->S[1]};
    float2* o[1] = {c->S[2]};
    launch_col(c, OP_DIV, in, o, spec_params(c, 0.f), nullptr);
    launch_c2r_scalar(c, c->S[2], out);
}

static void sp_vec(reg_ctx* c, int op, float coefA, const float* u, float* out) {
    launch_r2c_vec(c, u, u + c->N, c->S[0], c->S[1]);
    const float2* in[2] = {c->S[0], c->S[1]};
    float2* o[2] = {c->S[2], c->S[3]};
    launch_col(c, op, in, o, spec_params(c, coefA), nullptr);
    launch_c2r_vec(c, c->S[2], c->S[3], out, out + c->N);
}

// out = coefA A u + K b  (reduced gradient / Hessian assembly, Eq. (e:control-eq-elim), (e:inc-control-eq-elim))
static void sp_assemble(reg_ctx* c, float coefA, const float* u, const float* b, float* out) {
    launch_r2c_vec(c, u, u + c->N, c->S[0], c->S[1]);
    launch_r2c_vec(c, b, b + c->N, c->S[2], c->S[3]);
    const float2* in[4] = {c->S[0], c->S[1], c->S[2], c->S[3]};
    float2* o[2] = {c->S[4], c->S[5]};
    launch_col(c, OP_ASSEMBLE, in, o, spec_params(c, coefA), nullptr);
    launch_c2r_vec(c, c->S[4], c->S[5], out, out + c->N);
}

// ---- preconditioned coordinates y = Q v, Q^ = (beta_v A'^)^(1/2), A'(0) = 1 ----
// out = Pi0 y + Q^-1 K b (the gradient, or with y = s and b = b~ the Hessian product, in y)
static void sp_assemble_y(reg_ctx* c, const float* y, const float* b, float* out) {
    launch_r2c_vec(c, y, y + c->N, c->S[0], c->S[1]);
    launch_r2c_vec(c, b, b + c->N, c->S[2], c->S[3]);
    const float2* in[4] = {c->S[0], c->S[1], c->S[2], c->S[3]};
    float2* o[2] = {c->S[4], c->S[5]};
    launch_col(c, OP_ASSEMBLE_Y, in, o, spec_params(c, 0.f), nullptr);
    launch_c2r_vec(c, c->S[4], c->S[5], out, out + c->N);
}

// device slot <- h1 h2 sum |Q x|^2 = ||Q x||^2 (the v-space norm of a y-space gradient / residual)
static void sp_qnorm(reg_ctx* c, const float* x, int slot) {
    launch_r2c_vec(c, x, x + c->N, c->S[0], c->S[1]);
    const float2* in[2] = {c->S[0], c->S[1]};
    launch_col(c, OP_QNORM, in, nullptr, spec_params(c, 0.f), c->d_part);
    launch_finalize(c, c->d_part, col_blocks(c), c->d_scal + slot, 1.0, 0, 0);
}

// grad of a vector field: gv planes (d1 u1, d2 u1, d1 u2, d2 u2)
static void sp_grad_vec(reg_ctx* c, const float* u, float* gv) {
    sp_grad(c, u, gv);
    sp_grad(c, u + c->N, gv + 2 * (size_t)c->N);
}

// out = div T (2 planes) of a symmetric tensor T = (T11, T12, T22)
static void sp_div_tensor(reg_ctx* c, const float* T, float* out) {
    const size_t N = c->N;
    launch_r2c_vec(c, T, T + N, c->S[0], c->S[1]);
    const float2* in0[2] = {c->S[0], c->S[1]};
    float2* o0[1] = {c->S[2]};
    launch_col(c, OP_DIV, in0, o0, spec_params(c, 0.f), nullptr);
    launch_r2c_vec(c, T + N, T + 2 * N, c->S[0], c->S[1]);
    float2* o1[1] = {c->S[3]};
    launch_col(c, OP_DIV, in0, o1, spec_params(c, 0.f), nullptr);
    launch_c2r_vec(c, c->S[2], c->S[3], out, out + N);
}

// Shear model with a mass source (App. A.2) or without a constraint: out = -beta_v div T + b
// + P(beta_v div T' - b), T' = T - 2 eta_bar Et (eta_bar in d_scal[SL_ETABAR]), P the
// multiplier OP_MASSP (mass source) or 0 (gamma = 0).  T = 2 eta E[v] and Et = E[v] for the
// reduced gradient; T = 2 eta (I + Q) E[v~] and Et = E[v~] for the Hessian (Et is overwritten).
static void shear_mass_assemble(reg_ctx* c, const float* T, float* Et, const float* b, float* out) {
    const long long N = c->N;
    const float bv = (float)c->beta_v;
    sp_div_tensor(c, T, c->gtmp);
    if (c->pmode == PROJ_MASS) {
        launch_axpby(c, 3 * N, -2.f, Et, 1.f, const_cast<float*>(T), SL_ETABAR, SL_ONE, Et);  // Et := T - 2 eta_bar Et
        sp_div_tensor(c, Et, c->gtmp + 2 * N);
        launch_axpby(c, 2 * N, bv, c->gtmp + 2 * N, -1.f, const_cast<float*>(b), -1, -1, c->vx);  // beta_v div T' - b
        sp_vec(c, OP_MASSP, 0.f, c->vx, c->vx);
    }
    launch_axpby(c, 2 * N, -bv, c->gtmp, 1.f, const_cast<float*>(b), -1, -1, out);
    if (c->pmode == PROJ_MASS) launch_axpby(c, 2 * N, 1.f, c->vx, 1.f, out, -1, -1, out);
}

// out = P_L(coefA div T + b), T = 3 planes (shear model)
static void sp_divt_proj(reg_ctx* c, float coefA, const float* T, const float* b, float* out) {
    const size_t N = c->N;
    launch_r2c_vec(c, T, T + N, c->S[0], c->S[1]);
    launch_r2c_vec(c, T + 2 * N, b, c->S[2], c->S[3]);
    launch_r2c_scalar(c, b + N, c->S[4]);
    const float2* in[5] = {c->S[0], c->S[1], c->S[2], c->S[3], c->S[4]};
    float2* o[2] = {c->S[5], c->S[0]};
    launch_col(c, OP_DIVT_PROJ, in, o, spec_params(c, coefA), nullptr);
    launch_c2r_vec(c, c->S[5], c->S[0], out, out + N);
}

// regularization energy into d_scal[SL_JREG]
static void reg_energy(reg_ctx* c, const float* v) {
    if (c->shear_model) {
        sp_grad_vec(c, v, c->gtmp);
        int np = launch_shear_strain(c, c->gtmp, (float)c->nu, nullptr, nullptr, nullptr, c->d_part);
        const double coef = c->beta_v * (2.0 * c->nu / (c->nu + 1.0)) * hh(c);
        launch_finalize(c, c->d_part, np, c->d_scal + SL_JREG, coef, 0, 0);
        if (c->pmode == PROJ_MASS) {
            // + (beta_w / 2) <(-Lap + I) w, w>, w = div v (OP_ENERGY with the beta_v part off)
            SpecParams P = spec_params(c, 0.f);
            P.ebv = 0.0;
            launch_r2c_vec(c, v, v + c->N, c->S[0], c->S[1]);
            const float2* in[2] = {c->S[0], c->S[1]};
            launch_col(c, OP_ENERGY, in, nullptr, P, c->d_part);
            launch_finalize(c, c->d_part, col_blocks(c), c->d_scal + SL_JREG, 1.0, 1, 0);
        }
        return;
    }
    launch_r2c_vec(c, v, v + c->N, c->S[0], c->S[1]);
    const float2* in[2] = {c->S[0], c->S[1]};
    launch_col(c, OP_ENERGY, in, nullptr, spec_params(c, 0.f), c->d_part);
    launch_finalize(c, c->d_part, col_blocks(c), c->d_scal + SL_JREG, 1.0, 0, 0);
}

static float* mh(reg_ctx* c, int j) { return c->m_hist + (size_t)j * c->N; }
static float* gmh(reg_ctx* c, int j) { return c->gm_hist + (size_t)j * 2 * c->N; }

// State equation (Eq. (e:state-eq-elim)), Heun in time: fills m_hist[0..nt], gm_hist[0..nt].
// The column pass transforms only d1 (OP_GRAD1); d2 is diagonal in the row
// spectra and is formed by the row kernel from the stage's own spectrum S[0].
// init (nullable): the field transported instead of the template m_T.
static void state_solve(reg_ctx* c, const float* v, int nt, const float* init = nullptr) {
    const float h = 1.0f / (float)nt;
    const float* m0 = init ? init : c->mT;
    if (c->use_tc && !c->full_newton) {
        TcArgs a = {};
        a.nt = nt; a.h = h; a.v = v; a.mT = m0; a.m_hist = c->m_hist; a.gm_hist = c->gm_hist; a.us = c->w0;
        launch_transport_cluster(c, TC_STATE, a);
        return;
    }
    cudaMemcpyAsync(mh(c, 0), m0, sizeof(float) * c->N, cudaMemcpyDeviceToDevice, c->stream);
    launch_r2c_scalar(c, mh(c, 0), c->S[0]);
    const float2* in[1] = {c->S[0]};
    float2* G[1] = {c->S[1]};
    const SpecParams P = spec_params(c, 0.f);
    for (int j = 0; j < nt; ++j) {
        launch_col(c, OP_GRAD1, in, G, P, nullptr);
        AdvArgs a = {};
        a.G1 = c->S[1]; a.G2 = nullptr; a.Sd2 = c->S[0];
        a.uj = mh(c, j); a.us = nullptr; a.v = v;
        a.gm = nullptr; a.vt = nullptr;
        a.u_out = c->w0; a.grad_out = gmh(c, j); a.S_out = c->S[0];
        a.h = h; a.stage = 1;
        launch_row_adv(c, a);
        launch_col(c, OP_GRAD1, in, G, P, nullptr);
        a.us = c->w0; a.u_out = mh(c, j + 1); a.grad_out = nullptr; a.stage = 2;
        launch_row_adv(c, a);
    }
    float2* G2[2] = {c->S[1], c->S[2]};
    launch_col(c, OP_GRAD, in, G2, P, nullptr);
    launch_c2r_vec(c, c->S[1], c->S[2], gmh(c, nt), gmh(c, nt) + c->N);
}

// Adjoint (Eq. (e:adj-eq-elim)) or Gauss-Newton incremental adjoint
// (Eq. (e:inc-adj-eq-elim)) backward in time from lam_nt = ca*a + cb*cf, with
// the body force b = int lam grad m dt (trapezoid) accumulated into bout.
// lhist (nullable): store lam_j at lhist + j N for j = 0..nt (the full Newton matvec reads it).
static void adjoint_solve(reg_ctx* c, const float* v, int nt, const float* a, float ca, const float* cf, float cb,
                          float* bout, double* part_jdata, float* lhist = nullptr) {
    const float h = 1.0f / (float)nt;
    if (c->use_tc && !part_jdata && !lhist) {
        TcArgs t = {};
        t.nt = nt; t.h = h; t.v = v; t.gm_hist = c->gm_hist; t.lj = c->w1; t.ls = c->w2;
        t.adj_a = a; t.adj_ca = ca; t.adj_c = cf; t.adj_cb = cb; t.b = bout;
        launch_transport_cluster(c, TC_ADJOINT, t);
        return;
    }
    float* lst = c->w2;
    auto lam_at = [&](int j) { return lhist ? lhist + (size_t)j * c->N : c->w1; };
    launch_adj_init(c, a, ca, cf, cb, v, lam_at(nt), bout, gmh(c, nt), 0.5f * h, c->S[1], c->S[2], part_jdata);
    const float2* Fin[2] = {c->S[1], c->S[2]};
    float2* D[1] = {c->S[0]};
    const SpecParams P = spec_params(c, 0.f);
    for (int j = nt; j >= 1; --j) {
        launch_col(c, OP_DIV1, Fin, D, P, nullptr);
        AdjArgs s1 = {};
        s1.D = c->S[0]; s1.lj = lam_at(j); s1.ls = nullptr; s1.v = v; s1.l_out = lst;
        s1.b = nullptr; s1.gm = nullptr; s1.w = 0.f; s1.F1 = c->S[1]; s1.F2 = c->S[2]; s1.h = h; s1.stage = 1;
        launch_row_adj(c, s1);
        launch_col(c, OP_DIV1, Fin, D, P, nullptr);
        AdjArgs s2 = s1;
        s2.ls = lst; s2.l_out = lam_at(j - 1); s2.stage = 2;
        s2.b = bout; s2.gm = gmh(c, j - 1); s2.w = (j - 1 == 0) ? 0.5f * h : h;
        if (j == 1) { s2.F1 = nullptr; s2.F2 = nullptr; }
        launch_row_adj(c, s2);
    }
}

static float* lamh(reg_ctx* c, int j) { return c->lam_hist + (size_t)j * c->N; }
static float* gmth(reg_ctx* c, int j) { return c->gmt_hist + (size_t)j * 2 * c->N; }

// Full-Newton incremental adjoint (Eq. (e:inc-adj-eq-elim) with the lambda term), backward from
// lam~_nt = -m~_nt (c->w3): the flux of every divergence is lam~ v + lam v~ with lam from the
// gradient's adjoint history at the time the divergence is evaluated, and the incremental body
// force is b~ = sum_j w_j (lam~_j grad m_j + lam_j grad m~_j) (trapezoid).
static void inc_adjoint_full(reg_ctx* c, const float* v, const float* vt, int nt, float* bout) {
    const float h = 1.0f / (float)nt;
    float* lam = c->w1;
    float* lst = c->w2;
    launch_adj_init(c, nullptr, 0.f, c->w3, -1.f, v, lam, bout, gmh(c, nt), 0.5f * h, c->S[1], c->S[2], nullptr,
                    lamh(c, nt), vt, gmth(c, nt));
    const float2* Fin[2] = {c->S[1], c->S[2]};
    float2* D[1] = {c->S[0]};
    const SpecParams P = spec_params(c, 0.f);
    for (int j = nt; j >= 1; --j) {
        launch_col(c, OP_DIV1, Fin, D, P, nullptr);
        AdjArgs s1 = {};
        s1.D = c->S[0]; s1.lj = lam; s1.ls = nullptr; s1.v = v; s1.l_out = lst;
        s1.b = nullptr; s1.gm = nullptr; s1.w = 0.f; s1.F1 = c->S[1]; s1.F2 = c->S[2]; s1.h = h; s1.stage = 1;
        s1.lsrc = lamh(c, j - 1); s1.vt = vt; s1.gmt = nullptr;
        launch_row_adj(c, s1);
        launch_col(c, OP_DIV1, Fin, D, P, nullptr);
        AdjArgs s2 = s1;
        s2.ls = lst; s2.l_out = lam; s2.stage = 2;
        s2.b = bout; s2.gm = gmh(c, j - 1); s2.w = (j - 1 == 0) ? 0.5f * h : h;
        s2.gmt = gmth(c, j - 1);
        if (j == 1) { s2.F1 = nullptr; s2.F2 = nullptr; }
        launch_row_adj(c, s2);
    }
}

// Incremental state (Eq. (e:inc-state-eq-elim)); leaves m~(1) in c->w3.
// m~(0) = 0 is passed as u_j = nullptr to both stages of the first step.  gmt (nullable):
// store grad m~_j at gmt + j 2N for j = 0..nt (the full Newton matvec reads it).
// gm_fixed (nullable): a source gradient used at every time instead of the grad m history.
static void inc_state_solve(reg_ctx* c, const float* v, const float* vt, int nt, float* gmt = nullptr,
                            const float* gm_fixed = nullptr) {
    const float h = 1.0f / (float)nt;
    float* mj = c->w3;
    float* ms = c->w0;
    const float2* in[1] = {c->S[0]};
    float2* G[1] = {c->S[1]};
    const SpecParams P = spec_params(c, 0.f);
    for (int j = 0; j < nt; ++j) {
        AdvArgs a = {};
        if (j > 0) {
            launch_col(c, OP_GRAD1, in, G, P, nullptr);
            a.G1 = c->S[1]; a.Sd2 = c->S[0];
        }
        a.uj = (j > 0) ? mj : nullptr; a.us = nullptr; a.v = v; a.gm = gm_fixed ? gm_fixed : gmh(c, j); a.vt = vt;
        a.u_out = ms; a.grad_out = gmt ? gmt + (size_t)j * 2 * c->N : nullptr; a.S_out = c->S[0]; a.h = h;
        a.stage = 1;
        // the first launch of the solve: v~ may come from the launch just before (Q^-1 s in
        // preconditioned coordinates, or a caller's kernel), so it is read after the wait
        a.late = (j == 0) ? 1 : 0;
        launch_row_adv(c, a);
        a.late = 0;
        launch_col(c, OP_GRAD1, in, G, P, nullptr);
        a.G1 = c->S[1]; a.Sd2 = c->S[0];
        a.us = ms; a.gm = gm_fixed ? gm_fixed : gmh(c, j + 1); a.u_out = mj; a.stage = 2; a.grad_out = nullptr;
        a.S_out = (j + 1 < nt) ? c->S[0] : nullptr;
        launch_row_adv(c, a);
    }
    if (gmt) sp_grad(c, mj, gmt + (size_t)nt * 2 * c->N);
}

// ---------------------------------------------------------------------------
// objective / gradient / matvec
// ---------------------------------------------------------------------------
static int read_scalars(reg_ctx* c) {
    CK(cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(double) * SL_COUNT, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return REG_OK;
}

static int ensure_nt(reg_ctx* c, int nt) { return alloc_hist(c, nt); }

// forward solve + J (device slots SL_JDATA, SL_JREG)
// Regularization energy from y = Q v (reg_solve in preconditioned coordinates)
static void reg_energy_y(reg_ctx* c, const float* y) {
    launch_r2c_vec(c, y, y + c->N, c->S[0], c->S[1]);
    const float2* in[2] = {c->S[0], c->S[1]};
    launch_col(c, OP_ENERGY_Y, in, nullptr, spec_params(c, 0.f), c->d_part);
    launch_finalize(c, c->d_part, col_blocks(c), c->d_scal + SL_JREG, 1.0, 0, 0);
}

// y != nullptr: v = Q^-1 y and the regularization energy is taken from y
static void objective_launches(reg_ctx* c, const float* v, int nt, const float* y = nullptr) {
    state_solve(c, v, nt);
    // J_data = 0.5 ||m_R - m_1||^2
    launch_axpby(c, c->N, 1.f, c->mR, -1.f, mh(c, nt), -1, -1, c->w1);
    int np = launch_dot_partial(c, c->w1, c->w1, c->N, c->d_part);
    launch_finalize(c, c->d_part, np, c->d_scal + SL_JDATA, 0.5 * hh(c), 0, 0);
    if (y)
        reg_energy_y(c, y);
    else
        reg_energy(c, v);
}

static int objective_dev(reg_ctx* c, const float* v, int nt, const float* y = nullptr) {
    RET(ensure_nt(c, nt));
    return run_seq(c, GK_OBJECTIVE, v, y, nt, [&] { objective_launches(c, v, nt, y); });
}

static void gradient_launches(reg_ctx* c, const float* v, float* g, int nt) {
    adjoint_solve(c, v, nt, c->mR, 1.f, mh(c, nt), -1.f, c->bvec, nullptr, c->full_newton ? c->lam_hist : nullptr);
    if (c->shear_model) {
        sp_grad_vec(c, v, c->gtmp);
        launch_shear_strain(c, c->gtmp, (float)c->nu, c->E_lin, c->eta_lin, c->T3, nullptr);
        // mean viscosity of the linearization point (App. A.2: eta = eta^ + eta_bar)
        const int np = launch_sum_partial(c, c->eta_lin, c->N, c->d_part);
        launch_finalize(c, c->d_part, np, c->d_scal + SL_ETABAR, 1.0 / (double)c->N, 0, 0);
        if (c->pmode == PROJ_LERAY) {
            sp_divt_proj(c, -(float)c->beta_v, c->T3, c->bvec, g);
        } else {
            cudaMemcpyAsync(c->T3b, c->E_lin, sizeof(float) * 3 * c->N, cudaMemcpyDeviceToDevice, c->stream);
            shear_mass_assemble(c, c->T3, c->T3b, c->bvec, g);
        }
    } else {
        sp_assemble(c, (float)c->beta_v, v, c->bvec, g);
    }
    if (v != c->v_lin)
        cudaMemcpyAsync(c->v_lin, v, sizeof(float) * 2 * c->N, cudaMemcpyDeviceToDevice, c->stream);
}

static int gradient_dev(reg_ctx* c, const float* v, float* g, int nt) {
    RET(objective_dev(c, v, nt));
    RET(run_seq(c, GK_GRADIENT, v, g, nt, [&] { gradient_launches(c, v, g, nt); }));
    c->nt_lin = nt;
    c->have_lin = true;
    return REG_OK;
}

// Gradient in preconditioned coordinates: g_y = Q^-1 g_v = Pi0 y + Q^-1 K b, at v = Q^-1 y
static int gradient_dev_y(reg_ctx* c, const float* v, const float* y, float* gy, int nt) {
    RET(objective_dev(c, v, nt, y));
    RET(run_seq(c, GK_GRADIENT_Y, v, y, nt, [&] {  // gy is always c->g
        adjoint_solve(c, v, nt, c->mR, 1.f, mh(c, nt), -1.f, c->bvec, nullptr, c->full_newton ? c->lam_hist : nullptr);
        sp_assemble_y(c, y, c->bvec, gy);
        if (v != c->v_lin)
            cudaMemcpyAsync(c->v_lin, v, sizeof(float) * 2 * c->N, cudaMemcpyDeviceToDevice, c->stream);
    }));
    c->nt_lin = nt;
    c->have_lin = true;
    return REG_OK;
}

// Incremental state and Gauss-Newton incremental adjoint of a matvec (Algorithm 2's product):
// m~(1) in c->w3, b~ in c->bvec.  The cluster path runs both sweeps in one launch.
static void inc_solves(reg_ctx* c, const float* vt, int nt) {
    if (c->full_newton) {
        inc_state_solve(c, c->v_lin, vt, nt, c->gmt_hist);
        inc_adjoint_full(c, c->v_lin, vt, nt, c->bvec);
        return;
    }
    if (c->use_tc) {
        TcArgs a = {};
        a.nt = nt; a.h = 1.0f / (float)nt; a.v = c->v_lin; a.vt = vt; a.gm_hist = c->gm_hist;
        a.uj = c->w3; a.us = c->w0; a.lj = c->w1; a.ls = c->w2;
        a.adj_a = nullptr; a.adj_ca = 0.f; a.adj_c = nullptr; a.adj_cb = -1.f; a.b = c->bvec;
        launch_transport_cluster(c, TC_MATVEC, a);
        return;
    }
    inc_state_solve(c, c->v_lin, vt, nt);
    adjoint_solve(c, c->v_lin, nt, nullptr, 0.f, c->w3, -1.f, c->bvec, nullptr);
}

// Hessian product in preconditioned coordinates: H_y s = Q^-1 H_v Q^-1 s = Pi0 s + Q^-1 K b~(v~ = Q^-1 s)
static void matvec_launches_y(reg_ctx* c, const float* s, float* Hs) {
    const int nt = c->nt_lin;
    sp_vec(c, OP_QINV, 0.f, s, c->vtil);
    inc_solves(c, c->vtil, nt);
    sp_assemble_y(c, s, c->bvec, Hs);
}

static void matvec_launches(reg_ctx* c, const float* vt, float* Hvt) {
    const int nt = c->nt_lin;
    inc_solves(c, vt, nt);
    if (c->shear_model) {
        sp_grad_vec(c, vt, c->gtmp);
        launch_shear_second(c, c->gtmp, c->E_lin, c->eta_lin, (float)c->nu, c->T3);
        if (c->pmode == PROJ_LERAY) {
            sp_divt_proj(c, -(float)c->beta_v, c->T3, c->bvec, Hvt);
        } else {
            launch_shear_strain(c, c->gtmp, (float)c->nu, c->T3b, nullptr, nullptr, nullptr);  // E[v~]
            shear_mass_assemble(c, c->T3, c->T3b, c->bvec, Hvt);
        }
    } else {
        sp_assemble(c, (float)c->beta_v, vt, c->bvec, Hvt);
    }
}

static int matvec_dev(reg_ctx* c, const float* vt, float* Hvt) {
    if (!c->have_lin) return reg_fail(REG_ERR_STATE, "reg_hessian_matvec called before reg_gradient");
    return run_seq(c, GK_MATVEC, vt, Hvt, c->nt_lin, [&] { matvec_launches(c, vt, Hvt); });
}

static void precond_dev(reg_ctx* c, const float* r, float* z) {
    sp_vec(c, OP_PRECOND, 0.f, r, z);
}

// ---------------------------------------------------------------------------
// C ABI: unit operators
// ---------------------------------------------------------------------------
#define CTX_CHECK(c) if (!(c)) return reg_fail(REG_ERR_ARG, "ctx is NULL")

extern "C" int reg_spectral_grad(reg_ctx* c, const float* f, float* out) {
    CTX_CHECK(c);
    RET(check_ptr(f, "f")); RET(check_ptr(out, "grad_f"));
    sp_grad(c, f, out);
    CKL();
    return REG_OK;
}

extern "C" int reg_spectral_div(reg_ctx* c, const float* u, float* out) {
    CTX_CHECK(c);
    RET(check_ptr(u, "u")); RET(check_ptr(out, "div_u"));
    sp_div(c, u, out);
    CKL();
    return REG_OK;
}

extern "C" int reg_apply_reg(reg_ctx* c, const float* v, float* out) {
    CTX_CHECK(c);
    RET(check_ptr(v, "v")); RET(check_ptr(out, "out"));
    if (c->shear_model) {
        sp_grad_vec(c, v, c->gtmp);
        launch_shear_strain(c, c->gtmp, (float)c->nu, nullptr, nullptr, c->T3, nullptr);
        // beta_v A[v] = -beta_v div(2 eta E), without projection: use the divergence of each row of T
        const size_t N = c->N;
        launch_r2c_vec(c, c->T3, c->T3 + N, c->S[0], c->S[1]);
        const float2* in0[2] = {c->S[0], c->S[1]};
        float2* o0[1] = {c->S[2]};
        launch_col(c, OP_DIV, in0, o0, spec_params(c, 0.f), nullptr);
        launch_r2c_vec(c, c->T3 + N, c->T3 + 2 * N, c->S[0], c->S[1]);
        float2* o1[1] = {c->S[3]};
        launch_col(c, OP_DIV, in0, o1, spec_params(c, 0.f), nullptr);
        launch_c2r_vec(c, c->S[2], c->S[3], out, out + N);
        launch_axpby(c, 2 * (long long)N, -(float)c->beta_v, out, 0.f, out, -1, -1, out);
    } else {
        sp_vec(c, OP_REG, (float)c->beta_v, v, out);
    }
    CKL();
    return REG_OK;
}

extern "C" int reg_apply_proj(reg_ctx* c, const float* b, float* out) {
    CTX_CHECK(c);
    RET(check_ptr(b, "b")); RET(check_ptr(out, "out"));
    sp_vec(c, OP_PROJ, 0.f, b, out);
    CKL();
    return REG_OK;
}

extern "C" int reg_apply_precond_sqrt(reg_ctx* c, const float* x, float* out, int inverse) {
    CTX_CHECK(c);
    RET(check_ptr(x, "x")); RET(check_ptr(out, "out"));
    sp_vec(c, inverse ? OP_QINV : OP_QMUL, 0.f, x, out);
    CKL();
    return REG_OK;
}

int apply_smooth_proj(reg_ctx* c, float a, const float* b, float* out) {
    CTX_CHECK(c);
    RET(check_ptr(b, "b")); RET(check_ptr(out, "out"));
    sp_vec(c, OP_SMOOTH_PROJ, a, b, out);
    CKL();
    return REG_OK;
}

extern "C" int reg_apply_precond(reg_ctx* c, const float* r, float* out) {
    CTX_CHECK(c);
    RET(check_ptr(r, "r")); RET(check_ptr(out, "out"));
    precond_dev(c, r, out);
    CKL();
    return REG_OK;
}

extern "C" int reg_objective(reg_ctx* c, const float* v, float* m1, double* J) {
    CTX_CHECK(c);
    RET(check_ptr(v, "v"));
    if (m1) RET(check_ptr(m1, "m1"));
    RET(objective_dev(c, v, c->nt));
    c->have_lin = false;  // history now belongs to this v, but grad/adjoint data do not
    if (m1) CK(cudaMemcpyAsync(m1, mh(c, c->nt), sizeof(float) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    if (J) {
        RET(read_scalars(c));
        *J = c->h_scal[SL_JDATA] + c->h_scal[SL_JREG];
        if (!std::isfinite(*J)) return reg_fail(REG_ERR_NAN, "objective is not finite");
    }
    return REG_OK;
}

extern "C" int reg_gradient(reg_ctx* c, const float* v, float* g, double* J) {
    CTX_CHECK(c);
    RET(check_ptr(v, "v")); RET(check_ptr(g, "g"));
    RET(gradient_dev(c, v, g, c->nt));
    if (J) {
        RET(read_scalars(c));
        *J = c->h_scal[SL_JDATA] + c->h_scal[SL_JREG];
        if (!std::isfinite(*J)) return reg_fail(REG_ERR_NAN, "objective is not finite");
    }
    return REG_OK;
}

extern "C" int reg_body_force(reg_ctx* c, float* b_out) {
    CTX_CHECK(c);
    RET(check_ptr(b_out, "b_out"));
    if (!c->have_lin) return reg_fail(REG_ERR_STATE, "no body force: call reg_gradient first");
    CK(cudaMemcpyAsync(b_out, c->bvec, sizeof(float) * 2 * c->N, cudaMemcpyDeviceToDevice, c->stream));
    return REG_OK;
}

extern "C" int reg_hessian_matvec(reg_ctx* c, const float* vt, float* Hvt) {
    CTX_CHECK(c);
    RET(check_ptr(vt, "vt")); RET(check_ptr(Hvt, "Hvt"));
    return matvec_dev(c, vt, Hvt);
}

// ---------------------------------------------------------------------------
// Newton-Krylov solve (Algorithm 1) with PCG (Algorithm 2)
// ---------------------------------------------------------------------------
static int dot_dev(reg_ctx* c, const float* x, const float* y, int slot) {
    int np = launch_dot_partial(c, x, y, 2 * (long long)c->N, c->d_part);
    launch_finalize(c, c->d_part, np, c->d_scal + slot, hh(c), 0, 0);
    return REG_OK;
}

static int nt_for(reg_ctx* c, const float* v, const reg_solve_opts& o, double* cfl_out) {
    int np = launch_maxnorm_partial(c, v, c->N, c->d_part);
    launch_finalize(c, c->d_part, np, c->d_scal + SL_VMAX, 1.0, 0, 1);
    if (read_scalars(c) != REG_OK) return -1;
    const double vmax = c->h_scal[SL_VMAX];
    const int n = c->n1 > c->n2 ? c->n1 : c->n2;
    int nt = c->nt;
    if (o.nt_policy == REG_NT_CFL) {
        const int need = (int)std::ceil(vmax * n / (2.0 * M_PI * o.cfl_max));
        if (need > nt) nt = need;
    }
    if (cfl_out) *cfl_out = vmax * n / (2.0 * M_PI * nt);
    return nt;
}

// PCG (Algorithm 2) on H vt = -g; returns #matvecs.  One PCG iteration is a
// single launch sequence (matvec, <s, Hs>, updates of vt and r with
// kappa = <r, z> / <s, Hs> computed on the device, ||r||^2, z = P r,
// <z, r>, s = z + mu s); the host reads <s, Hs> and ||r|| once per iteration
// for the curvature check and the stop test (Algorithm 2's break).  The
// update kernel does nothing when <s, Hs> <= 0, so vt and r keep their values
// from before that iteration.
//
// In preconditioned coordinates (c->ypath) the same iteration is CG on
// H_y = Q^-1 H Q^-1 without a preconditioner (z = r): its iterates are Q times
// those of PCG with P = Q^2 = beta_v A', and the stop test uses the v-space
// residual norm ||Q r_y|| = ||r_v||.
static int pcg_dev(reg_ctx* c, double gnorm, double eta, int maxit, int* hit_max, int* status) {
    const long long n2N = 2 * (long long)c->N;
    const double scale = hh(c);
    const bool yp = c->ypath;
    *status = REG_OK;
    RET(run_seq(c, yp ? GK_PCG_INIT_Y : GK_PCG_INIT, nullptr, nullptr, c->nt_lin, [&] {
        launch_fill(c, n2N, c->vt, 0.f);
        launch_axpby(c, n2N, -1.f, c->g, 0.f, c->r, -1, -1, c->r);  // r = -g
        if (yp) {
            cudaMemcpyAsync(c->s, c->r, sizeof(float) * n2N, cudaMemcpyDeviceToDevice, c->stream);
            dot_dev(c, c->r, c->r, SL_RZ);
        } else {
            precond_dev(c, c->r, c->z);
            cudaMemcpyAsync(c->s, c->z, sizeof(float) * n2N, cudaMemcpyDeviceToDevice, c->stream);
            dot_dev(c, c->r, c->z, SL_RZ);
        }
    }));
    int it = 0;
    *hit_max = 1;
    if (!c->have_lin) return reg_fail(REG_ERR_STATE, "PCG without a linearization point");
    for (int l = 0; l < maxit; ++l) {
        int st = run_seq(c, yp ? GK_PCG_ITER_Y : GK_PCG_ITER, nullptr, nullptr, c->nt_lin, [&] {
            if (yp)
                matvec_launches_y(c, c->s, c->Hs);
            else
                matvec_launches(c, c->s, c->Hs);
            dot_dev(c, c->s, c->Hs, SL_SHS);
            int np = launch_pcg_update(c, n2N, c->vt, c->s, c->r, c->Hs, c->d_part);
            if (yp) {
                sp_qnorm(c, c->r, SL_RNORM2);
                dot_dev(c, c->r, c->r, SL_RZNEW);
                launch_pcg_dir(c, n2N, c->r, c->s);
            } else {
                launch_finalize(c, c->d_part, np, c->d_scal + SL_RNORM2, scale, 0, 0);
                precond_dev(c, c->r, c->z);
                dot_dev(c, c->z, c->r, SL_RZNEW);
                launch_pcg_dir(c, n2N, c->z, c->s);
            }
            cudaMemcpyAsync(c->d_scal + SL_RZ, c->d_scal + SL_RZNEW, sizeof(double), cudaMemcpyDeviceToDevice,
                            c->stream);
        });
        if (st != REG_OK) { *status = st; return it; }
        ++it;
        if (read_scalars(c) != REG_OK) { *status = REG_ERR_CUDA; return it; }
        const double sHs = c->h_scal[SL_SHS];
        if (!std::isfinite(sHs)) { *status = REG_ERR_NAN; return it; }
        if (sHs <= 0.0) {
            // non-positive curvature: the update kernel left vt and r unchanged; in the first
            // iteration the step is the first direction s_0 = P r_0 (the oracle's choice)
            *hit_max = 0;
            if (it == 1) {
                if (yp)
                    cudaMemcpyAsync(c->vt, c->r, sizeof(float) * n2N, cudaMemcpyDeviceToDevice, c->stream);
                else
                    precond_dev(c, c->r, c->vt);
            }
            break;
        }
        const double rn = std::sqrt(c->h_scal[SL_RNORM2]);
        if (!std::isfinite(rn)) { *status = REG_ERR_NAN; return it; }
        if (rn < eta * gnorm) { *hit_max = 0; break; }
    }
    CKL();
    return it;
}

extern "C" int reg_solve(reg_ctx* c, float* v, const reg_solve_opts* opts, reg_solve_stats* stats) {
    CTX_CHECK(c);
    RET(check_ptr(v, "v_inout"));
    reg_solve_opts o;
    reg_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.tol > 0) || o.maxit_newton < 0 || o.maxit_pcg < 1 || o.max_ls < 1 || !(o.armijo_rho > 0 && o.armijo_rho < 1) ||
        !(o.cfl_max > 0))
        return reg_fail(REG_ERR_ARG, "invalid solve options");
    reg_solve_stats st;
    memset(&st, 0, sizeof(st));
    const long long n2N = 2 * (long long)c->N;
    const size_t vb = sizeof(float) * n2N;
    int n_pde = 0;
    double gref = 0.0;
    if (!o.warm_start) launch_fill(c, n2N, v, 0.f);
    // Quadratic H2 regularization iterates on y = Q v (Q^2 = beta_v A' is the
    // preconditioner): the FP32 rounding of v, amplified by beta_v |k|^4 in the
    // reduced gradient, would otherwise put a floor of about u beta_v max|k|^4 ||v||
    // under ||g|| (above 1e-2 ||g(0)|| from 128^2 on); in y the regularization
    // term is the identity and every other operator applied is smoothing.
    const bool yp = c->ypath;
    float* y = c->ybuf;
    if (yp) {
        if (o.warm_start) {
            sp_vec(c, OP_QMUL, 0.f, v, y);
            sp_vec(c, OP_QINV, 0.f, y, v);
        } else {
            launch_fill(c, n2N, y, 0.f);
        }
    }
    double cfl = 0.0;
    int nt = nt_for(c, v, o, &cfl);
    if (nt < 0) return reg_fail(REG_ERR_CUDA, "scalar readback failed");
    auto grad_at = [&](const float* vv, const float* yy) {
        return yp ? gradient_dev_y(c, vv, yy, c->g, nt) : gradient_dev(c, vv, c->g, nt);
    };
    auto gnorm2_to_slot = [&]() {
        if (yp)
            sp_qnorm(c, c->g, SL_GNORM2);  // ||g_v|| = ||Q g_y||
        else
            dot_dev(c, c->g, c->g, SL_GNORM2);
    };
    if (o.warm_start) {
        launch_fill(c, n2N, c->vtrial, 0.f);
        RET(gradient_dev(c, c->vtrial, c->g, c->nt));
        n_pde += 2;
        dot_dev(c, c->g, c->g, SL_GNORM2);
        RET(read_scalars(c));
        gref = std::sqrt(c->h_scal[SL_GNORM2]);
    }
    RET(grad_at(v, y));
    n_pde += 2;
    gnorm2_to_slot();
    RET(read_scalars(c));
    double J = c->h_scal[SL_JDATA] + c->h_scal[SL_JREG];
    double gnorm = std::sqrt(c->h_scal[SL_GNORM2]);
    if (!o.warm_start) gref = gnorm;
    // Algorithm 2's forcing term is relative to the gradient at the initial iterate
    // (the warm start, if any); the stopping test stays relative to g_ref = g(0).
    const double gstart = gnorm;
    st.J0 = J;
    int status = REG_OK;
    int k = 0;
    if (!std::isfinite(J) || !std::isfinite(gnorm)) status = REG_ERR_NAN;
    while (status == REG_OK) {
        if (gref == 0.0 || gnorm / gref <= o.tol) break;
        if (k >= o.maxit_newton) { status = REG_ERR_MAXIT; break; }
        const double eta = std::fmin(0.5, std::sqrt(gnorm / gstart));
        int hit = 0, pst = REG_OK;
        const int it = pcg_dev(c, gnorm, eta, o.maxit_pcg, &hit, &pst);
        st.n_mv += it;
        n_pde += 2 * it;
        st.n_pcg_maxit += hit;
        if (pst != REG_OK) { status = pst; break; }
        dot_dev(c, c->g, c->vt, SL_GV);
        RET(read_scalars(c));
        double gv = c->h_scal[SL_GV];
        if (!(gv < 0.0)) {
            // preconditioned steepest descent: -P^-1 g_v, i.e. -g_y in y
            if (yp)
                cudaMemcpyAsync(c->vt, c->g, vb, cudaMemcpyDeviceToDevice, c->stream);
            else
                precond_dev(c, c->g, c->vt);
            launch_axpby(c, n2N, 0.f, c->vt, -1.f, c->vt, -1, -1, c->vt);
            dot_dev(c, c->g, c->vt, SL_GV);
            RET(read_scalars(c));
            gv = c->h_scal[SL_GV];
        }
        double alpha = 1.0;
        bool accepted = false;
        double Jt = J;
        for (int ls = 0; ls < o.max_ls; ++ls) {
            if (yp) {
                launch_axpby(c, n2N, (float)alpha, c->vt, 1.f, y, -1, -1, c->ytrial);
                sp_vec(c, OP_QINV, 0.f, c->ytrial, c->vtrial);
                RET(objective_dev(c, c->vtrial, nt, c->ytrial));
            } else {
                launch_axpby(c, n2N, (float)alpha, c->vt, 1.f, v, -1, -1, c->vtrial);
                RET(objective_dev(c, c->vtrial, nt));
            }
            n_pde += 1;
            st.n_ls += 1;
            RET(read_scalars(c));
            Jt = c->h_scal[SL_JDATA] + c->h_scal[SL_JREG];
            if (std::isfinite(Jt) && Jt <= J + o.armijo_c1 * alpha * gv) { accepted = true; break; }
            alpha *= o.armijo_rho;
        }
        if (!accepted) {
            status = REG_ERR_LINESEARCH;
            // restore the linearization data of the current iterate for a consistent return
            RET(grad_at(v, y));
            n_pde += 2;
            break;
        }
        CK(cudaMemcpyAsync(v, c->vtrial, vb, cudaMemcpyDeviceToDevice, c->stream));
        if (yp) CK(cudaMemcpyAsync(y, c->ytrial, vb, cudaMemcpyDeviceToDevice, c->stream));
        ++k;
        nt = nt_for(c, v, o, &cfl);
        if (nt < 0) return reg_fail(REG_ERR_CUDA, "scalar readback failed");
        RET(grad_at(v, y));
        n_pde += 2;
        gnorm2_to_slot();
        RET(read_scalars(c));
        J = c->h_scal[SL_JDATA] + c->h_scal[SL_JREG];
        gnorm = std::sqrt(c->h_scal[SL_GNORM2]);
        if (!std::isfinite(J) || !std::isfinite(gnorm)) status = REG_ERR_NAN;
    }
    // mismatch measure (Appendix F): ||m_R - m_1||^2 / ||m_R - m_T||^2
    launch_axpby(c, c->N, 1.f, c->mR, -1.f, c->mT, -1, -1, c->w0);
    {
        int np = launch_dot_partial(c, c->w0, c->w0, c->N, c->d_part);
        launch_finalize(c, c->d_part, np, c->d_scal + SL_DOT0, hh(c), 0, 0);
    }
    RET(read_scalars(c));
    const double r0 = c->h_scal[SL_DOT0];
    const double r1 = 2.0 * c->h_scal[SL_JDATA];
    st.n_newton = k;
    st.n_pde = n_pde;
    st.status = status;
    st.nt_used = nt;
    st.J = J;
    st.gnorm_rel = gref > 0 ? gnorm / gref : 0.0;
    st.rnorm_rel_sq = r0 > 0 ? r1 / r0 : 0.0;
    st.cfl = cfl;
    st.cfl_warn = cfl > o.cfl_max ? 1 : 0;
    if (stats) *stats = st;
    CKL();
    if (status == REG_ERR_NAN) return reg_fail(REG_ERR_NAN, "objective or gradient became non-finite");
    if (status == REG_ERR_LINESEARCH) return reg_fail(REG_ERR_LINESEARCH, "Armijo line search failed");
    if (status == REG_ERR_MAXIT) return reg_fail(REG_ERR_MAXIT, "Newton iteration cap reached");
    return status;
}

extern "C" int reg_register_host(reg_ctx* c, const float* mT_host, const float* mR_host, float* v_host,
                                 const reg_solve_opts* opts, reg_solve_stats* stats) {
    CTX_CHECK(c);
    if (!mT_host || !mR_host || !v_host) return reg_fail(REG_ERR_ARG, "host buffer is NULL");
    const size_t N = c->N;
    CK(cudaMemcpyAsync(c->mT, mT_host, sizeof(float) * N, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->mR, mR_host, sizeof(float) * N, cudaMemcpyHostToDevice, c->stream));
    c->have_lin = false;
    float* v = c->vtmp2;
    if (opts && opts->warm_start)
        CK(cudaMemcpyAsync(v, v_host, sizeof(float) * 2 * N, cudaMemcpyHostToDevice, c->stream));
    const int st = reg_solve(c, v, opts, stats);
    if (st == REG_ERR_ARG || st == REG_ERR_CUDA || st == REG_ERR_NOMEM) return st;
    CK(cudaMemcpyAsync(v_host, v, sizeof(float) * 2 * N, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return st;
}

// ---------------------------------------------------------------------------
// displacement field (Eq. (e:displacement)) and label overlap (Appendix F)
// ---------------------------------------------------------------------------
extern "C" int reg_displacement(reg_ctx* c, const float* v, float* u_out) {
    CTX_CHECK(c);
    RET(check_ptr(v, "v")); RET(check_ptr(u_out, "u_out"));
    const int nt = c->nt;
    const size_t N = c->N;
    // Component a solves d_t u_a + grad u_a . v = v_a from u_a = 0: the incremental-state
    // stage with source -(e . grad) where grad := v at every time and e = -(unit vector a),
    // so that the source is exactly v_a in FP32.
    float* e = c->vtmp;
    for (int comp = 0; comp < 2; ++comp) {
        launch_fill(c, 2 * (long long)N, e, 0.f);
        launch_fill(c, N, e + comp * N, -1.f);
        inc_state_solve(c, v, e, nt, nullptr, v);
        CK(cudaMemcpyAsync(u_out + comp * N, c->w3, sizeof(float) * N, cudaMemcpyDeviceToDevice, c->stream));
    }
    CKL();
    return REG_OK;
}

extern "C" int reg_label_overlap(reg_ctx* c, const float* v, const float* labels_T, const float* labels_R,
                                 float* transported, double* measures) {
    CTX_CHECK(c);
    RET(check_ptr(v, "v")); RET(check_ptr(labels_T, "labels_T")); RET(check_ptr(labels_R, "labels_R"));
    if (transported) RET(check_ptr(transported, "transported"));
    if (!measures) return reg_fail(REG_ERR_ARG, "measures is NULL");
    const int nt = c->nt;
    RET(ensure_nt(c, nt));
    // Gaussian filter, standard deviation 3 h_x (h_x = 2 pi / n1): symbol exp(-sigma^2 |k|^2 / 2)
    const double hx = 2.0 * M_PI / c->n1;
    const float a = (float)(0.5 * 9.0 * hx * hx);
    float* sm = c->vtmp;
    launch_r2c_scalar(c, labels_T, c->S[0]);
    const float2* in[1] = {c->S[0]};
    float2* o[1] = {c->S[1]};
    launch_col(c, OP_SMOOTH, in, o, spec_params(c, a), nullptr);
    launch_c2r_scalar(c, c->S[1], sm);
    state_solve(c, v, nt, sm);  // overwrites the state history
    c->have_lin = false;
    if (transported)
        CK(cudaMemcpyAsync(transported, mh(c, nt), sizeof(float) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    const int np = launch_overlap_counts(c, mh(c, nt), labels_R, 0.5f, c->d_part);
    for (int q = 0; q < 3; ++q) launch_finalize(c, c->d_part + q * np, np, c->d_scal + SL_DOT0 + q, 1.0, 0, 0);
    CKL();
    RET(read_scalars(c));
    const double nT = c->h_scal[SL_DOT0], nR = c->h_scal[SL_DOT1], nB = c->h_scal[SL_DOT2];
    const double nU = nT + nR - nB;
    measures[0] = nU > 0 ? nB / nU : 1.0;                    // Jaccard
    measures[1] = nT + nR > 0 ? 2.0 * nB / (nT + nR) : 1.0;  // Dice
    measures[2] = nT > 0 ? (nT - nB) / nT : 0.0;             // false positive error
    measures[3] = nR > 0 ? (nR - nB) / nR : 0.0;             // false negative error
    return REG_OK;
}

// ---------------------------------------------------------------------------
// deformation gradient (Eq. (e:def-grad)) and its measures (Appendix F)
// ---------------------------------------------------------------------------
static void detgrad_launches(reg_ctx* c, const float* v, float* detF, int nt) {
    const size_t N = c->N;
    const float h = 1.0f / (float)nt;
    sp_grad_vec(c, v, c->gv);
    float* Fa = c->F;     // F_j
    float* Fb = c->gtmp;  // F_{j+1} (ping-pong)
    launch_fill(c, 4 * (long long)N, Fa, 0.f);  // F(0) = I
    launch_fill(c, N, Fa, 1.f);
    launch_fill(c, N, Fa + 3 * N, 1.f);
    for (int j = 0; j < nt; ++j) {
        for (int comp = 0; comp < 4; ++comp) sp_grad(c, Fa + comp * N, c->gF + 2 * comp * N);
        launch_defgrad_stage(c, 1, Fa, nullptr, c->gF, c->gv, v, h, c->Fs);
        for (int comp = 0; comp < 4; ++comp) sp_grad(c, c->Fs + comp * N, c->gF + 2 * comp * N);
        launch_defgrad_stage(c, 2, Fa, c->Fs, c->gF, c->gv, v, h, Fb);
        float* t = Fa; Fa = Fb; Fb = t;
    }
    const int np = launch_det_stats(c, Fa, detF, c->d_part);
    launch_finalize(c, c->d_part + 0 * np, np, c->d_scal + SL_DET0 + 0, 1.0, 0, 2);
    launch_finalize(c, c->d_part + 1 * np, np, c->d_scal + SL_DET0 + 1, 1.0 / (double)N, 0, 0);
    launch_finalize(c, c->d_part + 2 * np, np, c->d_scal + SL_DET0 + 2, 1.0, 0, 1);
    launch_finalize(c, c->d_part + 3 * np, np, c->d_scal + SL_DET0 + 3, 1.0, 0, 1);
    launch_finalize(c, c->d_part + 4 * np, np, c->d_scal + SL_DET0 + 4, 1.0 / (double)N, 0, 0);
}

extern "C" int reg_detgrad(reg_ctx* c, const float* v, float* detF, double* stats) {
    CTX_CHECK(c);
    RET(check_ptr(v, "v"));
    if (detF) RET(check_ptr(detF, "detF"));
    const int nt = c->nt;
    RET(run_seq(c, GK_DETGRAD, v, detF, nt, [&] { detgrad_launches(c, v, detF, nt); }));
    if (stats) {
        RET(read_scalars(c));
        for (int q = 0; q < 5; ++q) stats[q] = c->h_scal[SL_DET0 + q];
    }
    return REG_OK;
}

// ---------------------------------------------------------------------------
// instrumentation
// ---------------------------------------------------------------------------
static void drain_events(reg_ctx* c) {
    cudaStreamSynchronize(c->stream);
    for (auto g : c->timing_graphs) cudaGraphExecDestroy(g);
    c->timing_graphs.clear();
    if (c->events.empty()) return;
    for (auto& e : c->events) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e.a, e.b);
        c->tcount[e.kclass]++;
        c->tms[e.kclass] += ms;
        c->tbytes[e.kclass] += e.bytes;
    }
    c->events.clear();
}

extern "C" int reg_kernel_timing(reg_ctx* c, int enable) {
    CTX_CHECK(c);
    drain_events(c);
    for (int k = 0; k < KC_COUNT; ++k) { c->tcount[k] = 0; c->tms[k] = 0.0; c->tbytes[k] = 0.0; }
    c->timing = enable != 0;
    return REG_OK;
}

extern "C" int reg_kernel_time(reg_ctx* c, int kclass, long long* launches, double* ms, double* bytes) {
    CTX_CHECK(c);
    if (kclass < 0 || kclass >= KC_COUNT) return reg_fail(REG_ERR_ARG, "bad kernel class");
    drain_events(c);
    if (launches) *launches = c->tcount[kclass];
    if (ms) *ms = c->tms[kclass];
    if (bytes) *bytes = c->tbytes[kclass];
    return REG_OK;
}

extern "C" long long reg_launch_count(reg_ctx* c) { return c ? c->launches : 0; }
