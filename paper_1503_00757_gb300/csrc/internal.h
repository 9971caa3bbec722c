// Internal declarations shared by kernels.cu (device code and launchers) and
// api.cu (C ABI and Newton-Krylov orchestration).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/reg.h"

// Spectral operations applied by the column-pass kernel (per wavenumber k):
enum SpecOp {
    OP_GRAD = 0,     // 1 in -> 2 out: (i k1~ x, i k2~ x)
    OP_DIV = 1,      // 2 in -> 1 out: i k1~ x0 + i k2~ x1
    OP_REG = 2,      // 2 in -> 2 out: coefA A^(k) x
    OP_PROJ = 3,     // 2 in -> 2 out: K^(k) x
    OP_PRECOND = 4,  // 2 in -> 2 out: x / (beta_v A'^(k)), A'(0) = 1
    OP_ASSEMBLE = 5, // 4 in -> 2 out: coefA A^(k) x01 + K^(k) x23
    OP_ENERGY = 6,   // 2 in -> 0 out: FP64 sum of the quadratic regularization energy
    OP_DIVT_PROJ = 7, // 5 in -> 2 out: P_L(coefA * div(T) + b), T = (T11, T12, T22)
    OP_GRAD1 = 8,     // 1 in -> 1 out: i k1~ x (d2 is diagonal in the row spectra; see AdvArgs::Sd2)
    OP_DIV1 = 9,      // in[0] transformed, in[1] raw -> 1 out: i k1~ x0 + (i k2~ / n2) x1 (x1 not transformed)
    OP_SMOOTH_PROJ = 10, // 2 in -> 2 out: exp(-coefA |k|^2) P_L x (Gaussian low-pass, then Leray)
    // Preconditioned coordinates y = Q v, Q^ = (beta_v A'^)^(1/2), A'(0) = 1 (reg_solve, quadratic regularization):
    OP_QINV = 11,        // 2 in -> 2 out: Q^-1 x
    OP_QMUL = 12,        // 2 in -> 2 out: Q x
    OP_ASSEMBLE_Y = 13,  // 4 in -> 2 out: Pi0 x01 + Q^-1 K^ x23 (Pi0 drops k = 0): gradient / Hessian in y
    OP_QNORM = 14,       // 2 in -> 0 out: FP64 sum of |Q x|^2 (the v-norm of a y-space gradient or residual)
    OP_ENERGY_Y = 15,    // 2 in -> 0 out: FP64 regularization energy of v = Q^-1 x from x
    OP_SMOOTH = 16,      // 1 in -> 1 out: exp(-coefA |k|^2) x (Gaussian filter of a scalar field)
    OP_MASSP = 17        // 2 in -> 2 out: k~ k~^T x / (|k~|^2 m), m = 1 + 2 beta_v eta_bar / (beta_w (1 + |k|^2))
};

// Projection modes (Eq. (e:project-body-force)):
enum ProjMode { PROJ_IDENTITY = 0, PROJ_LERAY = 1, PROJ_MASS = 2 };

struct SpecParams {
    float scale;    // 1 / (n1 n2)
    float coefA;    // coefficient of A^ (beta_v for the gradient/Hessian)
    float beta_v;   // regularization weight
    float beta_w;   // mass-source weight (PROJ_MASS)
    int regnorm;    // 1 = H1, 2 = H2
    int pmode;      // ProjMode
    double escale;  // OP_ENERGY: h1 h2 / (n1 n2)
    double ebv;     // OP_ENERGY: beta_v / 2
    double ebw;     // OP_ENERGY: beta_w / 2 (0 unless PROJ_MASS)
    const double* eta_bar;  // OP_MASSP: device scalar, the mean viscosity of the shear model
};

enum KClass { KC_COL = 0, KC_ROWSTAGE = 1, KC_ROW = 2, KC_POINT = 3, KC_TRANSPORT = 4, KC_COUNT = 5 };

// Device-scalar slots (doubles) in reg_ctx::d_scal.
enum Slot {
    SL_JDATA = 0, SL_JREG = 1, SL_DOT0 = 2, SL_DOT1 = 3, SL_DOT2 = 4, SL_RZ = 5, SL_SHS = 6,
    SL_RZNEW = 7, SL_RNORM2 = 8, SL_VMAX = 9, SL_GNORM2 = 10, SL_GV = 11,
    SL_DET0 = 12, /* 5 slots */ SL_ETABAR = 17, SL_ONE = 18, SL_COUNT = 20
};

struct EventPair { cudaEvent_t a, b; int kclass; double bytes; };

// A captured launch sequence, replayed with cudaGraphLaunch.  Keyed by the
// kind of sequence, the caller pointers it was captured with and nt.
struct GraphEntry {
    int kind;
    const void* p0;
    const void* p1;
    int nt;
    cudaGraphExec_t exec;
    long long nkern;
};

struct reg_ctx {
    int n1, n2, N, log1, log2;
    int nt;          // requested nt
    int nt_cap;      // history capacity
    int regnorm;
    double beta_v, beta_w, shear, nu;
    int pmode;
    bool shear_model;
    cudaStream_t stream;

    // images and history
    float *mT, *mR;
    float *m_hist;   // (nt_cap + 1) * N
    float *gm_hist;  // (nt_cap + 1) * 2N
    // linearization point
    float* v_lin;    // 2N
    int nt_lin;
    bool have_lin;
    // shear-model linearization data: E(v) (3 planes) and eta (1 plane)
    float *E_lin, *eta_lin;

    // spectra (transposed packed layout, N/2 float2 each)
    float2 *S[6];
    // scalar work fields
    float *w0, *w1, *w2, *w3;
    // vector work fields (2N each)
    float *bvec, *vtmp, *vtmp2, *gtmp, *T3;  // T3: 3 planes
    float *T3b, *vx;  // shear model with a mass source: a second tensor (3 planes), a vector (2N)
    // PCG / solve workspace (2N each)
    float *g, *r, *z, *s, *Hs, *vt, *vtrial;
    // preconditioned coordinates y = Q v of reg_solve (2N each): iterate, trial iterate, Q^-1 of a direction
    float *ybuf, *ytrial, *vtil;
    bool ypath;      // reg_solve iterates on y (quadratic H2 regularization, see reg_solve)
    // det F workspace
    float *F, *Fs, *gF, *gv;  // 4N, 4N, 8N, 4N

    double* d_scal;  // SL_COUNT
    double* d_part;  // partial sums
    int npart;
    double* h_scal;  // pinned host mirror

    float2* tw;      // twiddle tables (REG_TW_TOTAL entries, fft.cuh layout)

    // full Newton Hessian (reg_set_hessian): adjoint history lam_j of the gradient and the
    // incremental state's gradient history grad m~_j (allocated while enabled)
    bool full_newton;
    float *lam_hist;   // (nt_cap + 1) * N
    float *gmt_hist;   // (nt_cap + 1) * 2N
    bool tc_ok;        // the cluster-resident transport kernel can run on this grid and device
    bool use_tc;       // transport solves run in the cluster-resident kernel (else the two-pass kernels)
    int tileR, tileC;  // rows per row-kernel CTA, spectrum columns per column-kernel CTA (0: default)
    int tileP;         // 1: RK2 row kernels prefetch their operands (used when tileR > 0)

    long long launches;
    bool pdl;         // launch with programmatic dependent launch (default on)
    bool use_graphs;
    std::vector<GraphEntry> graphs;
    std::vector<cudaGraphExec_t> timing_graphs;  // one-off captures made while timing is on
    bool timing;
    std::vector<EventPair> events;
    std::vector<cudaEvent_t> event_pool;
    long long tcount[KC_COUNT];
    double tms[KC_COUNT];
    double tbytes[KC_COUNT];
};

// ---- FFT tile choices (kernels.cu: defaults and limits; tune.cu: autotuner table) ----
void default_tiles(int n1, int n2, int* R, int* C, int* P);
bool tiles_valid(int n1, int n2, int R, int C, int P);
// tuned (R, C, P, D, T) for this device and grid, if reg_autotune has measured it (D: launch with
// PDL; T: transports in the cluster-resident kernel; T nullable)
bool tuned_tiles(int dev, int n1, int n2, int* R, int* C, int* P, int* D, int* T);

// ---- launchers (kernels.cu); all asynchronous on ctx->stream ----
cudaError_t k_init_twiddles(reg_ctx* ctx);
// host: fill the REG_TW_TOTAL twiddle entries (fft.cuh layout) from FP64 sin / cos
void fill_twiddles(float2* h);
// shared memory of a row kernel with R rows of length L, and of the column kernel with C columns
size_t row_smem(int R, int L);
size_t col_smem(int C, int L, bool div1);

void launch_r2c_scalar(reg_ctx* ctx, const float* f, float2* S);
void launch_r2c_vec(reg_ctx* ctx, const float* u1, const float* u2, float2* S1, float2* S2);
void launch_c2r_scalar(reg_ctx* ctx, const float2* S, float* f);
void launch_c2r_vec(reg_ctx* ctx, const float2* S1, const float2* S2, float* u1, float* u2);
void launch_col(reg_ctx* ctx, int op, const float2* const* in, float2* const* out, const SpecParams& P,
                double* part_out);

struct AdvArgs {
    const float2 *G1, *G2;  // spectra of d1 u_s, d2 u_s; G1 == nullptr -> zero gradient
    const float2* Sd2;      // G2 == nullptr: row spectrum of u_s, d2 u_s = (i k2~ / n2) Sd2
    const float *uj, *us;   // u_j (nullptr: u_j = 0) and the stage-2 input u* (stage 1: us unused)
    const float* v;         // velocity (2N)
    const float* gm;        // grad m at the source time (2N); nullptr -> no source
    const float* vt;        // incremental velocity (2N)
    float* u_out;           // stage result
    float* grad_out;        // nullable: receives grad u_s (2N)
    float2* S_out;          // nullable: packed spectrum of u_out
    float h;
    int stage;
    int late;               // 1: load every operand after waiting on the preceding kernel (an operand
                            // may have been written by the launch just before this one)
};
void launch_row_adv(reg_ctx* ctx, const AdvArgs& a);

struct AdjArgs {
    const float2* D;        // spectrum of div(lam_s v)
    const float *lj, *ls;   // lam_j, stage-2 input lam*
    const float* v;
    float* l_out;
    float* b;               // nullable: body force accumulator (2N), stage 2 only
    const float* gm;        // grad m at the output time
    float w;                // trapezoid weight
    float2 *F1, *F2;        // nullable: flux spectra of l_out
    float h;
    int stage;
    // full Newton (nullable lsrc = Gauss-Newton): flux l_out v + lsrc v~; stage 2 also b += w lsrc gmt
    const float* lsrc;      // adjoint state lam at the time of the next divergence
    const float* vt;        // incremental velocity (2N)
    const float* gmt;       // grad m~ at the output time (2N)
};
void launch_row_adj(reg_ctx* ctx, const AdjArgs& a);

// lam = ca * a + cb * c (a nullable); b = w lam gm; flux spectra of lam v;
// optional FP64 partials of 0.5 * sum(lam^2) * h1 h2.  Full Newton (lsrc != nullptr):
// b += w lsrc gmt and the flux is lam v + lsrc vt.
void launch_adj_init(reg_ctx* ctx, const float* a, float ca, const float* c, float cb, const float* v,
                     float* lam, float* b, const float* gm, float w, float2* F1, float2* F2, double* part,
                     const float* lsrc = nullptr, const float* vt = nullptr, const float* gmt = nullptr);

// ---- pointwise / reductions ----
// part[...] <- partial sums of sum_i x_i y_i over n elements; returns #partials
int launch_dot_partial(reg_ctx* ctx, const float* x, const float* y, long long n, double* part);
// part[...] <- partial sums of sum_i x_i over n elements; returns #partials
int launch_sum_partial(reg_ctx* ctx, const float* x, long long n, double* part);
int launch_maxnorm_partial(reg_ctx* ctx, const float* v, int N, double* part);
// out[slot] = scale * sum(part[0..np)) (+ out[slot] if accumulate); op 0 = sum, 1 = max, 2 = min
void launch_finalize(reg_ctx* ctx, const double* part, int np, double* out, double scale, int accumulate, int op);
// y = a * x + b * y, with optional device-scalar factor: if (num >= 0) a *= d_scal[num] / d_scal[den]
void launch_axpby(reg_ctx* ctx, long long n, float a, const float* x, float b, float* y, int num, int den,
                  float* out);
// PCG step: vt += kappa s; r -= kappa Hs; partial sum r^2; kappa = d_scal[SL_RZ] / d_scal[SL_SHS];
// no update when d_scal[SL_SHS] <= 0
int launch_pcg_update(reg_ctx* ctx, long long n, float* vt, const float* s, float* r, const float* Hs, double* part);
// s = z + (d_scal[SL_RZNEW] / d_scal[SL_RZ]) s
void launch_pcg_dir(reg_ctx* ctx, long long n, const float* z, float* s);
void launch_fill(reg_ctx* ctx, long long n, float* y, float val);

// label overlap: part[0 * nb + b], part[1 * nb + b], part[2 * nb + b] <- block b's counts of
// (f > thr), (L > 0.5) and both; returns nb
int launch_overlap_counts(reg_ctx* ctx, const float* f, const float* L, float thr, double* part);

// deformation gradient
void launch_defgrad_stage(reg_ctx* ctx, int stage, const float* F, const float* Fs, const float* gF,
                          const float* gv, const float* v, float h, float* out);
int launch_det_stats(reg_ctx* ctx, const float* F, float* detF, double* part);

// shear model
// from grad v (gv: d1v1, d2v1, d1v2, d2v2) compute E (3 planes) and eta; and
// optionally T = 2 eta E (3 planes) and energy partials
int launch_shear_strain(reg_ctx* ctx, const float* gv, float nu, float* E, float* eta, float* T, double* part);
// T' = 2 eta (E~ + q E), q = ((1-nu)/nu) (E : E~) / (E:E + eps^2), E~ from grad v~
void launch_shear_second(reg_ctx* ctx, const float* gvt, const float* E, const float* eta, float nu, float* T);

// timing hooks
// bytes: algorithmic bytes of the launch (each input read once, each output written once)
void ktimer_begin(reg_ctx* ctx, int kclass, double bytes);
void ktimer_end(reg_ctx* ctx);

int reg_fail(int status, const std::string& msg);

// out = exp(-a |k|^2) P_L b on the context's grid (velocity fields, device):
// the output map of the warm-start network (Gaussian low-pass, then Leray).
int apply_smooth_proj(reg_ctx* ctx, float a, const float* b, float* out);

// ---- cluster-resident transport solves (transport_cluster.cu) ----
enum TcMode { TC_STATE = 0, TC_ADJOINT = 1, TC_MATVEC = 2 };
struct TcArgs {
    int nt;
    float h;                 // 1 / nt
    const float* v;          // velocity (2N)
    const float* vt;         // incremental velocity (2N, TC_MATVEC)
    const float* mT;         // template (TC_STATE)
    float* m_hist;           // (nt+1) N: written by TC_STATE; m_nt read by TC_ADJOINT through adj_c
    float* gm_hist;          // 2 (nt+1) N: written by TC_STATE, read by the others
    float* uj;               // TC_MATVEC: m~_j (ends as m~_nt)
    float* us;               // stage-2 input of the forward sweep (u*)
    float* lj;               // adjoint lam_j
    float* ls;               // adjoint lam*
    const float* adj_a;      // lam_nt = adj_ca adj_a + adj_cb adj_c (adj_a nullable; TC_MATVEC uses uj for adj_c)
    float adj_ca;
    const float* adj_c;
    float adj_cb;
    float* b;                // body force (2N): written
    const float2* tw;        // twiddle table (set by the launcher)
};
// CTAs per cluster for an n x n grid, and how many such clusters fit on the current device
// at once (0: the cluster kernel cannot run on this grid or device)
int tc_cluster_size(int n);
int tc_max_active_clusters(int n1, int n2);
void launch_transport_cluster(reg_ctx* ctx, int mode, const TcArgs& a);
