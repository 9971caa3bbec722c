/*
 * reg.h - C ABI of the GB300 (sm_103a) implementation of the reduced-space
 * Gauss-Newton-Krylov solver for constrained H1/H2-regularized stationary-
 * velocity image registration of Mang & Biros, "Constrained H1-regularization
 * schemes for diffeomorphic image registration" (arXiv 1503.00757).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.  n1 x n2 nodes on the periodic domain [0, 2 pi)^2 (the paper's
 *   (-pi, pi)^2 shifted by a period, Sec. 1.5); node (i, j) is at
 *   x = (2 pi i / n1, 2 pi j / n2).  n1 and n2 are powers of two in [16, 1024].
 * Layout.  A scalar field is n1*n2 floats, row-major, index i*n2 + j (x^2
 *   fastest).  A vector field is two scalar planes back to back (component 1
 *   then component 2, 2*n1*n2 floats).  Buffers must be 16-byte aligned.
 * Memory.  Unless an entry point says "host", every float/double pointer is a
 *   DEVICE pointer owned by the caller.  The library never frees or retains a
 *   caller pointer beyond the call.  Scalar outputs (double*) are HOST pointers.
 *   The context owns its own device workspace (state history etc.).
 * Streams.  Work is issued on the context stream (reg_set_stream; default:
 *   the legacy default stream).  Entry points that return host scalars
 *   synchronize that stream; the others are asynchronous.
 * Errors.  Every entry point returns a reg_status.  Invalid arguments are
 *   rejected with REG_ERR_ARG before any launch.  A CUDA error is returned as
 *   REG_ERR_CUDA (the message is available from reg_last_error).  Non-finite
 *   objective or gradient values are reported as REG_ERR_NAN.
 * Threading.  A context is not thread-safe; distinct contexts are independent.
 * Precision.  Fields, FFTs and transport run in FP32; objective values,
 *   norms, inner products and the det(F) statistics are accumulated in FP64.
 */
#ifndef REG_H
#define REG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct reg_ctx reg_ctx;

typedef struct {
    int n1; /* nodes along x^1 (rows) */
    int n2; /* nodes along x^2 (columns, contiguous) */
} reg_grid;

enum reg_norm { REG_H1 = 1, REG_H2 = 2, REG_H3 = 3 };

enum reg_status {
    REG_OK = 0,
    REG_ERR_ARG = 1,
    REG_ERR_CUDA = 2,
    REG_ERR_NOMEM = 3,
    REG_ERR_NAN = 4,
    REG_ERR_LINESEARCH = 5,
    REG_ERR_PCG_MAXIT = 6, /* reported in stats, not returned */
    REG_ERR_TIMEOUT = 7,
    REG_WARN_CFL = 8,      /* reported in stats, not returned */
    REG_ERR_STATE = 9,     /* call order violated (e.g. matvec before gradient) */
    REG_ERR_MAXIT = 10     /* Newton iteration cap reached before the tolerance */
};

enum reg_nt_policy { REG_NT_FIXED = 0, REG_NT_CFL = 1 };

/* Options of the Newton-Krylov solve (Algorithm 1, Algorithm 2, Sec. 4).
 * reg_default_opts fills the defaults given in brackets. */
typedef struct {
    double tol;          /* [1e-2] stop when ||g_k|| / ||g_ref|| <= tol */
    int maxit_newton;    /* [50]  outer iteration cap */
    int maxit_pcg;       /* [100] Hessian matvecs per PCG solve */
    double armijo_c1;    /* [1e-4] sufficient decrease constant */
    double armijo_rho;   /* [0.5] backtracking factor */
    int max_ls;          /* [20]  backtracking steps before REG_ERR_LINESEARCH */
    int nt_policy;       /* [REG_NT_FIXED] or REG_NT_CFL */
    double cfl_max;      /* [0.25] CFL number targeted by REG_NT_CFL */
    int warm_start;      /* [0] 1: v_inout holds the initial guess; the stopping test
                            stays relative to g_ref = g(0), the PCG forcing term is
                            relative to the gradient at the initial guess */
} reg_solve_opts;

/* Statistics of one solve (the measures of the paper's Tab. 1 / Appendix F). */
typedef struct {
    int n_newton;        /* outer iterations */
    int n_mv;            /* Gauss-Newton Hessian matvecs */
    int n_pde;           /* hyperbolic PDE solves (state, adjoint, 2 per matvec) */
    int n_ls;            /* line-search objective evaluations */
    int n_pcg_maxit;     /* PCG solves that hit maxit_pcg */
    int status;          /* final reg_status */
    int nt_used;         /* time steps at the end of the solve */
    int cfl_warn;        /* 1 if the CFL number exceeded cfl_max (fixed policy) */
    double J0, J;        /* objective at the start / end */
    double gnorm_rel;    /* ||g_k*|| / ||g_ref|| */
    double rnorm_rel_sq; /* ||m_R - m_1||^2 / ||m_R - m_T||^2 (Appendix F) */
    double cfl;          /* CFL number max|v| nt^-1 / h_x at the end */
} reg_solve_stats;

/* Error string of the last failing call on this thread (never NULL). */
const char* reg_last_error(void);

void reg_default_opts(reg_solve_opts* opts);

/* Create a context.  Problem (Eq. (e:objective)-(e:constraint-divv)):
 *   nt       time steps of the RK2 transport solves (Sec. 4), >= 1;
 *   regnorm  REG_H1 or REG_H2 seminorm on v (Eq. (e:reg-v)), or REG_H3 (the
 *            triharmonic control equation App. A.1 names: symbol |k|^6);
 *   beta     beta_v > 0;
 *   gamma    beta_w of the mass-source H1 norm (Eq. (e:reg-w)); 0 disables the
 *            divergence constraint (the paper's gamma = 0); +INFINITY enforces
 *            div v = 0 (w = 0); a finite positive value is the mass-source
 *            weight beta_w;
 *   shear    s in (-1, 1); s != 0 selects the nonlinear Stokes model
 *            (Eq. (e:shear-control-reg-v)) with nu = (1 + s) / (1 - s); it
 *            requires REG_H1.  With 0 < gamma < inf the mass source is
 *            eliminated as in App. A.2 (M = 2 beta_v eta_bar (beta_w(-Lap +
 *            I))^-1 + I with eta_bar the mean viscosity); gamma = 0 applies
 *            no projection.
 * Allocates the device workspace on the current device. */
int reg_create(reg_grid grid, int nt, int regnorm, double beta, double gamma, double shear, reg_ctx** out);
void reg_destroy(reg_ctx* ctx);

/* Re-parameterize an existing context for another problem on the same grid
 * (same meaning and checks as reg_create); keeps the device workspace,
 * growing the state history if nt grows.  Invalidates the linearization point. */
int reg_set_params(reg_ctx* ctx, int nt, int regnorm, double beta, double gamma, double shear);

/* Issue all work on `stream` (a cudaStream_t; NULL = legacy default stream). */
int reg_set_stream(reg_ctx* ctx, void* stream);

/* Copy the template m_T and reference m_R (device, n1*n2 floats) into the
 * context (Eq. (e:objective), (e:init-transport-eq)). */
int reg_set_images(reg_ctx* ctx, const float* mT, const float* mR);

/* ---- spectral operators (Sec. 4, pseudospectral discretization) ---- */

/* grad f (2*n1*n2 out) of a scalar field f; odd symbol i k with the Nyquist
 * wavenumber set to 0. */
int reg_spectral_grad(reg_ctx* ctx, const float* f, float* grad_f);
/* div u (n1*n2 out) of a vector field u; same odd symbol. */
int reg_spectral_div(reg_ctx* ctx, const float* u, float* div_u);
/* beta_v A[v] (Eq. (e:var-reg-v)); for the shear model beta_v A[v] of
 * Eq. (e:1st-var-reg-v-nls). */
int reg_apply_reg(reg_ctx* ctx, const float* v, float* out);
/* K[b] (Eq. (e:project-body-force)); Leray projection for gamma = inf,
 * identity for gamma = 0. */
int reg_apply_proj(reg_ctx* ctx, const float* b, float* out);
/* (beta_v A)^-1 r with the k = 0 symbol replaced by 1 (Appendix E); the
 * inverse vector Laplacian for the shear model. */
int reg_apply_precond(reg_ctx* ctx, const float* r, float* out);

/* Square root of the preconditioner, Q = (beta_v A')^(1/2) with A'(0) = 1
 * (App. E.2): out = Q x (inverse = 0) or Q^-1 x (inverse != 0), per Fourier
 * mode, on a velocity field (2 n1 n2 floats, device).  reg_solve iterates on
 * y = Q v for the H2 and H3 seminorms. */
int reg_apply_precond_sqrt(reg_ctx* ctx, const float* x, float* out, int inverse);

/* ---- state solve, objective, adjoint, reduced gradient ---- */

/* Forward state solve (Eq. (e:state-eq-elim)) and objective J[v]
 * (Eq. (e:objective)).  m1 (nullable) receives m(t = 1); J (nullable, host). */
int reg_objective(reg_ctx* ctx, const float* v, float* m1, double* J);
/* Reduced gradient g = beta_v A[v] + K[b] (Eq. (e:control-eq-elim)), state
 * and adjoint solves of Algorithm 1.  g: 2*n1*n2 out; J (nullable, host).
 * Fixes the linearization point for reg_hessian_matvec. */
int reg_gradient(reg_ctx* ctx, const float* v, float* g, double* J);

/* ---- Gauss-Newton Hessian matvec ---- */

/* H v~ = beta_v B[v~] + L[b~] (Eq. (e:inc-control-eq-elim)) with the
 * Gauss-Newton approximation (lambda terms dropped, Sec. 4), or the full
 * Newton Hessian (reg_set_hessian), at the v of the last reg_gradient call
 * (REG_ERR_STATE otherwise). */
int reg_hessian_matvec(reg_ctx* ctx, const float* vt, float* Hvt);

/* Hessian of reg_hessian_matvec and reg_solve.  full = 0 (default): Gauss-
 * Newton (Sec. 4: lambda set to zero in Eq. (e:second-order-elim)).  full != 0:
 * the full Newton Hessian of Eq. (e:second-order-elim): the incremental
 * adjoint keeps its source -div(lam v~) and the incremental body force is
 * b~ = int lam~ grad m + lam grad m~ dt (trapezoid in time), with lam the
 * adjoint of the last reg_gradient (whose history the context then stores:
 * (nt+1) n1 n2 floats more, and 2 (nt+1) n1 n2 for grad m~).  This Hessian
 * need not be positive definite away from a minimizer; PCG stops at a
 * non-positive curvature and the line search falls back to the
 * preconditioned gradient step (reg_solve).  Transport solves then run on the
 * row/column kernel pairs (reg_set_transport is ignored).  Invalidates the
 * linearization point.  REG_ERR_NOMEM if the histories cannot be allocated. */
int reg_set_hessian(reg_ctx* ctx, int full);

/* Body force of the last reg_gradient (b = int lam grad m dt, Sec. 3.1) or
 * incremental body force of the last reg_hessian_matvec (b~ with the
 * Gauss-Newton approximation, Sec. 3.2 / Sec. 4), before the projection K:
 * b_out (device, 2*n1*n2).  REG_ERR_STATE if neither has run. */
int reg_body_force(reg_ctx* ctx, float* b_out);

/* ---- Newton-Krylov solve (Algorithms 1 and 2) ---- */

/* v_inout (device, 2*n1*n2): initial guess if opts->warm_start, else ignored
 * (v_0 = 0); receives the final velocity.  opts NULL = defaults.  stats
 * (nullable, host).  Returns REG_OK, REG_ERR_LINESEARCH, REG_ERR_MAXIT,
 * REG_ERR_NAN or an argument/CUDA error.  With the H2 or H3 seminorm (and no
 * shear term) the iteration runs on y = Q v, Q = (beta_v A')^(1/2) (see
 * reg_apply_precond_sqrt): the same Algorithms 1 and 2, with PCG on v
 * becoming unpreconditioned CG on y and every test taken on v-space norms,
 * so that the FP32 rounding of v is not amplified by beta_v |k|^4 (|k|^6 for
 * H3) in the gradient. */
int reg_solve(reg_ctx* ctx, float* v_inout, const reg_solve_opts* opts, reg_solve_stats* stats);

/* Same solve with HOST buffers: copies m_T, m_R (host, n1*n2 floats) to the
 * device, solves, and copies v (host, 2*n1*n2 floats; the initial guess when
 * opts->warm_start) back.  Synchronous. */
int reg_register_host(reg_ctx* ctx, const float* mT_host, const float* mR_host, float* v_host,
                      const reg_solve_opts* opts, reg_solve_stats* stats);

/* ---- batched registration of many independent pairs ---- */

/* One pair of a batch.  Inputs: grid, nt, regnorm, beta, gamma, shear (as in
 * reg_create), mT and mR (device, n1*n2 floats each), want_detgrad (1: also
 * run reg_detgrad on the solution).  In/out: v (device, 2*n1*n2 floats; the
 * initial guess when opts->warm_start, else ignored; receives the solution).
 * Outputs: stats, detgrad (min, mean, max det F1, max and mean D, when
 * want_detgrad) and status (the reg_solve / reg_detgrad return code). */
typedef struct {
    reg_grid grid;
    int nt;
    int regnorm;
    double beta, gamma, shear;
    const float* mT;
    const float* mR;
    float* v;
    int want_detgrad;
    reg_solve_stats stats;
    double detgrad[5];
    int status;
} reg_batch_item;

/* Solve `count` independent registrations (Algorithm 1 per pair) on the
 * current device with `nworkers` host workers (<= 0: 8), each issuing its
 * pairs on its own CUDA stream with per-grid-size contexts it creates once
 * and re-parameterizes per pair (reg_set_params), so the pairs' kernels run
 * concurrently.  Pairs are taken largest grid first.  Before the first pair
 * of a grid size is solved, reg_autotune picks that size's FFT tiles for
 * min(nworkers, 8) concurrent solves at the largest nt of the batch's pairs
 * of that size (once per process and device).  Every pair's result is identical to reg_solve on
 * that pair alone with a context created after that tuning.  Synchronous.  Returns REG_OK if
 * every pair returned REG_OK, else the first failing pair's status (each
 * item's own status is in item.status); REG_ERR_ARG for invalid arguments. */
int reg_solve_batch(reg_batch_item* items, int count, const reg_solve_opts* opts, int nworkers);

/* A persistent batch executor: the same scheduling as reg_solve_batch, but
 * its worker streams, per-grid-size contexts and their captured launch
 * sequences stay alive across calls (reg_solve_batch builds and frees one per
 * call).  Create on the device that will run the pairs (nworkers <= 0: 8). */
typedef struct reg_executor reg_executor;
int reg_executor_create(int nworkers, reg_executor** out);
int reg_executor_solve(reg_executor* ex, reg_batch_item* items, int count, const reg_solve_opts* opts);
void reg_executor_destroy(reg_executor* ex);

/* ---- autotuner of the FFT tiles and launch mode ---- */

/* Times the Gauss-Newton Hessian matvec (Algorithm 2's product with H, two
 * transport solves of nt steps) on an n1 x n2 grid with `concurrency` solves
 * running at once on their own streams (1: latency of one solve; > 1: the
 * throughput of that many, as in the batch executor), for every valid tile
 * choice (R rows per row-kernel CTA, C spectrum columns per column-kernel
 * CTA, P = 1 if the RK2 row kernels prefetch their operands before waiting on
 * the preceding kernel) with programmatic dependent launch on and off
 * (D, see reg_set_pdl), on the current device with zero images and velocity
 * and private streams, and records the fastest in a process-wide table;
 * contexts created afterwards on this device and grid use it (existing
 * contexts keep theirs).  Valid: R a multiple of 4 dividing n1,
 * 32 <= R n2 / 8 <= 512 threads; C a power of two >= 2 dividing n2 / 2,
 * 32 <= C n1 / 8 <= 256 threads; at most 227 KB of shared memory; P = 1 only
 * for n2 <= 512.  Every candidate is timed in two passes and keeps its faster
 * one.  A grid already in the table is not re-measured unless force != 0; a
 * cached answer sets *ms_per_matvec < 0, a measured one the winner's time per
 * matvec of the whole group.  Outputs are host pointers, each nullable.
 * Synchronous.
 * REG_ERR_ARG for a grid outside powers of two in [16, 1024], nt outside
 * [1, 4096] or concurrency outside [1, 16]. */
int reg_autotune(reg_grid grid, int nt, int concurrency, int force, int* rows_per_cta, int* cols_per_cta,
                 int* prefetch, int* pdl, double* ms_per_matvec);

/* The tiles and launch mode a context launches with (tuned, else the default
 * rule: the smallest R, C with at least 64 threads, P = 1 for n2 <= 512,
 * D = 1). */
int reg_tile_config(reg_ctx* ctx, int* rows_per_cta, int* cols_per_cta, int* prefetch, int* pdl);

/* Sets a context's tiles (validity as for reg_autotune; R = C = 0 restores
 * the default rule).  Results do not depend on the tiles except for the
 * summation order of FP64 reductions (objective, norms).  REG_ERR_ARG for
 * invalid tiles. */
int reg_set_tiles(reg_ctx* ctx, int rows_per_cta, int cols_per_cta, int prefetch);

/* ---- transport kernels ---- */

/* Selects how the transport solves (state, adjoint, and the incremental state and
 * adjoint of a Gauss-Newton matvec; Eqs. (e:state-eq-elim)-(e:inc-adj-eq-elim),
 * Heun steps of Sec. 4) run on this context:
 *   cluster != 0: one launch per solve (both sweeps of a matvec in one launch),
 *     resident in a thread-block cluster of max(1, n^2 / 16384) CTAs that keep
 *     the row spectra of the transported field in shared memory and exchange
 *     column slabs through distributed shared memory (square grids n x n,
 *     16 <= n <= 512, on devices with thread-block clusters);
 *   cluster == 0: a row kernel and a column kernel per Heun stage, the spectra
 *     passing through global memory (every grid).
 * Default: the two-kernel path (faster on a GB300 at every grid size and
 * concurrency measured: the cluster kernel keeps 16 warps per SM, too few to
 * hide the latency of its per-stage operand loads).  Results
 * agree to FP32 rounding (the transforms are the same; the order of a few
 * additions differs).  REG_ERR_ARG if cluster != 0 and this grid or device
 * cannot run it. */
int reg_set_transport(reg_ctx* ctx, int cluster);

/* The transport path of a context: *cluster = 1 for the cluster-resident
 * kernel; *ctas_per_cluster = its cluster size on this grid (0 if it cannot
 * run); *max_active_clusters = how many such clusters fit on the device at
 * once (cudaOccupancyMaxActiveClusters; independent solves on separate
 * streams run concurrently up to that number).  Host pointers, each nullable. */
int reg_transport_config(reg_ctx* ctx, int* cluster, int* ctas_per_cluster, int* max_active_clusters);

/* Programmatic dependent launch (default on): each kernel may start while its
 * predecessor finishes and waits on it in-kernel, which hides launch latency
 * for one solve; enable = 0 launches every kernel after its predecessor has
 * completed.  Results are identical either way. */
int reg_set_pdl(reg_ctx* ctx, int enable);

/* ---- arithmetic ceiling ---- */

/* FP32 FMA throughput of the current device, measured.  Not an operation of
 * the method: it is the arithmetic ceiling of the transform and RK2 kernels
 * (the pseudospectral FFTs and transport updates of Sec. 4 run in FP32 on the
 * CUDA cores), against which a matvec's FFT flop count is compared.  One wave
 * of 256-thread CTAs (SM count x CTAs resident per SM); each thread runs 16
 * independent FMA recurrences of 2048 steps.  After two warm-up launches,
 * three windows of five launches are timed with CUDA events; *tflops
 * (host, required) = 2 x FMAs per launch / the best window's time per launch,
 * in TFLOP/s; *ms_per_launch (host, nullable) = that time.  Runs on a stream
 * of its own, which it synchronizes; allocates 4 bytes of device memory for
 * the duration of the call.  REG_ERR_ARG if tflops is NULL, REG_ERR_NOMEM or
 * REG_ERR_CUDA if a CUDA call fails. */
int reg_fp32_peak(double* tflops, double* ms_per_launch);

/* ---- deformation gradient (Eq. (e:def-grad)) ---- */

/* Transports F (F(0) = I) with v; detF (nullable, device n1*n2) receives
 * det F1; stats (host, 5 doubles) receives min, mean, max of det F1 and max,
 * mean of D = ||F1 - I||_F (Appendix F). */
int reg_detgrad(reg_ctx* ctx, const float* v, float* detF, double* stats);

/* ---- deformation map and label overlap (App. D, App. F) ---- */

/* Displacement field u_1 = u(t = 1) of Eq. (e:displacement): d_t u + (grad u) v
 * = v, u(0) = 0, over the context's nt Heun steps (per component a transport
 * with the source v_a).  The deformation map is y = x - u_1 (Eulerian: where
 * the points originate from; App. D).  v: device, 2*n1*n2; u_out: device,
 * 2*n1*n2 (component planes).  Uses the context's work fields only;
 * asynchronous. */
int reg_displacement(reg_ctx* ctx, const float* v, float* u_out);

/* Label-map overlap after registration (the measures table of App. F and the
 * label evaluation of Sec. 5): the template label map (device, n1*n2 floats,
 * 1 inside the label, 0 outside) is smoothed with a Gaussian of standard
 * deviation 3 h_x, transported with v by the state equation
 * (Eq. (e:state-eq-elim), nt Heun steps) and thresholded at 0.5 (L_T); the
 * reference label map (device, n1*n2 floats, inside where > 0.5) is L_R.
 * measures (host, 4 doubles): Jaccard #(L_R and L_T) / #(L_R or L_T), Dice
 * 2 #(L_R and L_T) / (#L_R + #L_T), false positive error #(L_T minus L_R) /
 * #L_T, false negative error #(L_R minus L_T) / #L_R.  transported (device,
 * n1*n2 floats, nullable) receives the transported smoothed template labels
 * before the threshold.  Overwrites the state history, so the linearization
 * point is invalidated (REG_ERR_STATE for a matvec until the next
 * reg_gradient).  Synchronous. */
int reg_label_overlap(reg_ctx* ctx, const float* v, const float* labels_T, const float* labels_R,
                      float* transported, double* measures);

/* ---- learned warm start (the paper has no learned component) ---- */

/* An 8-layer 3x3 convolutional network with circular padding (channel
 * widths 2 -> 32 (x7) -> 2, ReLU between layers, layer l dilated by
 * min(d_l, H/8, W/32) with d = 1, 2, 4, 8, 8, 4, 2, 1) mapping an image pair
 * to a velocity.  Its output map is a Gaussian low-pass (symbol
 * exp(-sigma^2 |k|^2 / 2), sigma = 2 * 2 pi / max(H, W)) followed by the Leray
 * projection (Eq. (e:project-body-force) with w = 0), so that the prediction
 * satisfies div v = 0 and has no grid-scale noise.  BF16 activations and weights on the tensor cores
 * with FP32 accumulation; FP32 master weights; Adam (0.9, 0.999, 1e-8).
 * Parameters are a flat FP32 array: for each layer W (Cout, Cin, 3, 3), with
 * W[o, c, dy+1, dx+1] multiplying the input at (y+dy, x+dx), then b (Cout).
 * images: device, B x 2 x H x W floats (per sample m_T then m_R);
 * velocities / targets: device, B x 2 x H x W floats (component planes).
 * H, W powers of two in [32, 1024]; 1 <= B <= max_batch. */
typedef struct reg_net reg_net;
int reg_net_create(int H, int W, int max_batch, reg_net** out);
void reg_net_destroy(reg_net* net);
long long reg_net_num_params(reg_net* net);
int reg_net_set_stream(reg_net* net, void* stream);
/* Copy parameters in (device, num_params floats; resets the Adam state) / out. */
int reg_net_set_params(reg_net* net, const float* params);
int reg_net_get_params(reg_net* net, float* params);
/* Prediction v_out = s P G net(x), s the output scale (default 1). */
int reg_net_forward(reg_net* net, const float* images, int B, float* v_out);
/* Output scale s of reg_net_forward (0 < s <= 4; training and the loss use
 * s = 1): a warm start of s times the prediction; the warm-start pipeline
 * calibrates s on validation pairs. */
int reg_net_set_output_scale(reg_net* net, float scale);
/* loss = sum((P G net(x) - t)^2) / (2 M) (M = 2 B H W, host double) and, if grads
 * is not NULL, its gradient w.r.t. the flat parameters (device).  Synchronous. */
int reg_net_loss_grad(reg_net* net, const float* images, const float* targets, int B, double* loss, float* grads);
/* One Adam step with learning rate lr on that loss.  Synchronous (loss is read back). */
int reg_net_train_step(reg_net* net, const float* images, const float* targets, int B, float lr, double* loss);
/* Warm start for image pairs on the doubled grid (2H, 2W) from the network at H x W (the
 * resolution it was trained at): the images (device, B x 2 x 2H x 2W) are restricted by full
 * weighting (weights 1/4, 1/2, 1/4 per axis, periodic), the prediction P G net(x) on H x W is
 * prolonged bilinearly (periodic), and the fine grid's own output map P G (sigma = 2 h of that
 * grid) and the output scale s give v_out (device, B x 2 x 2H x 2W), divergence free on the fine
 * grid.  2H, 2W <= 1024.  The first call allocates a projection context and buffers. */
int reg_net_forward_fine(reg_net* net, const float* images, int B, float* v_out);
/* Convolution kernel of every forward and input-gradient convolution:
 * REG_CONV_TCGEN05 (default): 5th-generation tensor cores, FP32 accumulator in
 *   tensor memory; a persistent CTA per tile slot, MMAs issued by one thread.
 *   An MMA batch that does not complete within 1 s makes the kernel stop and
 *   set a flag; the next reg_net_forward / loss_grad / train_step call (and
 *   loss_grad / train_step themselves) then return REG_ERR_TIMEOUT.
 * REG_CONV_MMA_SYNC: warp-level mma.sync m16n8k16 tensor-core kernel.
 * Both accumulate the same products in FP32 (summation order differs). */
#define REG_CONV_TCGEN05 1
#define REG_CONV_MMA_SYNC 0
int reg_net_set_conv_kernel(reg_net* net, int kind);
/* Keep (on != 0) every layer's output gradient during reg_net_loss_grad /
 * train_step for reg_net_layer_tensor (allocates 8 x max_batch x H x W x 32
 * BF16 values on first use). */
int reg_net_set_record(reg_net* net, int on);
/* Copy one layer tensor of the last pass (device out, B x C x H x W floats,
 * B <= the batch of that pass):
 *   REG_NET_INPUT:       the BF16 input of layer l (C = Cin; l = 0: the packed images);
 *   REG_NET_OUTPUT:      its output after the ReLU (BF16, C = Cout), for the last layer
 *                        the FP32 raw network output (C = 2);
 *   REG_NET_OUTPUT_GRAD: the BF16 gradient w.r.t. the layer's pre-activation output as
 *                        the backward pass used it (C = Cout; reg_net_set_record), scaled by
 *                        M = 2 B H W (the 1 / M of the loss is applied to the parameter
 *                        gradients).  Asynchronous on the net's stream. */
#define REG_NET_INPUT 0
#define REG_NET_OUTPUT 1
#define REG_NET_OUTPUT_GRAD 2
int reg_net_layer_tensor(reg_net* net, int kind, int layer, int B, float* out);

/* ---- allocation-free entry point (the paper has no counterpart) ---- */

/* The spectral gradient of reg_spectral_grad for callers that cannot
 * allocate device memory: for example code whose device memory is owned by
 * another allocator that reserves it up front, or code that must not call a
 * synchronizing cudaMalloc / cudaFree.  No context is needed and nothing is
 * allocated: the scratch (three packed half spectra, 3 MiB) and the FFT
 * twiddle table are file-scope device arrays that every GPU which loads the
 * library holds until the process exits.
 *   grid      n1, n2 powers of two in [16, 1024] with n1 * n2 <= 512 * 512;
 *             larger grids are rejected with REG_ERR_ARG (the scratch limit).
 *   f         device, n1*n2 floats (input, row-major, 16-byte aligned);
 *   grad_f    device, 2*n1*n2 floats (output: d1 f then d2 f);
 *   stream    cudaStream_t the work is issued on (NULL = legacy default).
 * The first call on each device does that device's set-up (looks up the
 * arrays' device addresses, copies the twiddle table with cudaMemcpyToSymbol
 * and waits with cudaDeviceSynchronize until it has arrived, so that the
 * first call's kernels may run on any stream, non-blocking ones included),
 * so make the first call on a device before any stream capture begins.  All calls share the one scratch array and it keeps the
 * last call's contents; nothing in it has to start at zero because every
 * entry is written before it is read.  Calls that overlap on the GPU (other
 * streams, other host threads) race on the scratch: serialize them.
 * Asynchronous; returns REG_OK, REG_ERR_ARG or REG_ERR_CUDA. */
int reg_spectral_grad_static(reg_grid grid, const float* f, float* grad_f, void* stream);

/* ---- three-dimensional problems (the paper's Sec. 3 equations for d = 3) ---- */

/* One 3-D registration problem on the periodic box [0, 2 pi)^3 with the H1 seminorm
 * (A = -Lap), Heun's RK2 with nt steps and the trapezoidal rule in pseudo-time, as in 2-D.
 * n1, n2, n3: powers of two in [8, 256]; beta = beta_v > 0; gamma = beta_w: 0 (no
 * constraint), INFINITY (div v = 0), else the mass-source weight.  Real fields are
 * n1 x n2 x n3 floats, index (i1 n2 + i2) n3 + i3; vector fields (v, g, v~, H v~) are three
 * such fields back to back.  All pointers are device pointers owned by the caller.
 * Memory: about (3 nt + 30) n1 n2 n3 floats (the gradient history of the state is kept for
 * the matvecs).  Not thread-safe per context; calls run on the context's stream. */
typedef struct reg3_ctx reg3_ctx;
int reg3_create(int n1, int n2, int n3, int nt, double beta, double gamma, reg3_ctx** out);
void reg3_destroy(reg3_ctx* ctx);
int reg3_set_stream(reg3_ctx* ctx, void* stream);
/* Copies the template m_T and reference m_R in. */
int reg3_set_images(reg3_ctx* ctx, const float* mT, const float* mR);
/* Reduced gradient g = beta_v A v + K b (Eq. (e:control-eq-elim), b the body force of the
 * state and adjoint solves) and, if J is not NULL, the objective (host double; synchronous).
 * Fixes the linearization point of reg3_hessian_matvec.  REG_ERR_STATE before
 * reg3_set_images; REG_ERR_NAN if J is not finite. */
int reg3_gradient(reg3_ctx* ctx, const float* v, float* g, double* J);
/* Gauss-Newton matvec H v~ = beta_v A v~ + K b~ (Eqs. (e:inc-state-eq-elim),
 * (e:inc-adj-eq-elim), (e:inc-control-eq-elim)) at the v of the last reg3_gradient
 * (REG_ERR_STATE before one).  Asynchronous. */
int reg3_hessian_matvec(reg3_ctx* ctx, const float* vt, float* Hvt);
/* Algorithm 1 from v = 0 (v: device, overwritten with the result): inexact Gauss-Newton-Krylov
 * with Algorithm 2's PCG and the spectral preconditioner (beta_v A)^-1 (k = 0 symbol 1),
 * forcing eta_k = min(0.5, sqrt(||g_k|| / ||g_0||)), Armijo backtracking (c1 = 1e-4, halving,
 * 20 trials), stop at ||g|| <= tol ||g(0)||; at most maxit_newton Newton and maxit_pcg PCG
 * iterations.  stats (host, nullable, 7 doubles): Newton iterations, matvecs, line-search
 * trials, ||g|| / ||g(0)||, J, status, J(0) (filled on every return).  A trial whose J is
 * not finite (a step beyond the explicit scheme's stability) is rejected like one that fails
 * the decrease test.  Synchronous.  REG_ERR_LINESEARCH / REG_ERR_MAXIT when the search fails /
 * the cap is reached (v holds the last iterate). */
int reg3_solve(reg3_ctx* ctx, float* v, double tol, int maxit_newton, int maxit_pcg, double* stats);

/* ---- instrumentation ---- */

/* Per-kernel-class CUDA-event timing (off by default).  While enabled, every
 * kernel launch is bracketed by events on the context stream.
 * reg_kernel_time returns, for class `kclass`, the launch count, the summed
 * milliseconds and the summed algorithmic bytes (every input read once and
 * every output written once) since the last enable (host pointers, each
 * nullable).  Classes: 0 column FFT + multiplier kernels, 1 row FFT + RK2
 * stage kernels (advection / adjoint), 2 other row FFT kernels,
 * 3 pointwise / reduction kernels, 4 cluster-resident transport kernels (one
 * launch per transport solve, or per matvec for both of its solves). */
int reg_kernel_timing(reg_ctx* ctx, int enable);
int reg_kernel_time(reg_ctx* ctx, int kclass, long long* launches, double* ms, double* bytes);
/* Number of kernels this context has launched since creation. */
long long reg_launch_count(reg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* REG_H */
