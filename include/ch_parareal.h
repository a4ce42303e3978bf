/*
 * ch_parareal.h - C ABI of the GB300 (sm_103a) Parareal library for the Cahn-Hilliard equation
 *
 *     u_t + eps^2 Lap^2 u = Lap f(u),  f(u) = u^3 - u,  on (0,1)^d, u = Lap u = 0 on the boundary
 *
 * following Garai & Mandal, "Linear and Nonlinear Parareal Methods for the Cahn-Hilliard
 * Equation" (arXiv 2304.14074): Eq. 1.1 (problem), Section 2.1 (the schemes Eq. 2.3-2.5 on
 * the discrete Laplacian D_h of Eq. 3.2), Eq. 2.2 (Parareal), Eq. 3.17/3.18 (Newton for the
 * nonlinear scheme), Section 4 (coarse initial guess, error in L^inf(0,T; L^2)).
 *
 * Conventions shared by every entry point
 *  - Every function returns ch_status and never aborts. A handle keeps the first error
 *    ("sticky") with a message readable through ch_parareal_last_error(); later calls that
 *    need the device return it. A Newton or linear-solve failure (CH_ERR_NEWTON,
 *    CH_ERR_LINSOLVE: a non-converging or non-finite propagation, e.g. from non-finite initial
 *    data) belongs to the data, not to the handle: a successful set_initial*, set_eps or
 *    set_fine_nn clears it. Every other error stays until the handle is destroyed.
 *  - Grid: n interior nodes per direction, h = 1/(n+1); boundary values are implicit zeros.
 *    A state is the interior values, FP64, row-major (y outer, x inner in 2D), n^d entries.
 *  - Slice layout: slices 0..N of one problem are contiguous, slice 0 = u^0; problems follow
 *    one another: element (b, s, j) of a [batch][N+1][n^d] array is at (b (N+1) + s) n^d + j.
 *  - "_host" pointers are host memory; "_dev" pointers are device memory of the current
 *    device. Caller-owned buffers are never retained past the call.
 *  - A handle owns its device memory and is bound to one CUDA stream (cudaStream_t passed
 *    as void*; NULL = the legacy default stream). Work is enqueued on that stream; calls
 *    that return data to the host synchronise it. A handle is not thread-safe.
 *  - dim = 1: n in 1..2048. dim = 2: n + 1 in {16, 32, 64, 128, 256, 512} (the sine transform
 *    of the 2D solver is a radix-2 FFT of length 2(n+1)); D_h = I (x) D_1 + D_1 (x) I (the
 *    natural extension of Eq. 3.2). In 2D every linear solve is FP32 preconditioned CG in sine
 *    space against FP64 residuals (`precision` is ignored) and Newton totals in ch_stats are
 *    for the whole batch.
 */
#ifndef CH_PARAREAL_H
#define CH_PARAREAL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CH_OK = 0,
  CH_ERR_INVALID = 1,        /* bad argument, size or configuration                       */
  CH_ERR_OOM = 2,            /* device or host allocation failed                          */
  CH_ERR_CUDA = 3,           /* a CUDA runtime call failed (message has the CUDA error)   */
  CH_ERR_NEWTON = 4,         /* a Newton solve hit newton_max without converging          */
  CH_ERR_LINSOLVE = 5,       /* a linear solve produced a non-finite value                */
  CH_ERR_NOT_CONVERGED = 6,  /* Parareal stop rule not met within max_iters               */
  CH_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up                        */
  CH_ERR_STATE = 8           /* call out of order (e.g. run before set_initial)           */
} ch_status;

/* The five Parareal variants of Section 2.1 (fine propagator F / coarse propagator G). */
typedef enum {
  CH_PA_I = 0,    /* F = G = linear scheme Eq. 2.4 (LIN1)                    */
  CH_PA_II = 1,   /* F = G = linear scheme Eq. 2.5 (LIN2)                    */
  CH_PA_III = 2,  /* F = LIN2, G = LIN1                                      */
  CH_NPA_I = 3,   /* F = nonlinear scheme Eq. 2.3 (Newton), G = LIN1         */
  CH_NPA_II = 4   /* F = G = nonlinear scheme Eq. 2.3                        */
} ch_variant;

/* Time-stepping schemes of Section 2.1, for ch_propagate. */
typedef enum {
  CH_SCHEME_LIN1 = 0,  /* Eq. 2.4: (I - dt D diag(u^n)^2 + eps^2 dt D^2) u^{n+1} = (I - dt D) u^n  */
  CH_SCHEME_NL = 1,    /* Eq. 2.3 solved by Newton (Eq. 3.17/3.18) from Y_0 = u^n               */
  CH_SCHEME_LIN2 = 2   /* Eq. 2.5 with D on the implicit 2 dt term:
                          (I - 2 dt D + eps^2 dt D^2) u^{n+1} = u^n + dt D (u^n)^3 - 3 dt D u^n  */
} ch_scheme;

typedef struct {
  int dim;             /* 1 or 2                                                            */
  int n;               /* interior nodes per direction, h = 1/(n+1)       (Section 2.1)     */
  double eps;          /* interface parameter epsilon                      (Eq. 1.1)         */
  double T;            /* final time                                        (Eq. 1.1)         */
  int n_slices;        /* N; Delta T = T/N                                  (Section 2)       */
  int fine_steps;      /* J; fine step dt = Delta T / J                     (Section 2)       */
  int coarse_steps;    /* coarse steps per slice (>= 1), each of Delta T / coarse_steps      */
  int variant;         /* ch_variant                                                         */
  double newton_tol;   /* Newton stop: ||Y_{m+1} - Y_m||_inf <= newton_tol, or the FP64
                          rounding floor (an increment below sqrt(newton_tol) that fails to
                          halve the previous one); in 2D also when the iteration contracts
                          (rho = |d_m| / |d_{m-1}| < 1/2) and its estimated remaining error
                          rho / (1 - rho) |d_m| is <= newton_tol                             */
  int newton_max;      /* Newton iteration cap per step                                      */
  double tol;          /* Parareal stop: max_n ||U_n^k - U_n^{k-1}||_inf < tol; <= 0: never   */
  int max_iters;       /* Parareal iteration cap, 1 <= max_iters <= N                         */
  int precision;       /* 0: all solves FP64; 1: Newton's inner linear solves in FP32 against
                          FP64 residuals (the converged step is the FP64 root)                */
  int frozen;          /* 1: diag(u^2) replaced by I (analysis model of Section 3); test mode */
  double err_tol;      /* also stop a problem once max_n ||U_n^k - U_n^fine||_{L2_h} <= err_tol
                          (the error measure of Section 4; needs ch_parareal_compute_reference);
                          <= 0: off                                                          */
  double lin_tol;      /* 2D inner linear solves (the Jacobian system of each Newton iteration
                          of Eq. 3.17, and the refinement sweeps of Eq. 2.4 / 2.5): CG stops once
                          the preconditioned residual norm has dropped by this factor; in (0, 1),
                          <= 0 selects 1e-3. Newton's FP64 residual is unchanged, so the step
                          converges to the same FP64 root; a looser value trades more Newton
                          iterations for fewer CG iterations. Ignored in 1D (direct solves).   */
  int lin_max;         /* 2D: CG iterations per inner solve at most; <= 0 selects 60.         */
} ch_config;

#define CH_MAX_ITERS 1024

typedef struct {
  int iterations;                 /* completed Parareal iterations k                          */
  int converged;                  /* stop rule met                                            */
  double inc[CH_MAX_ITERS];       /* inc[k-1] = max_n ||U_n^k - U_n^{k-1}||_inf               */
  double err_l2[CH_MAX_ITERS];    /* err_l2[k] = max_n ||U_n^k - U_n^fine||_{L2_h}, L2_h norm
                                     = sqrt(h^d sum e^2) (Section 4); valid after
                                     ch_parareal_compute_reference, else -1                   */
  double err_max[CH_MAX_ITERS];   /* same error, max-abs                                      */
  double t_iter_ms[CH_MAX_ITERS]; /* t_iter_ms[k] = device time from the start of run to the
                                     end of iteration k (k = 0: the coarse initial sweep)     */
  long long newton_total;         /* Newton iterations of the fine sweeps of run, summed over
                                     fine steps (2D: and over the batch's units)               */
  int newton_max;                 /* most Newton iterations taken by one fine step            */
  long long fine_point_steps;     /* fine steps x interior points executed by run             */
  /* Whole-handle figures of the last run (same for every problem): device time of the
     fine-sweep kernel and of the coarse-sweep kernel summed over iterations, measured with
     events recorded around them inside the iteration graph, and the number of launches of
     the library's kernels during run. */
  double fine_sweep_ms;
  double coarse_sweep_ms;
  int fine_sweep_launches;
  int kernel_launches;
  long long inner_iterations;     /* 2D: CG iterations of the fine sweeps, summed over the units
                                     (problem-slices) they ran on                             */
  int coarse_model;               /* 1: this problem's coarse sweeps started with the learned
                                     propagator G_theta (ch_parareal_set_coarse_model)          */
  int coarse_fallback_iter;       /* iteration after which G_theta was replaced by the plain
                                     coarse step, -1 if it never was                          */
} ch_stats;

typedef struct ch_parareal ch_parareal;

/* Create a handle for `batch` independent problems sharing `cfg`. Allocates device memory
 * for the slice states, F(U_n^k), G(U_n^k), the reference solution and the histories.
 * Errors: CH_ERR_INVALID (cfg out of range: dim not 1 or 2, n outside the grids above, N < 1 or
 * N >= CH_MAX_ITERS, J < 1, coarse_steps < 1, eps, T or newton_tol not finite and > 0, tol,
 * err_tol or lin_tol not finite, lin_tol >= 1, lin_max > 10000, batch < 1, max_iters outside
 * 1..N), CH_ERR_OOM, CH_ERR_CUDA. */
ch_status ch_parareal_create(const ch_config* cfg, int batch, void* cuda_stream, ch_parareal** out);

/* u^0 of one problem from host memory, len = n^d values. */
ch_status ch_parareal_set_initial(ch_parareal* h, int problem, const double* u0_host, size_t len);

/* u^0 of all problems from host memory, [batch][n^d], len = batch n^d values. */
ch_status ch_parareal_set_initial_batch(ch_parareal* h, const double* u0_host, size_t len);

/* u^0 of all problems from device memory, [batch][n^d], len = batch n^d values. */
ch_status ch_parareal_set_initial_device(ch_parareal* h, const double* u0_dev, size_t len);

/* The sequential fine solution U^fine_{n+1} = F(U^fine_n) (the serial method Parareal converges
 * to, Section 2), computed on the device and kept as the reference of err_l2 / err_max. */
ch_status ch_parareal_compute_reference(ch_parareal* h);

/* Parareal (Eq. 2.2): coarse initial sweep U^0 (Section 4), then iterations of
 * [fine sweep over all not-yet-exact slices of all active problems in one persistent launch;
 *  sequential coarse sweep with the correction U_{n+1}^{k+1} = F(U_n^k) + (G(U_n^{k+1}) - G(U_n^k))
 *  and the increment / error norms], each iteration replayed as one CUDA graph, until every
 * problem meets a stop rule (tol or err_tol) or max_iters. Returns CH_ERR_NOT_CONVERGED (not
 * sticky) when a stop rule is set and some problem did not meet it, CH_ERR_NEWTON when a Newton
 * solve failed. */
ch_status ch_parareal_run(ch_parareal* h);

/* Final iterate U^k of one problem: (N+1) n^d values to host memory. */
ch_status ch_parareal_get_slices(ch_parareal* h, int problem, double* out_host, size_t len);

/* Final iterates of all problems to host memory: batch (N+1) n^d values. */
ch_status ch_parareal_get_slices_batch(ch_parareal* h, double* out_host, size_t len);

/* Final iterates of all problems to device memory: batch (N+1) n^d values. */
ch_status ch_parareal_get_slices_device(ch_parareal* h, double* out_dev, size_t len);

/* Reference (sequential fine) slices of one problem: (N+1) n^d values to host memory. */
ch_status ch_parareal_get_reference(ch_parareal* h, int problem, double* out_host, size_t len);

/* Statistics of the last run for one problem. */
ch_status ch_parareal_get_stats(ch_parareal* h, int problem, ch_stats* out);

/* The execution of a 2D handle's steps, fixed by its first reference or run (chosen by timing,
 * or by the environment): 0 CUDA graphs, 1 persistent cooperative kernel, 2 host-driven
 * launches, 3 one thread-block cluster per unit; -1 before that choice. 1D handles: the fine
 * sweep's CTA mapping, 0 the default or 1 the alternative (T/2 threads, twice the rows each).
 * CH_ERR_INVALID for a NULL argument. */
ch_status ch_parareal_get_execution(ch_parareal* h, int* out);

/* Releases the handle and its device memory; NULL is accepted. */
void ch_parareal_destroy(ch_parareal* h);

/* Message of the handle's first error ("" when none). */
const char* ch_parareal_last_error(const ch_parareal* h);

/* Static name of a status code. */
const char* ch_status_string(ch_status s);

/* Orthonormal 2D sine transform (DST-I in x and y, its own inverse) of `batch` FP32 n x n
 * fields: out = S X S, S_jk = sqrt(2/(n+1)) sin(pi j k / (n+1)). The diagonalising transform of
 * D_h (eigenvalues below Eq. 3.2) used by the 2D solver. in_dev != out_dev, device arrays
 * [batch][n][n]; n + 1 a power of two in 16..512. FP32 arithmetic: about 1e-7 of the largest
 * output for n <= 127 (FFTs of the odd extension, length 2(n + 1)), about 1e-6 for n = 255 and
 * 511 (FFTs of length n + 1 whose odd coefficients are running sums of FFT outputs).
 * Synchronises the stream. */
ch_status ch_sine_transform_2d(const float* in_dev, float* out_dev, int batch, int n, void* cuda_stream);

/* Stateless propagation (the fine or coarse propagator as a batched kernel): applies `nsteps`
 * steps of `scheme` with step `dt` to each of `batch` problems sharing cfg->n, cfg->eps,
 * cfg->newton_tol, cfg->newton_max, cfg->precision and cfg->frozen (the other cfg fields are
 * ignored). u_in_dev / u_out_dev: [batch][n^d] device arrays (may alias). newton_dev: NULL or
 * a device int array [batch] receiving the Newton iterations summed over the steps.
 * Enqueued on `cuda_stream`; synchronises it before returning and reports CH_ERR_NEWTON /
 * CH_ERR_LINSOLVE from the device status. */
ch_status ch_propagate(const ch_config* cfg, int batch, int scheme, double dt, int nsteps,
                       const double* u_in_dev, double* u_out_dev, int* newton_dev,
                       void* cuda_stream);

/* A-priori Parareal error bound of Section 3 for cfg's variant, grid and time stepping:
 *     max_j ||E_j^k|| <= factor_k max_j ||E_j^0||,
 *     factor_k = a^k min{ ((1 - b^(N-1)) / (1 - b))^k, C(N-1, k) }   (0 for k >= N),
 * a = ||P_J - P_c||, b = ||P_c|| for PA-I / PA-II / PA-III (Theorems 3.7, 3.9, 3.11: P_c the
 * coarse propagator P_1, P_2, P_1 applied cfg->coarse_steps times, P_J the fine one P_1, P_2, P_2
 * with dT / J applied J times, all of the frozen model diag(u^2) = I); a = lte_const dT^2 and
 * b = ||P_1|| (NPA-I, Theorem 3.16) or ||P_3|| (NPA-II, Theorem 3.21), lte_const > 0 being the
 * constant C_1 / C_2 of the local truncation error, which the paper fits to measurements.
 * Norms are Euclidean 2-norms, formed over the eigenvalues of D_h (1D: n modes, 2D: n^2;
 * n in 1..2048 for both dims). Writes out_host[0] = a, out_host[1] = b, out_host[2 + k] =
 * factor_k for k = 0..kmax (len >= kmax + 3). Runs on `cuda_stream` and synchronises it.
 * Errors: CH_ERR_INVALID (cfg fields out of range, kmax < 0, len too small, lte_const <= 0
 * for the nonlinear variants), CH_ERR_OOM, CH_ERR_CUDA. */
ch_status ch_parareal_theory_bound(const ch_config* cfg, double lte_const, int kmax, double* out_host,
                                   size_t len, void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Learned coarse propagator G_theta(U) = U + R(U). The paper has none: it replaces the plain
 * coarse step G of Eq. 2.2 (one LIN1 step of Delta T), and Parareal still reaches the fine
 * solution (slice n is exact after n iterations for any G), so G_theta changes iteration
 * counts and wall time only.
 *
 * R: six 3x3 convolutions with zero padding (u = 0 outside the interior grid), channels
 * 1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU after the first five; hidden activations BF16, the
 * four 32 -> 32 layers on the tensor cores (BF16 x BF16 -> FP32), first and last layers FP32.
 * Parameters: CH_GTHETA_PARAMS FP32 values, for layer l = 0..5 the weights W_l[3][3][Cout][Cin]
 * (tap (dy, dx) applies to u[y + dy - 1][x + dx - 1]) followed by the biases b_l[Cout].
 * A ch_gtheta handle owns an FP32 master copy with Adam moments and its device work space; it
 * is bound to one stream and is not thread-safe. Errors as for ch_parareal.
 */
#define CH_GTHETA_PARAMS 37601

typedef struct ch_gtheta ch_gtheta;

/* New network with He-normal weights from `seed` (last layer scaled by 0.1), zero biases. */
ch_status ch_gtheta_create(unsigned long long seed, void* cuda_stream, ch_gtheta** out);
void ch_gtheta_destroy(ch_gtheta* g);
const char* ch_gtheta_last_error(const ch_gtheta* g);

/* Parameters from / to host memory, len = CH_GTHETA_PARAMS. set_params resets Adam. */
ch_status ch_gtheta_set_params(ch_gtheta* g, const float* params_host, size_t len);
ch_status ch_gtheta_get_params(ch_gtheta* g, float* params_host, size_t len);

/* out = base + R(U) for `batch` FP64 n x n fields U = in_dev (device, [batch][n][n]); base_dev
 * NULL means base = U (the residual form U + R(U)). out may alias in or base; n >= 1. Enqueued
 * on the handle's stream. */
ch_status ch_gtheta_forward(ch_gtheta* g, const double* in_dev, const double* base_dev, double* out_dev, int batch,
                            int n);

/* The forward pass of `batch` FP64 n x n fields (device, [batch][n][n]) keeping every layer's
 * output, for checking each layer on its own: acts_dev (device, FP32) receives the hidden
 * activations a1..a5 as stored (BF16 values), [5][batch][n][n][32], followed by R(U)
 * [batch][n][n]; len must be batch n^2 (5 * 32 + 1). Synchronises. */
ch_status ch_gtheta_activations(ch_gtheta* g, const double* in_dev, int batch, int n, float* acts_dev, size_t len);

/* The loss of ch_gtheta_gradients and ch_gtheta_train. relative = 0 (the default): the mean
 * over the batch and the window [margin, S - margin)^2 of (R(in) - target)^2. relative = 1: the
 * mean over the batch of each crop's sum over the window of (R(in) - target)^2 divided by
 * E = sum of target^2 there + 1e-12 (window pixels): every crop counts by its relative error,
 * as the coarse step is judged (slices late in time, whose changes are small, weigh as much as
 * early ones). CH_ERR_INVALID for other values. */
ch_status ch_gtheta_set_loss(ch_gtheta* g, int relative);

/* Loss and gradients for one minibatch: in_dev, target_dev FP32 [batch][S][S] (device); loss as
 * set by ch_gtheta_set_loss (by default the mean over the batch and the window
 * [margin, S - margin)^2 of (R(in) - target)^2).
 * grad_host: CH_GTHETA_PARAMS FP32 values in the parameter layout (len must match);
 * loss_host: NULL or one float. Synchronises. */
ch_status ch_gtheta_gradients(ch_gtheta* g, const float* in_dev, const float* target_dev, int batch, int S,
                              int margin, float* grad_host, size_t len, float* loss_host);

/* Trains R on pairs of snapshots of the fine solver: states_dev FP64 [ntraj][nsnap][n][n]
 * (device; e.g. the reference slices of a ch_parareal handle), pair (s, s + stride) for
 * s < nsnap - stride. Each of `steps` Adam steps (learning rate lr, betas 0.9 / 0.999,
 * eps 1e-8) draws `batch` crops (trajectory, snapshot, position from SplitMix64(seed)) of
 * min(76, n + 12) pixels and fits R(crop of U_s) to the crop of U_{s+stride} - base_s on the
 * crop's interior (6 pixels in from each side). base_dev: NULL (base_s = U_s, the residual
 * form) or FP64 [ntraj][nsnap][n][n] with base_s = G(U_s), the plain coarse step over the pair's
 * interval (the correction form). Adam's moments carry over between calls (a learning-rate
 * schedule is a sequence of calls). losses_host: NULL or `steps` floats receiving the
 * minibatch losses. Synchronises. */
ch_status ch_gtheta_train(ch_gtheta* g, const double* states_dev, const double* base_dev, int ntraj, int nsnap,
                          int n, int stride, int steps, int batch, double lr, unsigned long long seed,
                          float* losses_host);

/* Forms of the learned coarse step. */
typedef enum {
  CH_GTHETA_RESIDUAL = 0,   /* G_theta(U) = U + R(U)                                         */
  CH_GTHETA_CORRECTION = 1  /* G_theta(U) = G(U) + R(U), G the plain coarse step (R trained on
                               F(U) - G(U), base_dev of ch_gtheta_train)                      */
} ch_gtheta_form;

/* Uses G_theta with these parameters (CH_GTHETA_PARAMS values, host) in form `form`
 * (ch_gtheta_form) as the coarse propagator of the next runs of a 2D handle; params_host =
 * NULL (len 0) restores the plain coarse step. The plain step stays as judge: when a problem's
 * Parareal increment grows from one iteration to the next, its remaining iterations use the
 * plain step (G(U_n^k) recomputed with it). CH_ERR_INVALID for dim = 1. */
ch_status ch_parareal_set_coarse_model(ch_parareal* h, const float* params_host, size_t len, int form);

/* Per-problem interface parameter eps (host array of `batch` values > 0) for a 2D handle,
 * replacing cfg->eps; each fine and coarse step of problem b then uses eps[b] (Eq. 1.1). The
 * reference solution must be recomputed afterwards. CH_ERR_INVALID for dim = 1. */
ch_status ch_parareal_set_eps(ch_parareal* h, const double* eps_host, size_t len);

/* Reference slices of all problems to device memory: batch (N+1) n^d values. */
ch_status ch_parareal_get_reference_device(ch_parareal* h, double* out_dev, size_t len);

/* Neumann-Neumann fine solver (Section 4.6), 1D, for variants whose fine propagator is the linear
 * scheme Eq. 2.4 (PA-I). Each fine step solves the mixed system u - dt D v = u^n,
 * eps^2 D u - c^2 u + v = -u^n (c^2 = (u^n)^2; 1 when frozen; its elimination of v is Eq. 2.4) by
 * Neumann-Neumann iteration over n_sub equal subdomains (n + 1 a multiple of n_sub, at least two
 * nodes per subdomain, n_sub <= 32): Dirichlet solves on the subdomains, the residual of the global
 * rows at the interface nodes, Neumann solves with it (interface rows shared half and half between
 * the two subdomains), and the interface values updated by theta times the sum of the two Neumann
 * solutions, until both updates (u and v) have Euclidean norm over the interfaces <= tol, at most
 * max_iter iterations per step (reaching the cap sets CH_ERR_NEWTON on the next run or
 * compute_reference). The paper's setting: n_sub = 8, theta = 1/4, tol = 1e-10. Parareal then
 * converges to the sequential solution of this fine solver; compute_reference uses it too.
 * ch_stats.newton_total / newton_max count NN iterations (summed over steps / largest per step).
 * n_sub = 0 restores the monolithic fine solve. Call between runs; invalidates the reference.
 * Errors: CH_ERR_INVALID (dim != 1, another fine scheme, arguments out of range), CH_ERR_CUDA. */
ch_status ch_parareal_set_fine_nn(ch_parareal* h, int n_sub, double theta, double tol, int max_iter);

/* ---------------------------------------------------------------------------------------
 * Ensembles of 2D problems on uneven grids and with different eps. The paper has no
 * counterpart (it solves one problem at a time); this batches independent 2D problems of
 * Eq. 1.1 whose grids differ. Problems are grouped by grid size n; each group is one Parareal
 * handle (all its (problem, slice) units batched in every launch, per-problem eps as in
 * ch_parareal_set_eps) on a stream of its own, and the groups run concurrently, each driven
 * by a host thread of the call. cfg gives everything but n and eps (dim must be 2);
 * n_per_problem / eps_per_problem: `nprob` values each (host). Problem indices are the
 * ensemble's own; buffers as for the single-problem calls of the problem's handle.
 * ch_ensemble_run returns CH_ERR_NOT_CONVERGED when some group did not meet its stop rule. */
typedef struct ch_ensemble ch_ensemble;

ch_status ch_ensemble_create(const ch_config* cfg, int nprob, const int* n_per_problem, const double* eps_per_problem,
                             ch_ensemble** out);
ch_status ch_ensemble_set_initial(ch_ensemble* e, int problem, const double* u0_host, size_t len);
ch_status ch_ensemble_compute_reference(ch_ensemble* e);
ch_status ch_ensemble_run(ch_ensemble* e);
ch_status ch_ensemble_get_slices(ch_ensemble* e, int problem, double* out_host, size_t len);
ch_status ch_ensemble_get_reference(ch_ensemble* e, int problem, double* out_host, size_t len);
ch_status ch_ensemble_get_stats(ch_ensemble* e, int problem, ch_stats* out);
int ch_ensemble_groups(const ch_ensemble* e);
void ch_ensemble_destroy(ch_ensemble* e);
const char* ch_ensemble_last_error(const ch_ensemble* e);

/* ---------------------------------------------------------------------------------------
 * Allocation-free solve. The paper has no counterpart: this is a library-level service.
 *
 * For callers that cannot call cudaMalloc: applications whose device memory belongs to
 * another allocator (a framework's caching pool that must not be bypassed, or a memory budget
 * fixed at start-up), and latency-critical loops where cudaMalloc/cudaFree would synchronise
 * the device. It runs the same Parareal kernels as ch_parareal_run, but every scratch buffer
 * (control block, per-problem histories, F(U_n^k), G(U_n^k)) lives in one file-scope device
 * array of CH_NOALLOC_SCRATCH_BYTES (16 MiB) that each GPU loading the library holds until the
 * process exits. It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 *  cfg, batch   as for ch_parareal_create (dim = 1); err_tol is ignored (there is no
 *               reference solution here), tol and max_iters apply.
 *  u0_dev       device, [batch][n] initial states.
 *  U_dev        device, [batch][N+1][n] output: the final iterate (slice 0 = u^0);
 *               len must equal batch (N+1) n.
 *  iterations_host  NULL or host int receiving the completed Parareal iterations.
 *  cuda_stream  stream the work is enqueued on; the call synchronises it before returning.
 *
 * Returns CH_ERR_INVALID for a bad argument and when the problem needs more scratch than the
 * array holds, i.e. CH_NOALLOC_SCRATCH_NEEDED(batch, N, n, max_iters) > CH_NOALLOC_SCRATCH_BYTES;
 * otherwise the codes of ch_parareal_run (CH_ERR_NEWTON, CH_ERR_LINSOLVE, CH_ERR_NOT_CONVERGED,
 * CH_ERR_CUDA).
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture begins. Every call
 * shares the one array and overwrites it (the parts that must start at zero are cleared by
 * each call), so calls whose work overlaps on the GPU, from several threads or streams, race
 * and must be serialised by the caller.
 */
#define CH_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
#define CH_NOALLOC_ALIGN256(x) ((((size_t)(x)) + 255) & ~(size_t)255)
#define CH_NOALLOC_SCRATCH_NEEDED(B, N, n, maxit)                                                  \
  ((size_t)256 +                                                                                     \
   CH_NOALLOC_ALIGN256(((size_t)(B) * (maxit) + 2 * (size_t)(B) * ((maxit) + 1)) * 8 + (size_t)(B) * 8 + \
                       (size_t)(B) * 16) +                                                         \
   2 * CH_NOALLOC_ALIGN256((size_t)(B) * (N) * (n) * 8))

ch_status ch_parareal_solve_noalloc(const ch_config* cfg, int batch, const double* u0_dev, double* U_dev,
                                    size_t len, int* iterations_host, void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Diagnostics. The paper has no counterpart: these check the library itself.
 *
 * Failure path of the bounded device-side waits. Every wait of the library's kernels on an
 * asynchronous event (an mbarrier completed by the tensor cores, a grid barrier) polls a bounded
 * number of times; one that runs out records an error that the host reports as CH_ERR_TIMEOUT,
 * and the kernel returns, so a lost event never hangs the device. This call launches one block
 * that waits, with that same routine and at most spin_limit polls (1 .. 2^26), on an mbarrier
 * that expects one arrival and that no thread ever arrives on. Returns CH_ERR_TIMEOUT when the
 * wait gave up and the kernel returned (the expected outcome; the context stays usable),
 * CH_ERR_INVALID for a spin_limit out of range, CH_ERR_OOM / CH_ERR_CUDA otherwise.
 * Synchronises `cuda_stream`. */
ch_status ch_wait_selftest(unsigned spin_limit, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* CH_PARAREAL_H */
