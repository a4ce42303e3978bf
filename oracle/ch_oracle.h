/*
 * CPU oracle for the Cahn-Hilliard Parareal methods (Garai & Mandal, arXiv 2304.14074).
 *
 * TEST INFRASTRUCTURE ONLY. Plain, sequential, FP64 reference written from the paper.
 * It shares no code with the GPU library; only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it. The product path never calls it.
 *
 * One dimension (Omega = (0,1)), n interior nodes x_j = j h, j = 1..n, h = 1/(n+1);
 * boundary values are zero (Section 2.1, the paper's j = 2..N_x-1 with N_x = n+2).
 * D_h = h^-2 tridiag(1,-2,1) (Eq. 3.2); D_h^2 = D_h D_h.
 *
 * Schemes (Section 2.1):
 *   ORC_LIN1  Eq. 2.4: (I - dt D_h diag(u^n)^2 + eps^2 dt D_h^2) u^{n+1} = (I - dt D_h) u^n
 *   ORC_NL    Eq. 2.3: u^{n+1} + eps^2 dt D_h^2 u^{n+1} - dt D_h (u^{n+1})^3 = (I - dt D_h) u^n,
 *             solved by the Newton iteration of Eq. 3.18 from Y_0 = u^n, stopping when
 *             ||Y_{m+1} - Y_m||_inf <= newton_tol, or (from the second increment on) when an
 *             increment below sqrt(newton_tol) fails to halve the previous one: the FP64
 *             rounding floor of the residual, about 1e-16 * 16 eps^2 dt / h^4 after J^-1,
 *             lies near 1e-12 on fine 1D grids (h = 1/1025).
 *   ORC_LIN2  Eq. 2.5 with the Laplacian on the implicit 2 dt term (as in Eq. 3.4a):
 *             (I - 2 dt D_h + eps^2 dt D_h^2) u^{n+1} = u^n + dt D_h (u^n)^3 - 3 dt D_h u^n
 * With `frozen` set, diag(u^2) is replaced by I (the analysis model of Section 3,
 * Eq. 3.3 / 3.4), which makes every scheme linear with constant coefficients.
 *
 * Parareal (Eq. 2.2): U_0^{k+1} = u^0,
 *   U_{n+1}^{k+1} = G(U_n^{k+1}) + F(U_n^k) - G(U_n^k), U^0 from the coarse propagator
 *   (Section 4), F = J fine steps of dt = T/(N J), G = coarse_steps steps of T/(N coarse_steps).
 *
 * Return codes: 0 ok, 1 invalid argument, 2 singular pivot, 3 Newton not converged.
 */
#ifndef CH_ORACLE_H
#define CH_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_LIN1 = 0, ORC_NL = 1, ORC_LIN2 = 2 };

typedef struct {
  int n;              /* interior nodes; h = 1/(n+1) */
  double eps;         /* interface parameter epsilon */
  double T;           /* final time */
  int N;              /* time slices */
  int J;              /* fine steps per slice */
  int coarse_steps;   /* coarse steps per slice */
  int fine_scheme;    /* ORC_* */
  int coarse_scheme;  /* ORC_* */
  double newton_tol;
  int newton_max;
  int frozen;         /* 1: diag(u^2) := I */
  double tol;         /* stop when max_n ||U_n^k - U_n^{k-1}||_inf < tol (tol <= 0: never) */
  int max_iters;      /* at most this many Parareal iterations (<= N) */
  int newton_form;    /* 0: Eq. 3.18 as printed, Y_{m+1} = J^{-1}(Yhat - 2 dt D_h Y_m^3);
                         1: the unsimplified Newton step Y_{m+1} = Y_m - J^{-1} H(Y_m), and the
                         linear steps (Eq. 2.4 / 2.5) taken from their residual the same way
                         from Y_0 = u^n. The two forms are the same steps; they differ only in
                         rounding, which measures how far two correct FP64 implementations can
                         drift apart (parity floor). */
} orc_params;

/* Manufactured forcing g(x,t) = sum_i a_i exp(b_i t) sin(m_i pi x), added as dt*g(t_{n+1}). */
typedef struct {
  int nmodes;
  const double* a;
  const double* b;
  const int* m;
} orc_forcing;

typedef struct {
  long long newton_total;  /* Newton iterations summed over steps */
  int newton_max_seen;     /* most Newton iterations in one step */
  long long steps;         /* time steps taken */
} orc_stats;

typedef struct {
  int iterations;          /* completed Parareal iterations k */
  int converged;           /* stop rule met */
  double inc[1024];        /* inc[k-1] = max_n ||U_n^k - U_n^{k-1}||_inf */
  double err_l2[1024];     /* err_l2[k] = max_n ||U_n^k - U^fine_n||_{L2_h}, k = 0..iterations */
  double err_max[1024];    /* same, max-abs */
  orc_stats st;
} orc_result;

/* out = D_h u */
int orc1d_dh_apply(int n, const double* u, double* out);

/* Gaussian elimination with partial pivoting on a banded matrix (kl sub-, ku super-diagonals).
 * `a` is n x (2 kl + ku + 1), row i holding columns i-kl .. i+kl+ku (fill space included);
 * overwritten by the factors. `b` is overwritten by the solution. */
int orc_band_solve(int n, int kl, int ku, double* a, double* b);

/* One time step of `scheme` with step dt; t_next = time at the end of the step (forcing only). */
int orc1d_step(const orc_params* p, int scheme, double dt, double t_next, const double* u,
               double* out, const orc_forcing* f, orc_stats* st);

/* nsteps steps from time t0. */
int orc1d_propagate(const orc_params* p, int scheme, double dt, int nsteps, double t0,
                    const double* u_in, double* u_out, const orc_forcing* f, orc_stats* st);

/* Sequential fine solution at the slice ends: Ufine[(N+1) n], Ufine_0 = u0. */
int orc1d_fine_solution(const orc_params* p, const double* u0, double* Ufine, orc_stats* st);

/* Parareal iterate after the stop rule: U[(N+1) n]. Ufine may be NULL (no error history). */
int orc1d_parareal(const orc_params* p, const double* u0, const double* Ufine, double* U,
                   orc_result* res);

/* Discrete Ginzburg-Landau energy (Eq. 1.2): h sum (u^2-1)^2/4 + eps^2/2 h u^T (-D_h) u. */
double orc1d_energy(int n, double eps, const double* u);

#ifdef __cplusplus
}
#endif
#endif
