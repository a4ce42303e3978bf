// One-dimensional Parareal kernels: shared declarations between the kernels and the host runtime.
#pragma once
#include <cuda_runtime.h>

namespace chg {

enum Scheme { SCHEME_LIN1 = 0, SCHEME_NL = 1, SCHEME_LIN2 = 2 };

// Device error bits (OR-ed into Ctrl::status).
enum : unsigned {
  ST_NEWTON = 1u,     // a Newton solve reached newton_max
  ST_NONFINITE = 2u,  // a solve produced a non-finite value
};

// Control block of one Parareal handle, in device memory.
struct Ctrl {
  int k;           // completed fine sweeps (Parareal iteration index)
  int next_unit;   // work counter of the persistent fine sweep
  int n_active;    // problems still iterating
  unsigned status; // error bits
};

// Per-problem device arrays.
struct ProblemState {
  int* active;                // 1 while the problem iterates
  int* iterations;            // completed iterations
  int* converged;             // stop rule met
  unsigned long long* newton_total;
  int* newton_max;
  double* inc;                // [B][maxit]
  double* err_l2;             // [B][maxit+1]
  double* err_max;            // [B][maxit+1]
};

struct Params1D {
  int n;             // interior nodes
  int B;             // problems
  int N;             // slices
  int J;             // fine steps per slice
  int coarse_steps;  // coarse steps per slice
  int fine_scheme;   // Scheme
  int coarse_scheme; // Scheme
  int precision;     // 0: FP64 solves; 1: FP32 inner solves of the fine steps, refined in FP64
  int frozen;
  int newton_max;
  int maxit;         // history stride
  double eps2;       // eps^2
  double h;          // 1/(n+1)
  double dt;         // fine step
  double dtc;        // coarse step
  double newton_tol;
  double tol;        // Parareal increment tolerance (<= 0: never)
  double err_tol;    // stop once the L2_h error against the reference is <= err_tol (<= 0: never)
  int alt;           // fine-sweep CTA mapping: 0 = default (T, P), 1 = (T/2, 2P) (autotuned)
  // Neumann-Neumann fine solver (Section 4.6; linear scheme Eq. 2.4 only): subdomains (0 = off),
  // relaxation, tolerance on the interface updates, iteration cap per step
  int nn_sub;
  double nn_theta;
  double nn_tol;
  int nn_max;
};

// Whether the fine sweep of p has an alternative CTA mapping (T/2 threads, 2P block rows each).
bool fine_sweep_has_alt(const Params1D& p);

// Launch helpers (implemented in ch1d.cu). All return cudaError_t of the launch.
cudaError_t launch_fine_sweep(const Params1D& p, const double* U, double* F, Ctrl* ctrl,
                              ProblemState ps, int grid, cudaStream_t st);
cudaError_t launch_coarse_sweep(const Params1D& p, double* U, const double* F, double* Gold,
                                const double* Uref, Ctrl* ctrl, ProblemState ps, int init,
                                cudaStream_t st);
cudaError_t launch_tally(const Params1D& p, Ctrl* ctrl, ProblemState ps, int* host_active,
                         cudaStream_t st);
cudaError_t launch_reference(const Params1D& p, double* Uref, Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_propagate(const Params1D& p, int scheme, double dt, int nsteps, const double* uin,
                             double* uout, int* newton, Ctrl* ctrl, cudaStream_t st);
// CTAs of the fine sweep that fit on the device at once (for the persistent grid).
cudaError_t fine_sweep_max_grid(const Params1D& p, int* grid);
// The linear schemes (Eq. 2.4 / 2.5) as fine steps with FP32 inner solves refined against FP64
// residuals (precision 1; implemented in ch1d_lin.cu): the same contracts as the launches above.
cudaError_t lin_fine_sweep_max_grid(const Params1D& p, int* grid);
cudaError_t launch_lin_fine_sweep(const Params1D& p, const double* U, double* F, Ctrl* ctrl, ProblemState ps,
                                  int grid, cudaStream_t st);
cudaError_t launch_lin_reference(const Params1D& p, double* Uref, Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_lin_propagate(const Params1D& p, int scheme, double dt, int nsteps, const double* uin,
                                 double* uout, int* newton, Ctrl* ctrl, cudaStream_t st);
// Neumann-Neumann fine solver (implemented in ch_nn.cu): whether p's sizes are supported, the
// persistent grid of its fine sweep, and the launches that replace the fine sweep and the
// sequential fine solution when p.nn_sub > 0.
bool nn_supported(const Params1D& p);
cudaError_t nn_max_grid(const Params1D& p, int* grid);
cudaError_t launch_nn_fine_sweep(const Params1D& p, const double* U, double* F, Ctrl* ctrl, ProblemState ps, int grid,
                                 cudaStream_t st);
cudaError_t launch_nn_reference(const Params1D& p, double* Uref, Ctrl* ctrl, cudaStream_t st);
// Largest n the kernels support.
constexpr int kMaxN1D = 4096;

}  // namespace chg
