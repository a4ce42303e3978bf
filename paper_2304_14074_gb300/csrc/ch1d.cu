// One-dimensional Parareal: host dispatch of the kernels of ch1d_steps.cuh (the FP64 paths and
// the nonlinear scheme with FP32 inner solves; the linear schemes with FP32 inner solves are
// launched from ch1d_lin.cu).
#include <algorithm>

#include "ch1d_steps.cuh"

namespace chg {

// End of an iteration: count active problems, advance k, reset the work counter.
__global__ void k_tally(int B, Ctrl* ctrl, ProblemState ps, int* host_active) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int local = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) local += ps.active[b] ? 1 : 0;
  atomicAdd(&cnt, local);
  __syncthreads();
  if (threadIdx.x == 0) {
    ctrl->n_active = cnt;
    ctrl->k += 1;
    ctrl->next_unit = 0;
    if (host_active) *host_active = cnt;
  }
}

// ------------------------------------------------------------------------- host dispatch

// The fine propagator is the nonlinear scheme with FP32 inner solves: the mixed-form kernels of
// this file. With a linear fine scheme and FP32 inner solves, ch1d_lin.cu launches them.
static bool fast_fine(const Params1D& p) { return p.fine_scheme == SCHEME_NL && p.precision == 1; }
static bool mixed_linear(int scheme, int precision) { return scheme != SCHEME_NL && precision == 1; }

// Fine-sweep mapping of the mixed-form path with the autotuned alternative: alt = 1 halves the
// threads per CTA and doubles the block rows per thread (more CTAs resident per SM, longer
// per-thread Thomas chunks, a shorter PCR on the separators).
#define CH_DISPATCH_TP_FINE(n, alt, ...)                  \
  do {                                                    \
    if (!(alt) || (n) <= 128) {                           \
      CH_DISPATCH_TP_FAST(n, __VA_ARGS__);                \
    } else if ((n) <= 256) {                              \
      constexpr int T_ = 32, P_ = 4;                      \
      __VA_ARGS__;                                        \
    } else if ((n) <= 512) {                              \
      constexpr int T_ = 64, P_ = 4;                      \
      __VA_ARGS__;                                        \
    } else if ((n) <= 1024) {                             \
      constexpr int T_ = 128, P_ = 4;                     \
      __VA_ARGS__;                                        \
    } else {                                              \
      constexpr int T_ = 128, P_ = 8;                     \
      __VA_ARGS__;                                        \
    }                                                     \
  } while (0)

bool fine_sweep_has_alt(const Params1D& p) { return fast_fine(p) && p.n > 128; }

cudaError_t fine_sweep_max_grid(const Params1D& p, int* grid) {
  if (p.nn_sub > 0) return nn_max_grid(p, grid);
  if (mixed_linear(p.fine_scheme, p.precision)) {
    cudaError_t e = lin_fine_sweep_max_grid(p, grid);
    CH_DISPATCH_TP(p.n, {
      if (e == cudaSuccess) e = prep(k_coarse_sweep<T_, P_>, sizeof(Smem1D<T_>));
    });
    return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (fast_fine(p)) {
    CH_DISPATCH_TP_FINE(p.n, p.alt, {
      const size_t smem = sizeof(Smem1D<T_>);
      e = prep(k_fine_sweep<T_, P_, MODE_MIXED_NL>, smem);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fine_sweep<T_, P_, MODE_MIXED_NL>, T_, smem);
    });
  } else {
    CH_DISPATCH_TP(p.n, {
      const size_t smem = sizeof(Smem1D<T_>);
      e = prep(k_fine_sweep<T_, P_, MODE_FP64>, smem);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fine_sweep<T_, P_, MODE_FP64>, T_, smem);
    });
  }
  CH_DISPATCH_TP(p.n, {
    if (e == cudaSuccess) e = prep(k_coarse_sweep<T_, P_>, sizeof(Smem1D<T_>));
  });
  if (per_sm < 1) per_sm = 1;
  // No more CTAs than units: a small batch then has its units spread over distinct SMs instead of
  // going to whichever resident CTAs take them first (several per SM share its FP64 pipe).
  const long long units = (long long)p.B * p.N;
  *grid = (int)std::min<long long>((long long)sms * per_sm, std::max<long long>(units, 1));
  return e;
}

cudaError_t launch_fine_sweep(const Params1D& p, const double* U, double* F, Ctrl* ctrl, ProblemState ps,
                              int grid, cudaStream_t st) {
  if (p.nn_sub > 0) return launch_nn_fine_sweep(p, U, F, ctrl, ps, grid, st);
  if (mixed_linear(p.fine_scheme, p.precision)) return launch_lin_fine_sweep(p, U, F, ctrl, ps, grid, st);
  cudaError_t e = cudaSuccess;
  if (fast_fine(p)) {
    CH_DISPATCH_TP_FINE(p.n, p.alt, {
      const size_t smem = sizeof(Smem1D<T_>);
      e = prep(k_fine_sweep<T_, P_, MODE_MIXED_NL>, smem);
      if (e == cudaSuccess) k_fine_sweep<T_, P_, MODE_MIXED_NL><<<grid, T_, smem, st>>>(p, U, F, ctrl, ps);
    });
  } else {
    CH_DISPATCH_TP(p.n, {
      const size_t smem = sizeof(Smem1D<T_>);
      e = prep(k_fine_sweep<T_, P_, MODE_FP64>, smem);
      if (e == cudaSuccess) k_fine_sweep<T_, P_, MODE_FP64><<<grid, T_, smem, st>>>(p, U, F, ctrl, ps);
    });
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

cudaError_t launch_coarse_sweep(const Params1D& p, double* U, const double* F, double* Gold,
                                const double* Uref, Ctrl* ctrl, ProblemState ps, int init, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  CH_DISPATCH_TP(p.n, {
    const size_t smem = sizeof(Smem1D<T_>);
    e = prep(k_coarse_sweep<T_, P_>, smem);
    if (e == cudaSuccess) {
      k_coarse_sweep<T_, P_><<<p.B, T_, smem, st>>>(p, U, F, Gold, Uref, ctrl, ps, init);
      e = cudaGetLastError();
    }
  });
  return e;
}

cudaError_t launch_tally(const Params1D& p, Ctrl* ctrl, ProblemState ps, int* host_active, cudaStream_t st) {
  k_tally<<<1, 256, 0, st>>>(p.B, ctrl, ps, host_active);
  return cudaGetLastError();
}

cudaError_t launch_reference(const Params1D& p, double* Uref, Ctrl* ctrl, cudaStream_t st) {
  if (p.nn_sub > 0) return launch_nn_reference(p, Uref, ctrl, st);
  if (mixed_linear(p.fine_scheme, p.precision)) return launch_lin_reference(p, Uref, ctrl, st);
  cudaError_t e = cudaSuccess;
  if (fast_fine(p)) {
    CH_DISPATCH_TP_FINE(p.n, p.alt, {
      const size_t smem = sizeof(Smem1D<T_>);
      e = prep(k_reference<T_, P_, MODE_MIXED_NL>, smem);
      if (e == cudaSuccess) k_reference<T_, P_, MODE_MIXED_NL><<<p.B, T_, smem, st>>>(p, Uref, ctrl);
    });
  } else {
    CH_DISPATCH_TP(p.n, {
      const size_t smem = sizeof(Smem1D<T_>);
      e = prep(k_reference<T_, P_, MODE_FP64>, smem);
      if (e == cudaSuccess) k_reference<T_, P_, MODE_FP64><<<p.B, T_, smem, st>>>(p, Uref, ctrl);
    });
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

cudaError_t launch_propagate(const Params1D& p, int scheme, double dt, int nsteps, const double* uin,
                             double* uout, int* newton, Ctrl* ctrl, cudaStream_t st) {
  if (mixed_linear(scheme, p.precision)) return launch_lin_propagate(p, scheme, dt, nsteps, uin, uout, newton, ctrl, st);
  cudaError_t e = cudaSuccess;
  if (scheme == SCHEME_NL && p.precision == 1) {
    CH_DISPATCH_TP_FAST(p.n, {
      const size_t smem = sizeof(Smem1D<T_>);
      e = prep(k_propagate<T_, P_, MODE_MIXED_NL>, smem);
      if (e == cudaSuccess)
        k_propagate<T_, P_, MODE_MIXED_NL><<<p.B, T_, smem, st>>>(p, scheme, dt, nsteps, uin, uout, newton, ctrl);
    });
  } else {
    CH_DISPATCH_TP(p.n, {
      const size_t smem = sizeof(Smem1D<T_>);
      e = prep(k_propagate<T_, P_, MODE_FP64>, smem);
      if (e == cudaSuccess)
        k_propagate<T_, P_, MODE_FP64><<<p.B, T_, smem, st>>>(p, scheme, dt, nsteps, uin, uout, newton, ctrl);
    });
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace chg
