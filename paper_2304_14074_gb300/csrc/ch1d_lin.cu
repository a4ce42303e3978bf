// One-dimensional Parareal: the linear schemes Eq. 2.4 (LIN1) and Eq. 2.5 (LIN2) as fine steps
// with FP32 inner solves refined against the scheme's FP64 residual (precision 1).
//
// GB300 issues FP64 at 1/64 of a warp per clock per SM sub-partition, so a CTA of one warp that
// solves a 128-point system in FP64 spends most of a step waiting on the FP64 pipe (about 560 FP64
// warp instructions per step in the block partition solver). Refinement moves the solver's
// arithmetic to the FP32 pipe and leaves FP64 to the residual (about twelve operations per point
// and iteration) and the update; with the cubic predictor a step takes one or two iterations.
// The step agrees with the FP64 direct solve to the FP64 rounding level (step_mixed).
// These kernels compile in their own translation unit to keep the build's longest one short.
#include <algorithm>

#include "ch1d_steps.cuh"

namespace chg {

#define CH_DISPATCH_LIN_MODE(scheme, ...)                                  \
  do {                                                                     \
    if ((scheme) == SCHEME_LIN1) {                                         \
      constexpr int M_ = MODE_MIXED_LIN1;                                  \
      __VA_ARGS__;                                                         \
    } else {                                                               \
      constexpr int M_ = MODE_MIXED_LIN2;                                  \
      __VA_ARGS__;                                                         \
    }                                                                      \
  } while (0)

cudaError_t lin_fine_sweep_max_grid(const Params1D& p, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  CH_DISPATCH_LIN_MODE(p.fine_scheme, CH_DISPATCH_TP_FAST(p.n, {
    const size_t smem = sizeof(Smem1D<T_>);
    e = prep(k_fine_sweep<T_, P_, M_>, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fine_sweep<T_, P_, M_>, T_, smem);
  }));
  if (per_sm < 1) per_sm = 1;
  // No more CTAs than units: a small batch then has its units spread over distinct SMs instead of
  // going to whichever resident CTAs take them first (several per SM share its FP64 pipe).
  const long long units = (long long)p.B * p.N;
  *grid = (int)std::min<long long>((long long)sms * per_sm, std::max<long long>(units, 1));
  return e;
}

cudaError_t launch_lin_fine_sweep(const Params1D& p, const double* U, double* F, Ctrl* ctrl, ProblemState ps,
                                  int grid, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  CH_DISPATCH_LIN_MODE(p.fine_scheme, CH_DISPATCH_TP_FAST(p.n, {
    const size_t smem = sizeof(Smem1D<T_>);
    e = prep(k_fine_sweep<T_, P_, M_>, smem);
    if (e == cudaSuccess) k_fine_sweep<T_, P_, M_><<<grid, T_, smem, st>>>(p, U, F, ctrl, ps);
  }));
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

cudaError_t launch_lin_reference(const Params1D& p, double* Uref, Ctrl* ctrl, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  CH_DISPATCH_LIN_MODE(p.fine_scheme, CH_DISPATCH_TP_FAST(p.n, {
    const size_t smem = sizeof(Smem1D<T_>);
    e = prep(k_reference<T_, P_, M_>, smem);
    if (e == cudaSuccess) k_reference<T_, P_, M_><<<p.B, T_, smem, st>>>(p, Uref, ctrl);
  }));
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

cudaError_t launch_lin_propagate(const Params1D& p, int scheme, double dt, int nsteps, const double* uin,
                                 double* uout, int* newton, Ctrl* ctrl, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  CH_DISPATCH_LIN_MODE(scheme, CH_DISPATCH_TP_FAST(p.n, {
    const size_t smem = sizeof(Smem1D<T_>);
    e = prep(k_propagate<T_, P_, M_>, smem);
    if (e == cudaSuccess)
      k_propagate<T_, P_, M_><<<p.B, T_, smem, st>>>(p, scheme, dt, nsteps, uin, uout, newton, ctrl);
  }));
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace chg
