// A-priori Parareal error bounds of Section 3 (declared in include/ch_parareal.h).
//
// The convergence theorems bound the error of iterate k by a^k min{((1 - b^(N-1)) / (1 - b))^k,
// C(N-1, k)} times the error of the coarse initial guess, with a = ||P_J - P_c|| and b = ||P_c||
// for the linear variants (Theorems 3.7, 3.9, 3.11) and a = C dT^2, b = ||P_c|| for the
// nonlinear ones (Theorems 3.16, 3.21). Every P is a rational function of the symmetric D_h, so
// its 2-norm is the largest modulus over the eigenvalues lambda of D_h: the factor of
// (I - i s D_h + eps^2 s D_h^2)^{-1} (I - i s D_h) on a mode with y = -lambda is
// g_i(s, y) = (1 + i s y) / (1 + i s y + eps^2 s y^2) (Lemma 3.1); the fine propagator applies it
// J times with s = dT / J, the coarse one m = coarse_steps times with s = dT / m. The modes are
// y = mu_p (1D) and mu_p + mu_q (2D), mu_p = (4/h^2) sin^2(p pi / (2(n+1))) (below Eq. 3.2).
#include <cuda_runtime.h>

#include <cmath>

#include "ch_parareal.h"

namespace {

__device__ __forceinline__ double g_factor(int i, double s, double e2, double y) {
  const double num = 1.0 + i * s * y;
  return num / (num + e2 * s * y * y);
}

__device__ __forceinline__ double mode_mu(int p, int n, double ih2) {
  const double s = sin(p * M_PI / (2.0 * (n + 1)));
  return 4.0 * ih2 * s * s;
}

// Largest |fine - coarse| and |coarse| over the modes, as the bit patterns of non-negative
// doubles (whose integer order is their numeric order): out[0] = a, out[1] = b.
__global__ void k_theory_norms(int n, int dim, double e2, double dT, int J, int fi, int ci, int cs,
                               unsigned long long* out) {
  const double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h);
  const long long modes = (dim == 1) ? n : (long long)n * n;
  double a = 0.0, b = 0.0;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < modes;
       m += (long long)gridDim.x * blockDim.x) {
    const int p = (dim == 1) ? (int)m : (int)(m / n);
    const double y = mode_mu(p + 1, n, ih2) + ((dim == 1) ? 0.0 : mode_mu((int)(m % n) + 1, n, ih2));
    const double gc = pow(g_factor(ci, dT / cs, e2, y), (double)cs);
    b = fmax(b, fabs(gc));
    if (fi > 0) a = fmax(a, fabs(pow(g_factor(fi, dT / J, e2, y), (double)J) - gc));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(a));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(b));
  }
}

// res[0] = a (or a_fixed when > 0), res[1] = b, res[2 + k] = the bound's factor for k = 0..kmax
// (C(N-1, k) through lgamma; the factor is formed in logarithms, 0 where a = 0 or k >= N).
__global__ void k_theory_factors(const unsigned long long* nb, double a_fixed, int N, int kmax, double* res) {
  const double b = __longlong_as_double((long long)nb[1]);
  const double a = (a_fixed > 0.0) ? a_fixed : __longlong_as_double((long long)nb[0]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    res[0] = a;
    res[1] = b;
  }
  const double ls1 = log((1.0 - pow(b, (double)(N - 1))) / (1.0 - b));
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= kmax; k += gridDim.x * blockDim.x) {
    double f;
    if (k == 0) {
      f = 1.0;
    } else if (k > N - 1) {
      f = 0.0;
    } else {
      const double lc = lgamma((double)N) - lgamma(k + 1.0) - lgamma((double)(N - k));
      f = exp(k * log(a) + fmin(k * ls1, lc));
    }
    res[2 + k] = f;
  }
}

}  // namespace

extern "C" ch_status ch_parareal_theory_bound(const ch_config* cfg, double lte_const, int kmax, double* out_host,
                                              size_t len, void* cuda_stream) {
  if (!cfg || !out_host || kmax < 0 || kmax > (1 << 20) || len < (size_t)kmax + 3) return CH_ERR_INVALID;
  if ((cfg->dim != 1 && cfg->dim != 2) || cfg->n < 1 || cfg->n > 2048 || !(cfg->eps > 0.0) ||
      !std::isfinite(cfg->eps) || !(cfg->T > 0.0) || !std::isfinite(cfg->T) || cfg->n_slices < 1 ||
      cfg->fine_steps < 1 || cfg->coarse_steps < 1 || cfg->variant < CH_PA_I || cfg->variant > CH_NPA_II)
    return CH_ERR_INVALID;
  static const int kFine[5] = {1, 2, 2, 0, 0}, kCoarse[5] = {1, 2, 1, 1, 3};
  const int fi = kFine[cfg->variant], ci = kCoarse[cfg->variant];
  const double dT = cfg->T / cfg->n_slices;
  double a_fixed = 0.0;
  if (fi == 0) {
    if (!(lte_const > 0.0) || !std::isfinite(lte_const)) return CH_ERR_INVALID;
    a_fixed = lte_const * dT * dT;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  (void)cudaGetLastError();
  unsigned long long* nb = nullptr;
  double* res = nullptr;
  cudaError_t e = cudaMalloc(&nb, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&res, ((size_t)kmax + 3) * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(nb, 0, 2 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    const long long modes = (cfg->dim == 1) ? cfg->n : (long long)cfg->n * cfg->n;
    const int blocks = (int)((modes + 255) / 256 < 608 ? (modes + 255) / 256 : 608);
    k_theory_norms<<<blocks, 256, 0, st>>>(cfg->n, cfg->dim, cfg->eps * cfg->eps, dT, cfg->fine_steps, fi, ci,
                                          cfg->coarse_steps, nb);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_theory_factors<<<(kmax + 256) / 256, 256, 0, st>>>(nb, a_fixed, cfg->n_slices, kmax, res);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_host, res, ((size_t)kmax + 3) * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(nb);
  cudaFree(res);
  if (e == cudaSuccess) return CH_OK;
  return e == cudaErrorMemoryAllocation ? CH_ERR_OOM : CH_ERR_CUDA;
}
