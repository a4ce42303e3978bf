// Allocation-free Parareal solve: ch_parareal_solve_noalloc (declared in ch_parareal.h).
//
// Some callers cannot call cudaMalloc: an application whose device memory is owned by another
// allocator (a framework's caching pool that must not be bypassed, or a budget fixed at
// start-up), or a latency-critical loop where cudaMalloc/cudaFree would synchronise the device.
// This entry point therefore keeps all of its scratch (control block, per-problem histories,
// F(U_n^k) and G(U_n^k)) in one file-scope device array of fixed size; the caller provides the
// inputs and the output. Every GPU that loads the library holds the array until the process
// exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ch1d.cuh"
#include "ch2d.cuh"
#include "ch_config_check.h"
#include "ch_ctx.cuh"
#include "ch_parareal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CH_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchAddr {
  unsigned long long ctx_id = 0;  // context the address was looked up in (0: none)
  void* addr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];

// Device address of the scratch array in the current device's current context. Host code must
// not use the symbol itself (it is a host-side stand-in). The address is looked up once per
// device (cudaGetSymbolAddress, with that device current) and again whenever that device's
// context has changed since, e.g. after cudaDeviceReset, which may reload the module at another
// address. Where the driver cannot identify the context, every call looks it up.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long id = chctx::current_id();
  if (id) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch[dev].ctx_id == id && g_scratch[dev].addr) {
      *out = g_scratch[dev].addr;
      return cudaSuccess;
    }
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  if (id != 0) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_scratch[dev].ctx_id = id;
    g_scratch[dev].addr = p;
  }
  *out = p;
  return cudaSuccess;
}

__global__ void k_fill_ones(int* a, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = 1;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" ch_status ch_parareal_solve_noalloc(const ch_config* cfg, int batch, const double* u0_dev,
                                               double* U_dev, size_t len, int* iterations_host,
                                               void* cuda_stream) {
  if (!cfg || !u0_dev || !U_dev || batch < 1) return CH_ERR_INVALID;
  std::string why;
  if (!chcfg::valid_run(cfg, chg2::supported_n, why) || cfg->dim != 1) return CH_ERR_INVALID;
  const size_t B = batch, N = cfg->n_slices, n = cfg->n, maxit = cfg->max_iters;
  if (len != B * (N + 1) * n) return CH_ERR_INVALID;
  if (CH_NOALLOC_SCRATCH_NEEDED(B, N, n, maxit) > CH_NOALLOC_SCRATCH_BYTES) return CH_ERR_INVALID;

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return CH_ERR_CUDA;

  // Layout inside the scratch array (each part 256-byte aligned).
  char* q = static_cast<char*>(base);
  chg::Ctrl* ctrl = reinterpret_cast<chg::Ctrl*>(q);
  q += align256(sizeof(chg::Ctrl));
  const size_t ps_bytes = (B * maxit + 2 * B * (maxit + 1)) * sizeof(double) + B * sizeof(unsigned long long) +
                          4 * B * sizeof(int);
  chg::ProblemState ps{};
  ps.inc = reinterpret_cast<double*>(q);
  ps.err_l2 = ps.inc + B * maxit;
  ps.err_max = ps.err_l2 + B * (maxit + 1);
  ps.newton_total = reinterpret_cast<unsigned long long*>(ps.err_max + B * (maxit + 1));
  ps.active = reinterpret_cast<int*>(ps.newton_total + B);
  ps.iterations = ps.active + B;
  ps.converged = ps.iterations + B;
  ps.newton_max = ps.converged + B;
  char* ps_base = q;
  q += align256(ps_bytes);
  double* F = reinterpret_cast<double*>(q);
  q += align256(B * N * n * sizeof(double));
  double* Gold = reinterpret_cast<double*>(q);

  chg::Params1D p{};
  p.n = cfg->n;
  p.B = batch;
  p.N = cfg->n_slices;
  p.J = cfg->fine_steps;
  p.coarse_steps = cfg->coarse_steps;
  const int v = cfg->variant;
  p.fine_scheme = (v == CH_PA_I) ? chg::SCHEME_LIN1 : (v == CH_NPA_I || v == CH_NPA_II) ? chg::SCHEME_NL : chg::SCHEME_LIN2;
  p.coarse_scheme = (v == CH_PA_II) ? chg::SCHEME_LIN2 : (v == CH_NPA_II) ? chg::SCHEME_NL : chg::SCHEME_LIN1;
  p.precision = cfg->precision;
  p.frozen = cfg->frozen ? 1 : 0;
  p.newton_max = cfg->newton_max;
  p.maxit = cfg->max_iters;
  p.eps2 = cfg->eps * cfg->eps;
  p.h = 1.0 / (cfg->n + 1);
  const double dT = cfg->T / cfg->n_slices;
  p.dt = dT / cfg->fine_steps;
  p.dtc = dT / cfg->coarse_steps;
  p.newton_tol = cfg->newton_tol;
  p.tol = cfg->tol;
  p.err_tol = 0.0;  // no reference solution in this entry point

  int grid = 0;
  if (chg::fine_sweep_max_grid(p, &grid) != cudaSuccess) return CH_ERR_CUDA;
  // The array keeps the previous call's contents: clear what must start at zero.
  cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(chg::Ctrl), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ps_base, 0, ps_bytes, st);
  if (e == cudaSuccess) {
    k_fill_ones<<<(batch + 255) / 256, 256, 0, st>>>(ps.active, batch);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(U_dev, (N + 1) * n * sizeof(double), u0_dev, n * sizeof(double), n * sizeof(double), B,
                          cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = chg::launch_coarse_sweep(p, U_dev, F, Gold, nullptr, ctrl, ps, 1, st);
  int k = 0;
  for (; e == cudaSuccess && k < cfg->max_iters; ++k) {
    e = chg::launch_fine_sweep(p, U_dev, F, ctrl, ps, grid, st);
    if (e == cudaSuccess) e = chg::launch_coarse_sweep(p, U_dev, F, Gold, nullptr, ctrl, ps, 0, st);
    if (e == cudaSuccess) e = chg::launch_tally(p, ctrl, ps, nullptr, st);
    int active = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&active, &ctrl->n_active, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && active == 0) {
      ++k;
      break;
    }
  }
  chg::Ctrl c{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c, ctrl, sizeof(chg::Ctrl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return CH_ERR_CUDA;
  if (iterations_host) *iterations_host = k;
  if (c.status & chg::ST_NONFINITE) return CH_ERR_LINSOLVE;
  if (c.status & chg::ST_NEWTON) return CH_ERR_NEWTON;
  if (cfg->tol > 0.0 && c.n_active > 0) return CH_ERR_NOT_CONVERGED;
  return CH_OK;
}
