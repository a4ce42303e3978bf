// C ABI of the learned coarse propagator G_theta (declared in include/ch_parareal.h).
#include <cuda_runtime.h>

#include <new>
#include <string>

#include "ch_parareal.h"
#include "ch_trace.cuh"
#include "ch_wait.cuh"
#include "gtheta.cuh"

static_assert(CH_GTHETA_PARAMS == chg3::kParams, "parameter count");

struct ch_gtheta {
  chg3::GTheta net;
  cudaStream_t st = nullptr;
  ch_status sticky = CH_OK;
  std::string msg;
};

namespace {

ch_status gfail(ch_gtheta* g, ch_status s, const std::string& m) {
  if (g && g->sticky == CH_OK) {
    g->sticky = s;
    g->msg = m;
  }
  return s;
}

ch_status gcuda(ch_gtheta* g, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return CH_OK;
  const std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return gfail(g, e == cudaErrorMemoryAllocation ? CH_ERR_OOM : CH_ERR_CUDA, m);
}

// A bounded tensor-core wait that gave up (tcgen05 path) makes the handle refuse further work.
ch_status check_waits(ch_gtheta* g) {
  if (g->net.wait_failures(g->st))
    return gfail(g, CH_ERR_TIMEOUT, "a bounded wait of the tensor-core convolution gave up");
  return CH_OK;
}

__global__ void k_wait_selftest(unsigned limit, int* out) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned mb = static_cast<unsigned>(__cvta_generic_to_shared(&bar));
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  __syncthreads();
  // expected arrivals: 1; no thread arrives, so phase 0 never completes
  const bool ok = chwait::mbar_wait(mb, 0u, limit);
  if (threadIdx.x == 0) *out = ok ? 1 : 2;
}

}  // namespace

extern "C" {

ch_status ch_gtheta_create(unsigned long long seed, void* cuda_stream, ch_gtheta** out) {
  if (!out) return CH_ERR_INVALID;
  *out = nullptr;
  ch_gtheta* g = new (std::nothrow) ch_gtheta();
  if (!g) return CH_ERR_OOM;
  (void)cudaGetLastError();
  g->st = static_cast<cudaStream_t>(cuda_stream);
  const cudaError_t e = g->net.init(seed, g->st);
  if (e != cudaSuccess) {
    g->net.release();
    delete g;
    return e == cudaErrorMemoryAllocation ? CH_ERR_OOM : CH_ERR_CUDA;
  }
  *out = g;
  return CH_OK;
}

void ch_gtheta_destroy(ch_gtheta* g) {
  if (!g) return;
  if (g->st) cudaStreamSynchronize(g->st);
  g->net.release();
  delete g;
}

const char* ch_gtheta_last_error(const ch_gtheta* g) { return g ? g->msg.c_str() : "NULL handle"; }

ch_status ch_gtheta_set_params(ch_gtheta* g, const float* params_host, size_t len) {
  if (!g) return CH_ERR_INVALID;
  if (!params_host || len != (size_t)CH_GTHETA_PARAMS) return gfail(g, CH_ERR_INVALID, "set_params: bad pointer or length");
  return gcuda(g, g->net.set_params(params_host, g->st), "set_params");
}

ch_status ch_gtheta_get_params(ch_gtheta* g, float* params_host, size_t len) {
  if (!g) return CH_ERR_INVALID;
  if (!params_host || len != (size_t)CH_GTHETA_PARAMS) return gfail(g, CH_ERR_INVALID, "get_params: bad pointer or length");
  return gcuda(g, g->net.get_params(params_host, g->st), "get_params");
}

ch_status ch_gtheta_forward(ch_gtheta* g, const double* in_dev, const double* base_dev, double* out_dev, int batch,
                            int n) {
  if (!g) return CH_ERR_INVALID;
  chtrace::Range range("G_theta forward");
  if (g->sticky != CH_OK) return g->sticky;
  if (!in_dev || !out_dev || batch < 1 || batch > 65535 || n < 1 || n > 65535)
    return gfail(g, CH_ERR_INVALID, "forward: bad arguments");
  return gcuda(g, g->net.forward64(in_dev, base_dev, out_dev, batch, n, g->st), "forward");
}

ch_status ch_gtheta_activations(ch_gtheta* g, const double* in_dev, int batch, int n, float* acts_dev, size_t len) {
  if (!g) return CH_ERR_INVALID;
  if (g->sticky != CH_OK) return g->sticky;
  if (!in_dev || !acts_dev || batch < 1 || batch > 65535 || n < 1 || n > 65535 ||
      len != (size_t)batch * n * n * (5 * 32 + 1))
    return gfail(g, CH_ERR_INVALID, "activations: bad arguments");
  ch_status s = gcuda(g, g->net.activations(in_dev, batch, n, acts_dev, g->st), "activations");
  if (s == CH_OK) s = gcuda(g, cudaStreamSynchronize(g->st), "activations: synchronize");
  if (s == CH_OK) s = check_waits(g);
  return s;
}

ch_status ch_gtheta_gradients(ch_gtheta* g, const float* in_dev, const float* target_dev, int batch, int S,
                              int margin, float* grad_host, size_t len, float* loss_host) {
  if (!g) return CH_ERR_INVALID;
  chtrace::Range range("G_theta gradients");
  if (g->sticky != CH_OK) return g->sticky;
  if (!in_dev || !target_dev || !grad_host || len != (size_t)CH_GTHETA_PARAMS || batch < 1 || S < 1 || S > 4096 ||
      margin < 0 || 2 * margin >= S)
    return gfail(g, CH_ERR_INVALID, "gradients: bad arguments");
  ch_status s = gcuda(g, g->net.grad_step(in_dev, target_dev, batch, S, margin, 0, g->st), "gradients");
  if (s != CH_OK) return s;
  s = gcuda(g, cudaMemcpyAsync(grad_host, g->net.grads(), len * sizeof(float), cudaMemcpyDeviceToHost, g->st),
            "gradients: copy");
  if (s != CH_OK) return s;
  float loss = 0.f;
  s = gcuda(g, g->net.read_losses(&loss, 1, g->st), "gradients: loss");
  if (s == CH_OK && loss_host) *loss_host = loss;
  if (s == CH_OK) s = check_waits(g);
  return s;
}

ch_status ch_gtheta_set_loss(ch_gtheta* g, int relative) {
  if (!g) return CH_ERR_INVALID;
  if (g->sticky != CH_OK) return g->sticky;
  if (relative != 0 && relative != 1) return gfail(g, CH_ERR_INVALID, "set_loss: relative must be 0 or 1");
  g->net.set_relative_loss(relative == 1);
  return CH_OK;
}

ch_status ch_gtheta_train(ch_gtheta* g, const double* states_dev, const double* base_dev, int ntraj, int nsnap,
                          int n, int stride, int steps, int batch, double lr, unsigned long long seed,
                          float* losses_host) {
  if (!g) return CH_ERR_INVALID;
  chtrace::Range range("G_theta training");
  if (g->sticky != CH_OK) return g->sticky;
  if (!states_dev || ntraj < 1 || stride < 1 || nsnap <= stride || n < 1 || n > 65535 || steps < 1 || batch < 1 ||
      batch > 65535 || !(lr > 0.0))
    return gfail(g, CH_ERR_INVALID, "train: bad arguments");
  ch_status s =
      gcuda(g, g->net.train(states_dev, base_dev, ntraj, nsnap, n, stride, steps, batch, lr, seed, g->st), "train");
  if (s == CH_OK && losses_host) s = gcuda(g, g->net.read_losses(losses_host, steps, g->st), "train: losses");
  if (s == CH_OK) s = check_waits(g);
  return s;
}

ch_status ch_wait_selftest(unsigned spin_limit, void* cuda_stream) {
  if (spin_limit < 1 || spin_limit > (1u << 26)) return CH_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  (void)cudaGetLastError();
  int* out = nullptr;
  if (cudaMalloc(&out, sizeof(int)) != cudaSuccess) return CH_ERR_OOM;
  int v = 0;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, st>>>(spin_limit, out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, out, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(out);
  if (e != cudaSuccess) return CH_ERR_CUDA;
  return v == 2 ? CH_ERR_TIMEOUT : (v == 1 ? CH_OK : CH_ERR_CUDA);
}

}  // extern "C"
