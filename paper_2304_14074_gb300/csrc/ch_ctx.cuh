// Identity of the current CUDA context, for caches of per-context state (kernel attributes set
// with cudaFuncSetAttribute, module symbol addresses). Such state belongs to a context, not to a
// device: cudaDeviceReset destroys the device's primary context and the next runtime call
// creates a new one, in which the attributes are unset and a module may load at another address.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

namespace chctx {

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

struct DriverFns {
  CtxGetCurrentFn get_current = nullptr;
  CtxGetIdFn get_id = nullptr;
};

// cuCtxGetCurrent / cuCtxGetId fetched through the runtime (no link against the driver library).
inline const DriverFns& driver_fns() {
  static DriverFns f;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f.get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f.get_id = reinterpret_cast<CtxGetIdFn>(p);
  });
  return f;
}

// Unique id of the current context (ids are never reused within a process), or 0 when there is
// no current context or the driver cannot tell.
inline unsigned long long current_id() {
  const DriverFns& f = driver_fns();
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!f.get_current || !f.get_id || f.get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (f.get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Cache key of per-context state: the context id, or (device + 1) << 48 when the id is unknown
// (then a reset device is not detected, as before contexts were tracked).
inline unsigned long long cache_key() {
  const unsigned long long id = current_id();
  if (id) return id;
  int dev = 0;
  cudaGetDevice(&dev);
  return (unsigned long long)(dev + 1) << 48;
}

}  // namespace chctx
