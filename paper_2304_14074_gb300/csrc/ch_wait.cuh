// Bounded waits on shared-memory mbarriers. Every device-side wait of the library has an
// iteration limit: a wait that runs out returns false, the kernel records an error flag that
// the host turns into CH_ERR_TIMEOUT, and the kernel returns instead of hanging the device.
#pragma once
#include <cstdint>

namespace chwait {

// Polls of a wait before it gives up (each poll is one mbarrier.try_wait, which itself suspends
// for a hardware-chosen time): far beyond the microseconds the library's waits take.
constexpr unsigned kSpins = 1u << 22;
// Second, longer wait of a kernel that has given up once and must still let the asynchronous
// operations it issued finish before it frees their resources.
constexpr unsigned kDrainSpins = 1u << 26;

// Waits until the phase with parity `parity` of the mbarrier at shared address `mbar` has
// completed, polling at most `limit` times. Returns true when it completed.
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity, unsigned limit) {
  unsigned done = 0;
  for (unsigned spins = 0;; ++spins) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (spins >= limit) return false;
  }
}

}  // namespace chwait
