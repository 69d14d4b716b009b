// Small inline-PTX helpers shared by the kernels (sm_103a).
#pragma once

#include <cstdint>

#include "kernels.h"

namespace mgiga {
namespace dev {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Bounded wait for the completion of an mbarrier phase: false after `limit`
// polls (the kernels use the default).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned phase, long long limit = kMbarPolls) {
  for (long long it = 0; it < limit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    if (ok) return true;
    __nanosleep(32);
  }
  return false;
}


}  // namespace dev
}  // namespace mgiga
