// Device-wide synchronisation shared by the set-up and time-loop kernels.
#pragma once

#include "internal.h"

namespace sbfwi {

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The wait
// is bounded: after `budget` clock cycles it records SBFWI_ETIMEOUT and gives up,
// so a broken launch returns an error instead of hanging the device.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, int* status, long long budget) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = gen;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > budget || *(volatile int*)status != 0) {
          atomicCAS(status, 0, SBFWI_ETIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace sbfwi
