// qpm_sync.cuh -- the grid-wide barrier of the persistent generation kernel, shared
// with the latency microbenchmark that measures it.
//
// A counter barrier: every CTA adds one arrival with a release reduction and waits,
// with acquire loads, for the count of its barrier; every wait is bounded by
// %globaltimer and records QPM_ERR_TIMEOUT in a shared error word when it runs out,
// after which every CTA returns (no trap).  Co-residency of all CTAs, which the waits
// need, comes from a cooperative launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "qpm.h"
#include "qpm_common.cuh"

namespace qpm {

struct Barrier {
  unsigned *count;   // arrivals, monotonically increasing (zeroed before the launch)
  int32_t *err;      // 0 ok, else a qpm_status
  unsigned long long timeout_ns;
};

__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// bounded wait (thread 0) until *p >= need; false when it ran out or another CTA failed.
// The error flag and the clock are looked at on the first failed poll and then on
// every 16th: each poll is an L2 round trip already, and a flag load after every poll
// (ordered behind the acquire) or after the success would add one more in series.
// A CTA that passes this wait just after another CTA gave up stops at the next one.
__device__ __forceinline__ bool wait_geq(const Barrier &b, const unsigned *p, unsigned need) {
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned spin = 0; (int)(ld_acquire(p) - need) < 0; ++spin) {
    if ((spin & 15u) == 0u) {
      if (*(volatile int32_t *)b.err != 0) return false;
      if (globaltimer_ns() - t0 > b.timeout_ns) {
        atomicCAS(b.err, 0, (int)QPM_ERR_TIMEOUT);
        return false;
      }
    }
  }
  return true;
}

// grid-wide barrier split into arrival and wait, so that independent work can
// run in between.  Every CTA adds one arrival (release) and then waits for the
// counter to reach (barriers passed) * gridDim.x (acquire).
__device__ __forceinline__ void grid_arrive(const Barrier &b, unsigned &target) {
  __syncthreads();
  target += gridDim.x;
  // the release orders this CTA's writes (made visible to thread 0 by the CTA
  // barrier above) before the arrival
  if (threadIdx.x == 0) red_release_add(b.count, 1u);
}

__device__ __forceinline__ bool grid_wait(const Barrier &b, unsigned target) {
  __shared__ int ok_sh;
  if (threadIdx.x == 0) ok_sh = wait_geq(b, b.count, target) ? 1 : 0;
  __syncthreads();
  return ok_sh != 0;
}

__device__ __forceinline__ bool grid_sync(const Barrier &b, unsigned &target) {
  grid_arrive(b, target);
  return grid_wait(b, target);
}

}  // namespace qpm
