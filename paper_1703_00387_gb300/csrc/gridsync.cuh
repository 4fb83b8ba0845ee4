// Grid-wide barrier with a bounded wait, for cooperative launches (all
// blocks co-resident): every block adds one to a counter in global memory and
// waits until it reaches `target`. Writes made by a block before the barrier
// are visible to every block after it. The wait gives up after limit_ns of
// wall time (%globaltimer): it then sets bit 0 of *err and returns false in
// every thread of the block, and the caller leaves the kernel.
#pragma once
#include <stdint.h>

namespace osmps {

constexpr uint64_t GRID_BARRIER_LIMIT_NS = 2000000000ull;

__device__ __forceinline__ uint64_t grid_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* err, int* s_ok,
                                             uint64_t limit_ns = GRID_BARRIER_LIMIT_NS) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    uint64_t t0 = 0;
    int ok = 1;
    for (unsigned it = 0;; ++it) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if ((int)(v - target) >= 0) break;
      if ((it & 63u) == 0) {
        const uint64_t now = grid_timer();
        if (it == 0) t0 = now;
        else if (now - t0 > limit_ns) {
          atomicOr(err, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

}  // namespace osmps
