// Grid-wide barriers of a cooperative launch (every block resident, which
// the launch guarantees), on two counter words in the caller's workspace:
// bar[0] counts arrivals, bar[1] blocks done.  Both are zero between
// launches: the last block out of the kernel resets them.  Every wait is
// bounded by a wall-clock limit; a wait that runs out records
// KF_DEVERR_TIMEOUT in the workspace's error word and reports failure, so the
// block can skip the work that needed the barrier.
#pragma once

#include <cstdint>

#include "kf_device.cuh"

namespace kf {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier number k (1, 2, ...) of the launch: every block adds one arrival,
// then waits until k * gridDim.x arrivals are in.  Call from every thread of
// every block (it contains __syncthreads); returns false in every thread of
// a block whose wait ran out.
__device__ __forceinline__ bool grid_barrier_bounded(unsigned* bar, unsigned k, uint64_t wait_ns, unsigned* err) {
  __shared__ int s_grid_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&bar[0], 1u);
    const unsigned target = k * gridDim.x;
    int ok = 1;
    if (ld_acquire_u32(&bar[0]) < target) {
      const uint64_t t0 = global_ns();
      while (ld_acquire_u32(&bar[0]) < target) {
        if (global_ns() - t0 > wait_ns) {
          ok = 0;
          atomicOr(err, KF_DEVERR_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
    s_grid_ok = ok;
  }
  __syncthreads();
  return s_grid_ok != 0;
}

// Leave the launch: the last block out sets both counters back to zero for
// the next launch on the same workspace.
__device__ __forceinline__ void grid_exit(unsigned* bar) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&bar[1], 1u) == gridDim.x - 1u) {
      bar[0] = 0u;
      bar[1] = 0u;
      __threadfence();
    }
  }
}

}  // namespace kf
