// Bounded grid barrier for persistent cooperative kernels.
#pragma once
#include <cuda_runtime.h>

namespace pgo {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s: only reached on a fault

// Wait limit of the grid barriers in ns (0: the 2 s default).  Each
// translation unit with grid barriers has its own copy, which a test hook
// shortens (set_barrier_limit_*); it is read only after 256 spins.
static __device__ unsigned long long g_barrier_limit_ns = 0ull;

// All blocks of the (co-resident) grid arrive; returns false if the wait
// exceeded the time limit or another block reported a timeout.  The counter
// is monotone within a launch (target advances by gridDim.x per barrier).
__device__ __forceinline__ bool grid_sync(unsigned* counter, int* abort_flag, unsigned& target) {
  __shared__ int ok;
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    ok = 1;
    red_release_add(counter, 1u);
    const unsigned long long t0 = globaltimer_ns();
    unsigned spins = 0;
    while (ld_acquire_u32(counter) < target) {
      if ((++spins & 255u) == 0u) {
        const unsigned long long lim = *(volatile unsigned long long*)&g_barrier_limit_ns;
        if (globaltimer_ns() - t0 > (lim ? lim : kBarrierTimeoutNs) || *(volatile int*)abort_flag) {
          atomicExch(abort_flag, 1);
          ok = 0;
          break;
        }
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

// Called by every block once after its last barrier: the last block to
// arrive resets the counter words so the next launch starts from zero.
__device__ __forceinline__ void grid_sync_release(unsigned* done_ticket, unsigned* counter, unsigned* abort_word) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(done_ticket, 1u);
    if (t == gridDim.x - 1) {
      *done_ticket = 0u;
      *counter = 0u;
      if (abort_word) *abort_word = 0u;
      __threadfence();
    }
  }
}

}  // namespace pgo
