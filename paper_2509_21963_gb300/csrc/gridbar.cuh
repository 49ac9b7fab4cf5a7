// gridbar.cuh -- bounded software grid barrier for cooperatively launched
// kernels (all CTAs co-resident by construction of cudaLaunchCooperativeKernel).
// A wait that outlives kBarrierBudget cycles records kDevTimeout in the status
// word and returns false (callers then return), so a lost CTA surfaces as an
// error code instead of a hung GPU.
#pragma once

#include "cur_internal.cuh"

namespace cur {

__device__ __forceinline__ void dev_set_err(DevStatus* st, int code) {
  if (st) atomicCAS(&st->err, 0, code);
}

// Arrive at a barrier of n CTAs and wait for the other n - 1 (one thread per
// CTA).  The counter only grows: the arrival that reads `prev` belongs to the
// barrier that completes at count = (prev / n + 1) n.  Nothing is reset, so the
// last arrival's atomic is itself the release, and waiters see it on their next
// poll.  This needs the counter at a multiple of n on entry (zeroed before the
// launch, or left there by completed barriers of the same n CTAs); 64 bits do
// not wrap in practice.  A wait that outlives kBarrierBudget cycles records
// kDevTimeout; a wait that sees an error recorded by another CTA gives up too.
__device__ __forceinline__ bool bar_arrive_wait(GridBar* bar, unsigned n, DevStatus* st) {
  __threadfence();  // this CTA's writes before its arrival
  const unsigned long long prev = atomicAdd(&bar->count, 1ULL);
  const unsigned long long target = (prev / n + 1) * n;
  if (prev + 1 != target) {
    volatile unsigned long long* vc = &bar->count;
    const long long t0 = clock64();
    unsigned spins = 0;
    while (*vc < target) {
      if ((++spins & 255u) == 0) {
        if (clock64() - t0 > kBarrierBudget) { dev_set_err(st, kDevTimeout); return false; }
        if (st && *((volatile int*)&st->err) != 0) return false;
      }
    }
  }
  __threadfence();  // the other CTAs' writes before theirs
  return true;
}

// Grid-wide barrier of a cooperative launch.  Returns true when every CTA
// arrived; false on timeout or when another CTA recorded an error while this
// one waited.  Must be called by all threads of the CTA.
__device__ __forceinline__ bool grid_barrier(GridBar* bar, DevStatus* st) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) s_ok = bar_arrive_wait(bar, gridDim.x, st) ? 1 : 0;
  __syncthreads();
  return s_ok != 0;
}

}  // namespace cur
