// gridbar.cuh -- bounded software grid barrier for cooperatively launched
// kernels (all CTAs co-resident by construction of cudaLaunchCooperativeKernel).
// A wait that outlives kBarrierBudget cycles records kDevTimeout in the status
// word and makes every later barrier return false, so a lost CTA surfaces as an
// error code instead of a hung GPU.
#pragma once

#include "cur_internal.cuh"

namespace cur {

__device__ __forceinline__ void dev_set_err(DevStatus* st, int code) {
  if (st) atomicCAS(&st->err, 0, code);
}

// Returns true when every CTA of the grid arrived; false on timeout or when a
// previous error was recorded.  Must be called by all threads of the CTA.
__device__ __forceinline__ bool grid_barrier(GridBar* bar, DevStatus* st) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = &bar->gen;
    unsigned g = *vgen;
    __threadfence();
    unsigned prev = atomicAdd(&bar->count, 1u);
    if (prev == gridDim.x - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > kBarrierBudget) { ok = 0; dev_set_err(st, kDevTimeout); break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (st && *((volatile int*)&st->err) != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace cur
