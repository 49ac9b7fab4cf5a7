// gridbar.cuh -- bounded software grid barrier for cooperatively launched
// kernels (all CTAs co-resident by construction of cudaLaunchCooperativeKernel).
// A wait that outlives kBarrierBudget cycles records kDevTimeout in the status
// word and returns false (callers then return), so a lost CTA surfaces as an
// error code instead of a hung GPU.
#pragma once

#include "cur_internal.cuh"

#include <climits>

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
__device__ __forceinline__ bool bar_arrive_wait(GridBar* bar, unsigned n, DevStatus* st,
                                                long long budget = kBarrierBudget) {
  __threadfence();  // this CTA's writes before its arrival
  const unsigned long long prev = atomicAdd(&bar->count, 1ULL);
  const unsigned long long target = (prev / n + 1) * n;
  if (prev + 1 != target) {
    volatile unsigned long long* vc = &bar->count;
    const long long t0 = clock64();
    unsigned spins = 0;
    while (*vc < target) {
      if ((++spins & 255u) == 0) {
        if (clock64() - t0 > budget) { dev_set_err(st, kDevTimeout); return false; }
        if (st && *((volatile int*)&st->err) != 0) return false;
      }
    }
  }
  __threadfence();  // the other CTAs' writes before theirs
  return true;
}

// The two halves of bar_arrive_wait, for work that overlaps the wait: arrive
// (one thread per CTA, after a __syncthreads that orders the CTA's writes)
// returns the count at which this barrier completes; wait spins for it with
// the same budget and error rules.
__device__ __forceinline__ unsigned long long bar_arrive(GridBar* bar, unsigned n) {
  __threadfence();
  const unsigned long long prev = atomicAdd(&bar->count, 1ULL);
  return (prev / n + 1) * n;
}

__device__ __forceinline__ bool bar_wait(GridBar* bar, unsigned long long target, DevStatus* st,
                                         long long budget = kBarrierBudget) {
  volatile unsigned long long* vc = &bar->count;
  const long long t0 = clock64();
  unsigned spins = 0;
  while (*vc < target) {
    if ((++spins & 255u) == 0) {
      if (clock64() - t0 > budget) { dev_set_err(st, kDevTimeout); return false; }
      if (st && *((volatile int*)&st->err) != 0) return false;
    }
  }
  __threadfence();
  return true;
}

// Release-ordered arrival (fire and forget): this thread's earlier writes, and
// those of its CTA ordered before it by a __syncthreads, become visible to a
// thread that later acquires the counter.
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void red_max_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Spin (acquire loads) until *cnt >= target; the same budget and error rules
// as bar_wait.  Loads after it see every write released before the arrivals.
__device__ __forceinline__ bool wait_count_acquire(const unsigned long long* cnt,
                                                   unsigned long long target, DevStatus* st,
                                                   long long budget = kBarrierBudget) {
  const long long t0 = clock64();
  unsigned spins = 0;
  while (ld_acquire_u64(cnt) < target) {
    if ((++spins & 63u) == 0) {
      if (clock64() - t0 > budget) { dev_set_err(st, kDevTimeout); return false; }
      if (st && *((volatile int*)&st->err) != 0) return false;
    }
  }
  return true;
}

// The best (largest value, then smallest index) of G per-CTA records written
// before a barrier: slot g holds its value at slot[g * stride] and its index
// (bit pattern of a long long) at slot[g * stride + 1].  Called by a whole
// warp; each lane issues its loads (up to eight) together, so reading the
// records costs one L2 round trip instead of one per 32 records.  Every lane
// returns the winner and its record number; records with value -1 and index
// LLONG_MAX stand for "no candidate", and when no record beats them the result
// is {-1, LLONG_MAX, -1}.
struct SlotWin {
  double a;
  long long i;
  int g;
};
__device__ __forceinline__ SlotWin warp_slot_best(const double* slot, size_t stride, int G,
                                                  int lane) {
  constexpr int kR = 8;
  double av[kR];
  long long iv[kR];
#pragma unroll
  for (int k = 0; k < kR; ++k) {
    const int g = lane + 32 * k;
    av[k] = -1.0;
    iv[k] = LLONG_MAX;
    if (g < G) {
      const double* s = slot + (size_t)g * stride;
      av[k] = __ldcg(s);
      iv[k] = __double_as_longlong(__ldcg(s + 1));
    }
  }
  SlotWin c{-1.0, LLONG_MAX, -1};
#pragma unroll
  for (int k = 0; k < kR; ++k) {
    const int g = lane + 32 * k;
    if (g < G && (av[k] > c.a || (av[k] == c.a && iv[k] < c.i))) {
      c.a = av[k];
      c.i = iv[k];
      c.g = g;
    }
  }
  for (int g = lane + 32 * kR; g < G; g += 32) {  // grids above 256 CTAs
    const double* s = slot + (size_t)g * stride;
    const double a = __ldcg(s);
    const long long i = __double_as_longlong(__ldcg(s + 1));
    if (a > c.a || (a == c.a && i < c.i)) { c.a = a; c.i = i; c.g = g; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double oa = __shfl_xor_sync(0xffffffffu, c.a, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, c.i, o);
    const int og = __shfl_xor_sync(0xffffffffu, c.g, o);
    if (oa > c.a || (oa == c.a && oi < c.i)) { c.a = oa; c.i = oi; c.g = og; }
  }
  return c;
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
