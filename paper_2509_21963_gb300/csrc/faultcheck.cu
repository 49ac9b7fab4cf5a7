// faultcheck.cu -- kernels that drive the library's bounded device waits past
// their limit on purpose, so that tests can check the timeout path (the error
// status, the kernel's return, a usable context afterwards) without faulting
// or hanging a GPU.  The paper has no counterpart.
//   * grid barrier (gridbar.cuh): `nblocks` CTAs arrive at a barrier that
//     expects one CTA more than the launch has;
//   * mbarrier wait (tc_ptx.cuh): one CTA waits for a phase that needs two
//     arrivals and gets one.
// Each wait gives up after `budget` cycles, records kDevTimeout in the status
// word and returns.
#include "gridbar.cuh"
#include "tc_ptx.cuh"

namespace cur {
namespace {

__global__ void barrier_timeout_kernel(GridBar* bar, unsigned expect, long long budget,
                                       DevStatus* st) {
  if (threadIdx.x == 0) bar_arrive_wait(bar, expect, st, budget);
}

__global__ void mbarrier_timeout_kernel(long long budget, DevStatus* st) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    tc::mbar_arrive(&bar);                     // one of the two arrivals the phase needs
    if (!tc::mbar_wait(&bar, 0, budget)) dev_set_err(st, kDevTimeout);
  }
}

}  // namespace

cudaError_t launch_timeout_check(const LaunchEnv& env, int which, int nblocks, long long budget,
                                 GridBar* bar, DevStatus* st) {
  if (which == 0) {
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), env.stream);
    if (e != cudaSuccess) return e;
    barrier_timeout_kernel<<<nblocks, 32, 0, env.stream>>>(bar, (unsigned)nblocks + 1, budget, st);
  } else {
    mbarrier_timeout_kernel<<<1, 32, 0, env.stream>>>(budget, st);
  }
  return cudaGetLastError();
}

}  // namespace cur
