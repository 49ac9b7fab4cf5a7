// probe.cu -- measured FP64 FMA rate of the device, the denominator of the
// FP64-pipe roofline figures (the FP64 form of the sketch on the SIMT pipe,
// the batched engine).  The paper has no counterpart: this is measurement
// plumbing.  Every thread runs eight independent FMA chains (enough to cover
// the pipe latency) in a grid of several CTAs per SM; CUDA events time it.
#include "../../include/cur_steps.h"
#include "ctx.cuh"
#include "cur_internal.cuh"

namespace cur {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) fma_probe_kernel(double seed, double* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed + threadIdx.x + c;
  const double a = 1.0000000001, b = 1e-12;
#pragma unroll 4
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 0.1234) sink[0] = s;   // keeps the chains live; never true for these inputs
}

}  // namespace
}  // namespace cur

using namespace cur;

extern "C" int cur_probe_fp64_tflops(cur_ctx* ctx, double* tflops) {
  if (!ctx || !tflops) return CUR_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) { cudaGetLastError(); return CUR_ECUDA; }
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = CUR_OK;
  const int blocks = ctx->num_sms * 8;
  if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    st = CUR_ECUDA;
  } else {
    fma_probe_kernel<<<blocks, 256, 0, ctx->stream>>>(1.0, sink);   // warm-up
    cudaEventRecord(e0, ctx->stream);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) fma_probe_kernel<<<blocks, 256, 0, ctx->stream>>>(1.0 + r, sink);
    cudaEventRecord(e1, ctx->stream);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      st = CUR_ECUDA;
    } else {
      const double flops = 2.0 * kChains * (double)kIters * 256.0 * blocks * reps;
      *tflops = flops / (ms * 1e-3) / 1e12;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  return st;
}
