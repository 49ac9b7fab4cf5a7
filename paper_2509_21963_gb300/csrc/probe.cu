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

// Latency probes: one warp runs a chain of kLatN dependent operations of one
// kind between two clock64 reads; cycles per operation go to cyc[kind].
constexpr int kLatN = 256;
enum LatKind {
  kLatDfma = 0, kLatDfmaOneLane, kLatDadd, kLatShflDadd, kLatDdiv, kLatDsqrt, kLatDsetp,
  kLatFfma, kLatShflI64Max, kLatL2Load, kLatKinds
};

__global__ void lat_fp_kernel(int kind, double seed, const long long* chain, double* sink,
                              long long* cyc) {
  const int lane = threadIdx.x & 31;
  double x = seed + lane * 1e-3;
  const double a = 1.0000001, b = 1e-9;
  if (kind == kLatDfmaOneLane && lane != 0) return;
  const long long t0 = clock64();
  switch (kind) {
    case kLatDfma: case kLatDfmaOneLane:
      for (int i = 0; i < kLatN; ++i) x = fma(x, a, b);
      break;
    case kLatDadd:
      for (int i = 0; i < kLatN; ++i) x = x + b;
      break;
    case kLatShflDadd:
      for (int i = 0; i < kLatN; ++i) x = x + __shfl_xor_sync(0xffffffffu, x, 1 + (i & 15)) * 1e-300;
      break;
    case kLatDdiv:
      for (int i = 0; i < kLatN; ++i) x = a / x;
      break;
    case kLatDsqrt:
      for (int i = 0; i < kLatN; ++i) x = sqrt(x) + b;
      break;
    case kLatDsetp:
      for (int i = 0; i < kLatN; ++i) x = x > b ? x * a : x + b;
      break;
    case kLatFfma: {
      float f = (float)seed;
      for (int i = 0; i < kLatN; ++i) f = fmaf(f, 1.0000001f, 1e-9f);
      x = f;
      break;
    }
    case kLatShflI64Max: {
      long long k = __double_as_longlong(x);
      for (int i = 0; i < kLatN; ++i) {
        const long long o = __shfl_xor_sync(0xffffffffu, k, 1 + (i & 15));
        k = o > k ? o : k + 1;
      }
      x = (double)k;
      break;
    }
    case kLatL2Load: {   // dependent L2 loads (the chain is a permutation of 0..4095)
      long long idx = lane;
      for (int i = 0; i < kLatN; ++i) idx = __ldcg(chain + idx);
      x = (double)idx;
      break;
    }
  }
  const long long t1 = clock64();
  if (lane == 0) cyc[kind] = t1 - t0;
  if (x == 0.123) sink[0] = x;   // keeps the chain live; never true for these inputs
}

}  // namespace
}  // namespace cur

using namespace cur;

extern "C" int cur_probe_latency(cur_ctx* ctx, double* cycles, int n) {
  if (!ctx || !cycles || n < 1) return CUR_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) { cudaGetLastError(); return CUR_ECUDA; }
  constexpr int kChain = 4096;
  long long* dev = nullptr;   // chain[kChain], cyc[kLatKinds], sink
  int st = CUR_OK;
  if (cudaMalloc(&dev, sizeof(long long) * (kChain + kLatKinds + 1)) != cudaSuccess) {
    cudaGetLastError();
    return CUR_ECUDA;
  }
  long long host[kChain];
  for (int i = 0; i < kChain; ++i) host[i] = (long long)((i * 577 + 1031) % kChain);
  long long* chain = dev;
  long long* cyc = dev + kChain;
  double* sink = reinterpret_cast<double*>(dev + kChain + kLatKinds);
  if (cudaMemcpyAsync(chain, host, sizeof(host), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    st = CUR_ECUDA;
  for (int k = 0; k < kLatKinds && st == CUR_OK; ++k) {
    for (int rep = 0; rep < 2; ++rep)   // the second run is the measured one (warm)
      lat_fp_kernel<<<1, 32, 0, ctx->stream>>>(k, 1.5, chain, sink, cyc);
  }
  long long c[kLatKinds];
  if (st == CUR_OK &&
      (cudaGetLastError() != cudaSuccess ||
       cudaMemcpyAsync(c, cyc, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
       cudaStreamSynchronize(ctx->stream) != cudaSuccess)) {
    cudaGetLastError();
    st = CUR_ECUDA;
  }
  if (st == CUR_OK)
    for (int k = 0; k < n; ++k) cycles[k] = k < kLatKinds ? (double)c[k] / kLatN : 0.0;
  cudaFree(dev);
  return st;
}

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
