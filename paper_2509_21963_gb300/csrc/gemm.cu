// gemm.cu -- FP64 general matrix product with fused sum of squares, used by
// the residual updates of IterativeCUR (arXiv 2509.21963, Algorithm 1's row
// and column residuals in the Lemma 1 form) and by the FP64 sketch Y = G A.
//
// All of these products are FP64; GB300 executes FP64 on a reduced-rate
// pipe, so a plain register-tiled SIMT kernel (64x64 tile, 4x4 per thread)
// already saturates it and sits far above its memory roofline.  The epilogue
// fuses beta*C and the per-tile sum of squares that the stopping test
// ||S^col||_F needs (Algorithm 1's rho_k); partial sums are reduced in a fixed
// order so results are deterministic.
#include "cur_internal.cuh"

namespace cur {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <bool B_F32>
__device__ __forceinline__ double loadB(const void* B, int64_t idx) {
  if (B_F32) return (double)static_cast<const float*>(B)[idx];
  return static_cast<const double*>(B)[idx];
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;  // valid in thread 0
}

template <bool B_F32>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs g) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  __shared__ double red[NT / 32];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)blockIdx.y * BM, col0 = (int64_t)blockIdx.x * BN;
  int64_t kbeg = 0, kend = g.K;
  if (g.ksplit > 1) {
    int64_t kc = (g.K + g.ksplit - 1) / g.ksplit;
    kc = (kc + BK - 1) / BK * BK;
    kbeg = (int64_t)blockIdx.z * kc;
    kend = min(g.K, kbeg + kc);
  }
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int s = 0; s < (BM * BK) / NT; ++s) {
      int e = tid + NT * s;
      int mm, kk;
      if (!g.transA) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      int64_t gr = row0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gr < g.M && gk < kend)
        v = g.transA ? g.A[gk * g.lda + gr] : g.A[gr * g.lda + gk];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int s = 0; s < (BK * BN) / NT; ++s) {
      int e = tid + NT * s;
      int nn, kk;
      if (!g.transB) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      int64_t gc = col0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gc < g.N && gk < kend)
        v = g.transB ? loadB<B_F32>(g.B, gc * g.ldb + gk) : loadB<B_F32>(g.B, gk * g.ldb + gc);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  if (g.ksplit > 1) {
    double* P = g.partial + (int64_t)blockIdx.z * g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int64_t r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
        if (r < g.M && c < g.N) P[r * g.N + c] = acc[i][j];
      }
    return;
  }
  double ss = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      if (r < g.M && c < g.N) {
        double d = g.alpha * acc[i][j];
        if (g.beta != 0.0) d = fma(g.beta, g.Cin[r * g.ldcin + c], d);
        g.D[r * g.ldd + c] = d;
        ss = fma(d, d, ss);
      }
    }
  if (g.sumsq_part) {
    double s = block_sum(ss, red);
    if (tid == 0) g.sumsq_part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// D = alpha * sum_z partial[z] + beta * Cin, over a flat index range.
__global__ void __launch_bounds__(NT) splitk_reduce_kernel(GemmArgs g, int64_t per_cta) {
  __shared__ double red[NT / 32];
  int64_t total = g.M * g.N;
  int64_t beg = (int64_t)blockIdx.x * per_cta, end = min(total, beg + per_cta);
  double ss = 0.0;
  for (int64_t e = beg + threadIdx.x; e < end; e += NT) {
    double s = 0.0;
    for (int z = 0; z < g.ksplit; ++z) s += g.partial[(int64_t)z * total + e];
    int64_t r = e / g.N, c = e - r * g.N;
    double d = g.alpha * s;
    if (g.beta != 0.0) d = fma(g.beta, g.Cin[r * g.ldcin + c], d);
    g.D[r * g.ldd + c] = d;
    ss = fma(d, d, ss);
  }
  if (g.sumsq_part) {
    double s = block_sum(ss, red);
    if (threadIdx.x == 0) g.sumsq_part[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(NT) sum_parts_kernel(const double* parts, int64_t n, double* out) {
  __shared__ double red[NT / 32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += NT) s += parts[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[0] = s;
}

// Skinny products of the residual updates: D (M x N) = alpha op(A) B + beta Cin
// with a small M (b or c rows), any K, a wide row-major B.  One thread owns 8
// rows of one output column; op(A) is staged through shared memory in K
// chunks of 32 and read as a broadcast, B is read coalesced along the column
// index.  The grid has ceil(N/256) x ceil(M/8) small CTAs (hundreds), which the
// block scheduler balances over the SMs without a half-empty last wave.
constexpr int kSkRows = 8, kSkK = 32, kSkThreads = 256;

template <bool TA>
__global__ void __launch_bounds__(kSkThreads) gemm_skinny_kernel(GemmArgs g) {
  __shared__ double As[kSkRows][kSkK];
  __shared__ double red[kSkThreads / 32];
  const int tid = threadIdx.x;
  const int64_t j = (int64_t)blockIdx.x * kSkThreads + tid;
  const int64_t r0 = (int64_t)blockIdx.y * kSkRows;
  double acc[kSkRows];
#pragma unroll
  for (int r = 0; r < kSkRows; ++r) acc[r] = 0.0;
  for (int64_t k0 = 0; k0 < g.K; k0 += kSkK) {
    {
      const int r = tid / kSkK, kk = tid % kSkK;   // 256 threads = 8 x 32 entries
      const int64_t gr = r0 + r, gk = k0 + kk;
      double v = 0.0;
      if (gr < g.M && gk < g.K) v = TA ? g.A[gk * g.lda + gr] : g.A[gr * g.lda + gk];
      As[r][kk] = v;
    }
    __syncthreads();
    if (j < g.N) {
      const int kend = (int)min((int64_t)kSkK, g.K - k0);
      const double* B = static_cast<const double*>(g.B) + k0 * g.ldb + j;
      for (int kk = 0; kk < kend; ++kk) {
        const double b = B[(int64_t)kk * g.ldb];
#pragma unroll
        for (int r = 0; r < kSkRows; ++r) acc[r] = fma(As[r][kk], b, acc[r]);
      }
    }
    __syncthreads();
  }
  double ss = 0.0;
  if (j < g.N) {
#pragma unroll
    for (int r = 0; r < kSkRows; ++r) {
      const int64_t gr = r0 + r;
      if (gr >= g.M) break;
      double d = g.alpha * acc[r];
      if (g.beta != 0.0) d = fma(g.beta, g.Cin[gr * g.ldcin + j], d);
      g.D[gr * g.ldd + j] = d;
      ss = fma(d, d, ss);
    }
  }
  if (g.sumsq_part) {
    double s = block_sum(ss, red);
    if (tid == 0) g.sumsq_part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

constexpr int64_t kReducePerCta = 8192;

}  // namespace

// The one-thread-per-column kernel for up to 256 output rows (b = 50 and
// b = 250 both measured faster than the 64 x 64 tiles on GB300).
static bool use_skinny(const GemmArgs& g) {
  return !g.transB && !g.b_is_f32 && g.ksplit <= 1 && g.M <= 256;
}

int64_t gemm_num_sumsq_parts(const GemmArgs& g) {
  if (use_skinny(g))
    return ((g.N + kSkThreads - 1) / kSkThreads) * ((g.M + kSkRows - 1) / kSkRows);
  if (g.ksplit > 1) return (g.M * g.N + kReducePerCta - 1) / kReducePerCta;
  return ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
}

cudaError_t launch_gemm(const LaunchEnv& env, const GemmArgs& g) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  int ks = g.ksplit < 1 ? 1 : g.ksplit;
  GemmArgs a = g;
  a.ksplit = ks;
  if (g.K <= 0) {  // D = beta * Cin (no product)
    a.alpha = 0.0;
  }
  if (use_skinny(a)) {
    dim3 grid((unsigned)((g.N + kSkThreads - 1) / kSkThreads), (unsigned)((g.M + kSkRows - 1) / kSkRows));
    if (a.transA) gemm_skinny_kernel<true><<<grid, kSkThreads, 0, env.stream>>>(a);
    else gemm_skinny_kernel<false><<<grid, kSkThreads, 0, env.stream>>>(a);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((g.N + BN - 1) / BN), (unsigned)((g.M + BM - 1) / BM), (unsigned)ks);
  if (a.b_is_f32) gemm_kernel<true><<<grid, NT, 0, env.stream>>>(a);
  else gemm_kernel<false><<<grid, NT, 0, env.stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || ks == 1) return e;
  int64_t nblk = (g.M * g.N + kReducePerCta - 1) / kReducePerCta;
  splitk_reduce_kernel<<<(unsigned)nblk, NT, 0, env.stream>>>(a, kReducePerCta);
  return cudaGetLastError();
}

cudaError_t launch_sum_parts(const LaunchEnv& env, const double* parts, int64_t n, double* out) {
  sum_parts_kernel<<<1, NT, 0, env.stream>>>(parts, n, out);
  return cudaGetLastError();
}

}  // namespace cur
