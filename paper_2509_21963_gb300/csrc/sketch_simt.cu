// sketch_simt.cu -- the initial sketch Y = G A of IterativeCUR (arXiv
// 2509.21963, Algorithm 1) in FP64 arithmetic on the SIMT FP64 pipe.
//
// GB300 runs FP64 at about 2 DFMA/clk/SM, so this pass is bound by that pipe,
// not by HBM: the design goal is to keep the pipe busy on every SM for the
// whole pass.  Two choices do that:
//   * rows of Y in groups of 4 per warp (c = 55 pads to 56, not to a 64-row
//     tile), 2 columns per lane, so no warp issues FMAs for padding rows
//     beyond the last group;
//   * the K range (rows of A) is split into many equal work units so that
//     every SM receives nearly the same number of units (no half-empty last
//     wave); partial sums go to a scratch buffer and are reduced in a fixed
//     order, which keeps the result deterministic.
// A and G tiles are staged through shared memory; A may be FP64 or FP32
// (converted exactly to FP64 on load).
#include "cur_internal.cuh"

namespace cur {
namespace {

constexpr int kRowsPerWarp = 4;
constexpr int kMaxWarps = 16;              // 64 rows of Y per CTA
constexpr int kCols = 64;                  // columns of Y per CTA (2 per lane)
constexpr int kKT = 32;                    // rows of A per shared-memory stage

// Two consecutive elements of A (the second only if `two`), 8/16-byte vector
// load when `vec` says the address is aligned for it.
template <bool F32>
__device__ __forceinline__ double2 load_a2(const void* A, int64_t off, bool vec, bool two) {
  if (F32) {
    const float* p = static_cast<const float*>(A) + off;
    if (vec && two) {
      float2 v = *reinterpret_cast<const float2*>(p);
      return make_double2(v.x, v.y);
    }
    return make_double2(p[0], two ? (double)p[1] : 0.0);
  }
  const double* p = static_cast<const double*>(A) + off;
  if (vec && two) return *reinterpret_cast<const double2*>(p);
  return make_double2(p[0], two ? p[1] : 0.0);
}

struct SketchArgs {
  const double* G; int64_t ldg; int c;
  const void* A; int64_t lda; int64_t m, n;
  int64_t kunit;      // rows of A per work unit (multiple of kKT)
  int ks;             // number of K units
  double* out;        // ks == 1: Y (c x n); else partial [ks][c][n]
  double* sumsq_part; // ks == 1: per-CTA sums of squares (optional)
  bool vec_ok;        // A rows 16-byte aligned for the 2-wide loads
};

template <bool F32>
__global__ void __launch_bounds__(kMaxWarps * 32) sketch_kernel(SketchArgs g) {
  __shared__ __align__(16) double As[kKT][kCols];
  __shared__ double Gs[kMaxWarps * kRowsPerWarp][kKT + 1];
  __shared__ double red[kMaxWarps];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nthreads = blockDim.x;
  const int row0 = blockIdx.y * kMaxWarps * kRowsPerWarp;
  const int rows_here = min(kMaxWarps * kRowsPerWarp, g.c - row0);
  const int64_t col0 = (int64_t)blockIdx.x * kCols;
  const int z = blockIdx.z;
  const int64_t kbeg = (int64_t)z * g.kunit;
  const int64_t kend = min(g.m, kbeg + g.kunit);

  double acc[kRowsPerWarp][2];
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) acc[r][0] = acc[r][1] = 0.0;

  for (int64_t k0 = kbeg; k0 < kend; k0 += kKT) {
    // stage A(k0:k0+kKT, col0:col0+64): each thread moves 2-wide pieces
    for (int e = tid; e < kKT * (kCols / 2); e += nthreads) {
      int kk = e / (kCols / 2), cc = 2 * (e % (kCols / 2));
      int64_t gk = k0 + kk, gc = col0 + cc;
      double2 v = make_double2(0.0, 0.0);
      if (gk < kend && gc < g.n) v = load_a2<F32>(g.A, gk * g.lda + gc, g.vec_ok, gc + 1 < g.n);
      *reinterpret_cast<double2*>(&As[kk][cc]) = v;
    }
    // stage G(row0 : row0+rows_here, k0:k0+kKT)
    for (int e = tid; e < rows_here * kKT; e += nthreads) {
      int rr = e / kKT, kk = e % kKT;
      int64_t gk = k0 + kk;
      Gs[rr][kk] = gk < kend ? g.G[(int64_t)(row0 + rr) * g.ldg + gk] : 0.0;
    }
    __syncthreads();
    const int rbase = wid * kRowsPerWarp;
    if (row0 + rbase < g.c) {  // warps wholly past the last row only stage tiles
#pragma unroll 8
    for (int kk = 0; kk < kKT; ++kk) {
      double2 a = *reinterpret_cast<const double2*>(&As[kk][2 * lane]);
#pragma unroll
      for (int r = 0; r < kRowsPerWarp; ++r) {
        double gv = Gs[rbase + r][kk];
        acc[r][0] = fma(gv, a.x, acc[r][0]);
        acc[r][1] = fma(gv, a.y, acc[r][1]);
      }
    }
    }
    __syncthreads();
  }

  double ss = 0.0;
  const int64_t gc = col0 + 2 * lane;
#pragma unroll
  for (int r = 0; r < kRowsPerWarp; ++r) {
    int row = row0 + wid * kRowsPerWarp + r;
    if (row >= g.c) continue;
    double* o = g.out + ((int64_t)z * g.c + row) * g.n;
    if (gc < g.n) { o[gc] = acc[r][0]; ss = fma(acc[r][0], acc[r][0], ss); }
    if (gc + 1 < g.n) { o[gc + 1] = acc[r][1]; ss = fma(acc[r][1], acc[r][1], ss); }
  }
  if (g.ks == 1 && g.sumsq_part) {
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
    if (lane == 0) red[wid] = ss;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < (nthreads >> 5); ++w) s += red[w];
      g.sumsq_part[((int64_t)blockIdx.y * gridDim.x) + blockIdx.x] = s;
    }
  }
}

// Y = sum_z partial[z] in a fixed order, plus per-CTA sums of squares.
__global__ void __launch_bounds__(256) sketch_reduce_kernel(const double* partial, int ks,
                                                            int64_t total, double* Y,
                                                            double* sumsq_part, int64_t per_cta) {
  __shared__ double red[8];
  int64_t beg = (int64_t)blockIdx.x * per_cta, end = min(total, beg + per_cta);
  double ss = 0.0;
  for (int64_t e = beg + threadIdx.x; e < end; e += 256) {
    double s = 0.0;
    for (int z = 0; z < ks; ++z) s += partial[(int64_t)z * total + e];
    Y[e] = s;
    ss = fma(s, s, ss);
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    sumsq_part[blockIdx.x] = s;
  }
}

constexpr int64_t kReducePerCta = 16384;

}  // namespace

SketchPlan plan_sketch_simt(const LaunchEnv& env, int64_t c, int64_t m, int64_t n) {
  SketchPlan p;
  int64_t tiles = ((n + kCols - 1) / kCols) * ((c + kMaxWarps * kRowsPerWarp - 1) / (kMaxWarps * kRowsPerWarp));
  int64_t kt_total = (m + kKT - 1) / kKT;
  // about 24 work units per SM; each unit at least 4 stages of A
  int64_t target = 24LL * env.num_sms;
  int64_t ks = (target + tiles - 1) / tiles;
  int64_t ks_max = (kt_total + 3) / 4;
  if (ks > ks_max) ks = ks_max;
  if (ks < 1) ks = 1;
  int64_t kt_per = (kt_total + ks - 1) / ks;
  p.kunit = kt_per * kKT;
  p.ks = (int)((m + p.kunit - 1) / p.kunit);
  p.partial_doubles = p.ks > 1 ? (size_t)p.ks * c * n : 0;
  p.sumsq_parts = p.ks > 1 ? (c * n + kReducePerCta - 1) / kReducePerCta : tiles;
  return p;
}

cudaError_t launch_sketch_simt(const LaunchEnv& env, const SketchPlan& p, const double* G,
                               int64_t ldg, int64_t c, const void* A, bool a_f32, int64_t lda,
                               int64_t m, int64_t n, double* Y, double* partial,
                               double* sumsq_part) {
  SketchArgs g;
  g.G = G; g.ldg = ldg; g.c = (int)c; g.A = A; g.lda = lda; g.m = m; g.n = n;
  g.kunit = p.kunit; g.ks = p.ks;
  g.out = p.ks > 1 ? partial : Y;
  g.sumsq_part = sumsq_part;
  g.vec_ok = (lda % 2 == 0) && ((reinterpret_cast<uintptr_t>(A) & (a_f32 ? 7 : 15)) == 0);
  const int row_blocks = (int)((c + kMaxWarps * kRowsPerWarp - 1) / (kMaxWarps * kRowsPerWarp));
  const int rows_first = (int)(c < kMaxWarps * kRowsPerWarp ? c : kMaxWarps * kRowsPerWarp);
  const int warps = (rows_first + kRowsPerWarp - 1) / kRowsPerWarp;
  dim3 grid((unsigned)((n + kCols - 1) / kCols), (unsigned)row_blocks, (unsigned)p.ks);
  // every row block launches the same warp count; the last one masks rows >= c
  if (a_f32) sketch_kernel<true><<<grid, warps * 32, 0, env.stream>>>(g);
  else sketch_kernel<false><<<grid, warps * 32, 0, env.stream>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || p.ks == 1) return e;
  int64_t total = c * n;
  int64_t nblk = (total + kReducePerCta - 1) / kReducePerCta;
  sketch_reduce_kernel<<<(unsigned)nblk, 256, 0, env.stream>>>(partial, p.ks, total, Y, sumsq_part,
                                                                kReducePerCta);
  return cudaGetLastError();
}

// Row-block form for copies that overlap the sketch: the ks slices of
// G(:, rows) A(rows, :) go to `slices` (ks * c * n doubles, no reduction);
// launch_sketch_reduce sums all slices of all row blocks in a fixed order.
cudaError_t launch_sketch_simt_slices(const LaunchEnv& env, const SketchPlan& p, const double* G,
                                      int64_t ldg, int64_t c, const void* A, bool a_f32,
                                      int64_t lda, int64_t m, int64_t n, double* slices) {
  SketchArgs g;
  g.G = G; g.ldg = ldg; g.c = (int)c; g.A = A; g.lda = lda; g.m = m; g.n = n;
  g.kunit = p.kunit; g.ks = p.ks;
  g.out = slices;
  g.sumsq_part = nullptr;
  g.vec_ok = (lda % 2 == 0) && ((reinterpret_cast<uintptr_t>(A) & (a_f32 ? 7 : 15)) == 0);
  const int row_blocks = (int)((c + kMaxWarps * kRowsPerWarp - 1) / (kMaxWarps * kRowsPerWarp));
  const int rows_first = (int)(c < kMaxWarps * kRowsPerWarp ? c : kMaxWarps * kRowsPerWarp);
  const int warps = (rows_first + kRowsPerWarp - 1) / kRowsPerWarp;
  dim3 grid((unsigned)((n + kCols - 1) / kCols), (unsigned)row_blocks, (unsigned)p.ks);
  if (a_f32) sketch_kernel<true><<<grid, warps * 32, 0, env.stream>>>(g);
  else sketch_kernel<false><<<grid, warps * 32, 0, env.stream>>>(g);
  return cudaGetLastError();
}

int64_t sketch_reduce_parts(int64_t c, int64_t n) { return (c * n + kReducePerCta - 1) / kReducePerCta; }

cudaError_t launch_sketch_reduce(const LaunchEnv& env, const double* slices, int nslices,
                                 int64_t c, int64_t n, double* Y, double* sumsq_part) {
  const int64_t total = c * n;
  const int64_t nblk = (total + kReducePerCta - 1) / kReducePerCta;
  sketch_reduce_kernel<<<(unsigned)nblk, 256, 0, env.stream>>>(slices, nslices, total, Y,
                                                                sumsq_part, kReducePerCta);
  return cudaGetLastError();
}

}  // namespace cur
