// resid_tc.cu -- the residual products of IterativeCUR's loop (Algorithm 1's
// row residual S^row = A(:,J_k) - C U R(:,J_k) and the factor R_k =
// A(I_k,:) - C U R(I_k,:) in the Lemma 1 form of Sec. 4.2:
//   D(n, i) -= sum_k P(i, k) Q(n, k)
// with P = L (m x r) or Rt^T (n x r) and Q = Rt(:,J_k)^T or L(I_k,:)) on the
// BF16 tensor cores with FP32 accumulation.  Every FP64 factor entry is split
// into NP BF16 planes x = x_0 + x_1 (+ x_2) + e (|e| <~ 2^-(8 NP + 1) |x|); the
// product keeps the plane pairs (a, b) with a + b < NP (3 MMAs for two planes,
// 6 for three), so its relative error is of order 2^-(8 NP) plus the FP32
// accumulation over r terms.  FP64 stays for A, D and everything else.
//
// Layout: the planes are K-major (row i of P holds P(i, 0..r) contiguously,
// row pitch ldp, a multiple of 64 elements), so 64-wide K tiles load with TMA
// and a 128-byte swizzle straight into the operand layout of tcgen05.mma
// (both operands K-major).  One CTA per 128 rows of P: warp 0 loads the NP
// P tiles and NP Q tiles of each 64-wide K chunk into a stage ring, warp 1
// issues the MMAs into one 128 x N FP32 accumulator in tensor memory, warps
// 2-5 subtract the accumulator from D (FP64, rows n, columns i) at the end.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "cur_internal.cuh"
#include "tc_ptx.cuh"

namespace cur {
namespace {

using namespace tc;

constexpr int kRTile = 128;            // rows of P per CTA (MMA M)
constexpr int kKTile = 64;             // K per stage (one 128-byte swizzled row)
constexpr int kRThreads = 192;         // 6 warps
constexpr int kRMaxN = 128;            // N (rows of Q) per launch
constexpr uint32_t kRTmemCols = 128;

template <int NP>
struct RLayout {
  static constexpr int kStages = NP == 2 ? 3 : 2;
  static constexpr int kPBytes = kRTile * kKTile * 2;           // 16 KB
  static constexpr int kQBytes = kRMaxN * kKTile * 2;           // 16 KB (N <= 128)
  static constexpr int kStageBytes = NP * (kPBytes + kQBytes);
  static constexpr int kBarOffset = kStages * kStageBytes;
  static constexpr int kTotal = kBarOffset + 256 + 1024;       // + barriers, alignment slack
};

struct RArgs {
  int64_t M;          // rows of P (columns of D)
  int N;              // rows of Q (rows of D), <= kRMaxN
  int64_t K;          // contraction length (r)
  double* D;          // N x M, row pitch ldd
  int64_t ldd;
  int* err;
};

template <int NP>
__global__ void __launch_bounds__(kRThreads, 1)
    resid_tc_kernel(const __grid_constant__ CUtensorMap mapP0, const __grid_constant__ CUtensorMap mapP1,
                    const __grid_constant__ CUtensorMap mapP2, const __grid_constant__ CUtensorMap mapQ0,
                    const __grid_constant__ CUtensorMap mapQ1, const __grid_constant__ CUtensorMap mapQ2,
                    RArgs g) {
  using L = RLayout<NP>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOffset);
  uint64_t* full = bars;                     // [kStages] tiles landed
  uint64_t* empty = full + L::kStages;       // [kStages] MMAs done with the stage
  uint64_t* accf = empty + L::kStages;       // every MMA done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);
  int* s_abort = reinterpret_cast<int*>(tmem_slot + 1);
  const CUtensorMap* mp[3] = {&mapP0, &mapP1, &mapP2};
  const CUtensorMap* mq[3] = {&mapQ0, &mapQ1, &mapQ2};

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)blockIdx.x * kRTile;
  const int nk = (int)((g.K + kKTile - 1) / kKTile);
  if (threadIdx.x == 0) {
    for (int s = 0; s < L::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, kRTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto abort_now = [&]() {
    atomicCAS(g.err, 0, kDevTimeout);
    *((volatile int*)s_abort) = 1;
  };
  auto aborted = [&]() { return *((volatile int*)s_abort) != 0; };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      for (int t = 0; t < nk; ++t) {
        const int s = t % L::kStages;
        if (aborted()) break;
        if (t >= L::kStages && !mbar_wait(&empty[s], ((t / L::kStages) - 1) & 1)) { abort_now(); break; }
        uint8_t* st = smem + s * L::kStageBytes;
        mbar_expect_tx(&full[s], (uint32_t)L::kStageBytes);   // whole boxes (out-of-range rows are zero-filled)
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          tma_load_2d(st + p * L::kPBytes, mp[p], &full[s], t * kKTile, (int)row0);
          tma_load_2d(st + NP * L::kPBytes + p * L::kQBytes, mq[p], &full[s], t * kKTile, 0);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kRTile, (g.N + 15) & ~15);
      bool ok = true;
      for (int t = 0; t < nk && ok; ++t) {
        const int s = t % L::kStages;
        if (!mbar_wait(&full[s], (t / L::kStages) & 1)) { ok = false; break; }
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * L::kStageBytes);
#pragma unroll
        for (int kk = 0; kk < kKTile / 16; ++kk) {
#pragma unroll
          for (int a = 0; a < NP; ++a)
#pragma unroll
            for (int b = 0; a + b < NP; ++b) {
              const uint32_t pa = st + a * L::kPBytes + kk * 32;
              const uint32_t qb = st + NP * L::kPBytes + b * L::kQBytes + kk * 32;
              mma_bf16(tmem, desc_sw128(pa), desc_sw128(qb), idesc,
                       (t == 0 && kk == 0 && a == 0 && b == 0) ? 0u : 1u);
            }
        }
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(accf);
      else abort_now();
    }
  } else {
    // ---------------- epilogue: D(n, i) -= acc(i, n) ----------------
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int64_t i = row0 + q * 32 + lane;
    bool ok = true;
    if (nk > 0 && !mbar_wait(accf, 0)) ok = false;
    if (ok && !aborted()) {
      tc_fence_after();
      for (int n0 = 0; n0 < g.N; n0 += 8) {
        uint32_t r[8];
        tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)n0, r);
        tmem_wait_ld();
        if (i < g.M) {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (n0 + e < g.N) {
              double* d = g.D + (int64_t)(n0 + e) * g.ldd + i;
              *d -= (double)__uint_as_float(r[e]);
            }
        }
      }
    } else if (!ok) {
      abort_now();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kRTmemCols);
  }
}

// FP64 entries src[t * st + i * si] (t < nt, i < M) -> plane entries
// plane_p[i * ldp + k0 + t]: x = x_0 + x_1 (+ x_2) + e, x_p in BF16 (round to
// nearest), each from the FP64 remainder of the previous ones.
__global__ void split_planes_kernel(const double* __restrict__ src, int64_t st, int64_t si, int64_t nt,
                                    int64_t M, __nv_bfloat16* p0, __nv_bfloat16* p1,
                                    __nv_bfloat16* p2, int64_t ldp, int64_t k0, bool negate) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  for (int64_t t = 0; t < nt; ++t) {
    double x = src[t * st + i * si];
    if (negate) x = -x;
    const __nv_bfloat16 h0 = __double2bfloat16(x);
    x -= (double)__bfloat162float(h0);
    const __nv_bfloat16 h1 = __double2bfloat16(x);
    const int64_t o = i * ldp + k0 + t;
    p0[o] = h0;
    p1[o] = h1;
    if (p2) {
      x -= (double)__bfloat162float(h1);
      p2[o] = __double2bfloat16(x);
    }
  }
}

// Rows idx[n] of the planes (entries 0..kp) -> dst_p[n * ldq + k].
__global__ void gather_plane_rows_kernel(const __nv_bfloat16* __restrict__ p0,
                                         const __nv_bfloat16* __restrict__ p1,
                                         const __nv_bfloat16* __restrict__ p2, int64_t ldp,
                                         int64_t prows, const int64_t* __restrict__ idx, int N,
                                         int64_t kp, __nv_bfloat16* q0, __nv_bfloat16* q1,
                                         __nv_bfloat16* q2, int64_t ldq) {
  const int n = blockIdx.y;
  const int64_t src = idx[n];
  const bool ok = src >= 0 && src < prows;
  const int64_t nv = kp / 8;   // 16-byte vectors (kp is a multiple of 64)
  for (int64_t v = threadIdx.x + (int64_t)blockIdx.x * blockDim.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x) {
    const uint4 z = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4*>(q0 + n * ldq)[v] = ok ? reinterpret_cast<const uint4*>(p0 + src * ldp)[v] : z;
    reinterpret_cast<uint4*>(q1 + n * ldq)[v] = ok ? reinterpret_cast<const uint4*>(p1 + src * ldp)[v] : z;
    if (q2)
      reinterpret_cast<uint4*>(q2 + n * ldq)[v] = ok ? reinterpret_cast<const uint4*>(p2 + src * ldp)[v] : z;
  }
}

// Per-CTA sums of squares of X (rows x cols, pitch ld), in a fixed order:
// parts[blockIdx.x] (summed by launch_sum_parts).
__global__ void sumsq_parts_kernel(const double* __restrict__ X, int64_t rows, int64_t cols,
                                   int64_t ld, double* parts) {
  __shared__ double red[8];
  double s = 0.0;
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rr = e / cols, cc = e - rr * cols;
    const double x = X[rr * ld + cc];
    s = fma(x, x, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    parts[blockIdx.x] = t;
  }
}

bool make_plane_map(CUtensorMap* map, const __nv_bfloat16* base, int64_t K, int64_t rows,
                    int64_t ld, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc || !base) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)(K > 0 ? K : 1), (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kKTile, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, gdim, gstride, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int64_t resid_plane_pitch(int64_t kmax) { return (kmax + 63) / 64 * 64; }

constexpr int kSumsqBlocks = 304;
int64_t resid_sumsq_parts() { return kSumsqBlocks; }

cudaError_t launch_sumsq_parts(const LaunchEnv& env, const double* X, int64_t rows, int64_t cols,
                               int64_t ld, double* parts) {
  sumsq_parts_kernel<<<kSumsqBlocks, 256, 0, env.stream>>>(X, rows, cols, ld, parts);
  return cudaGetLastError();
}

cudaError_t launch_split_planes(const LaunchEnv& env, const double* src, int64_t st, int64_t si,
                                int64_t nt, int64_t M, __nv_bfloat16* const* planes, int np,
                                int64_t ldp, int64_t k0, bool negate) {
  if (nt <= 0 || M <= 0) return cudaSuccess;
  split_planes_kernel<<<(unsigned)((M + 255) / 256), 256, 0, env.stream>>>(
      src, st, si, nt, M, planes[0], planes[1], np > 2 ? planes[2] : nullptr, ldp, k0, negate);
  return cudaGetLastError();
}

cudaError_t launch_gather_plane_rows(const LaunchEnv& env, __nv_bfloat16* const* planes, int np,
                                     int64_t ldp, int64_t prows, const int64_t* idx, int N,
                                     int64_t kp, __nv_bfloat16* const* dst, int64_t ldq) {
  if (N <= 0 || kp <= 0) return cudaSuccess;
  dim3 grid((unsigned)std::min<int64_t>((kp / 8 + 127) / 128, 64), (unsigned)N);
  gather_plane_rows_kernel<<<grid, 128, 0, env.stream>>>(
      planes[0], planes[1], np > 2 ? planes[2] : nullptr, ldp, prows, idx, N, kp, dst[0], dst[1],
      np > 2 ? dst[2] : nullptr, ldq);
  return cudaGetLastError();
}

cudaError_t launch_resid_tc(const LaunchEnv& env, int np, __nv_bfloat16* const* P, int64_t ldp,
                            int64_t M, __nv_bfloat16* const* Q, int64_t ldq, int N, int64_t K,
                            double* D, int64_t ldd, int* err) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  if ((np != 2 && np != 3) || N > kRMaxN || ldp % 64 || ldq % 64) return cudaErrorInvalidValue;
  CUtensorMap mP[3], mQ[3];
  for (int p = 0; p < 3; ++p) {
    const int src = p < np ? p : 0;   // unused maps repeat plane 0
    if (!make_plane_map(&mP[p], P[src], K, M, ldp, kRTile) ||
        !make_plane_map(&mQ[p], Q[src], K, N, ldq, kRMaxN))
      return cudaErrorInvalidValue;
  }
  RArgs g;
  g.M = M; g.N = N; g.K = K; g.D = D; g.ldd = ldd; g.err = err;
  const unsigned grid = (unsigned)((M + kRTile - 1) / kRTile);
  cudaError_t e;
  if (np == 2) {
    e = smem_opt_in((const void*)resid_tc_kernel<2>, RLayout<2>::kTotal);
    if (e != cudaSuccess) return e;
    resid_tc_kernel<2><<<grid, kRThreads, RLayout<2>::kTotal, env.stream>>>(mP[0], mP[1], mP[2],
                                                                             mQ[0], mQ[1], mQ[2], g);
  } else {
    e = smem_opt_in((const void*)resid_tc_kernel<3>, RLayout<3>::kTotal);
    if (e != cudaSuccess) return e;
    resid_tc_kernel<3><<<grid, kRThreads, RLayout<3>::kTotal, env.stream>>>(mP[0], mP[1], mP[2],
                                                                             mQ[0], mQ[1], mQ[2], g);
  }
  return cudaGetLastError();
}

}  // namespace cur
