// sketch_tc.cu -- precision form of the initial sketch Y = G A of IterativeCUR
// (arXiv 2509.21963, Algorithm 1; Sec. 3.4 names the sketch as a primary
// cost) on the 5th-generation tensor cores (tcgen05, kind::f16, BF16 operands,
// FP32 accumulators in tensor memory).
//
// Arithmetic (exact by construction):
//   * G_q = clamp(rint(16 Z), -127, 127): the Gaussian sketch rounded to 8-bit
//     integers (every value exact in BF16).
//   * each column j of A (FP32) gets the scale 2^E_j with max_k |A(k,j)| < 2^E_j
//     (colmax pre-pass), and every entry is written with S signed base-256
//     digits d_s (|d_s| <= 256, exact in BF16): fix_S(x) = 2^(E_j-8S) sum d_s 256^s.
//   * one MMA product is |q d| <= 127 * 256 = 32512; a chunk of 512 rows sums to
//     at most 16646144 < 2^24, so the FP32 accumulator of each digit slice is an
//     exact integer.
//     Chunks are drained to int64 (exact) and combined over the K range; the
//     FP64 result 2^(E_j-8S) sum_s 256^s D_s is exact as long as it fits 53
//     bits (it does for S <= 3: < 2^47).
// So Y = G_q fix_S(A) exactly for S = 1, 2, 3 (the "BF16", "hi+lo" and
// "hi+mid+lo" forms, accurate to 2^-8S of each column's largest entry).  With
// S = 4 the int64 sums are still exact but may exceed 2^53, so Y is the exact
// value rounded once to FP64 (at most half an ulp).
//
// Kernel structure (one persistent CTA per SM, 10 warps):
//   warp 0      TMA producer: A tile (64 rows x 128 columns FP32, no swizzle)
//               and G_q tile (c_pad rows x 64 k BF16, 128-byte swizzle = the
//               K-major SW128 operand layout) into a stage ring.
//   warp 1      MMA issuer (one elected thread): per stage and digit slice,
//               four M=128 N=c_pad K=16 MMAs into the slice's accumulator.
//   warps 2-9   converters: FP32 tile -> S BF16 digit tiles written in the
//               K-major SW128 layout (the transpose happens here), then the
//               chunk drain: tcgen05.ld of the accumulators -> int64.
// Accumulators are double-buffered by chunk so the MMA of chunk z+1 overlaps
// the drain of chunk z.  Every wait is bounded: on timeout the CTA records an
// error and leaves its loops.
#include <cuda.h>

#include "gridbar.cuh"
#include "tc_ptx.cuh"

namespace cur {
namespace {

using namespace tc;

constexpr int kTileK = 64;        // rows of A per stage = MMA K per stage
constexpr int kTileN = 128;       // columns of A per CTA tile = MMA M
constexpr int kChunkTiles = 8;    // stages per exact accumulation chunk (512 rows)
constexpr int kConvWarps = 8;
constexpr int kThreads = (2 + kConvWarps) * 32;

// Packed pairs of FP32 (Blackwell f32x2): each lane rounds like the scalar
// instruction, so the digits below are bit-identical to scalar arithmetic.
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}
// 1.5 * 2^23 in both lanes: (y + M) - M rounds |y| < 2^22 to the nearest
// integer (ties to even) through the FP32 adder.
constexpr uint64_t kMagic2 = 0x4B4000004B400000ull;
constexpr uint64_t k256x2 = 0x4380000043800000ull;  // 256.0f in both lanes

struct TcArgs {
  int64_t m, n;
  int c, c_pad;
  const int* colexp;       // E_j per column (pre-pass)
  unsigned long long* acc; // c x n int64 sums (two's complement), zeroed by the host
  int64_t kunit;           // rows of A per work unit (multiple of 512)
  int ks;                  // work units along K
  int64_t nstrips;         // column strips of 128
  int* err;                // device error word
};

// Dynamic shared memory: an A ring of NA FP32 tiles (64 x 128 = 32 KB each),
// freed by the converters, and an operand ring of 2 stages, each holding S
// digit tiles (128 x 64 BF16 = 16 KB) and the G_q tile (c_pad x 64 BF16),
// freed by the MMA commit.  NA is as deep as ~210 KB allows (2..4).
template <int S, int CP>
struct Layout {
  static constexpr int kOpBytes = kTileN * kTileK * 2;          // 16384
  static constexpr int kGBytes = CP * kTileK * 2;               // CP * 128
  static constexpr int kABytes = kTileK * kTileN * 4;           // 32768
  static constexpr int kOpStage = S * kOpBytes + kGBytes;
  static constexpr int kNO = 2;
  static constexpr int kBudget = 212 * 1024;
  static constexpr int kNAraw = (kBudget - kNO * kOpStage) / kABytes;
  static constexpr int kNA = kNAraw > 4 ? 4 : (kNAraw < 2 ? 2 : kNAraw);
  static constexpr int kOpOffset = kNA * kABytes;
  static constexpr int kBarOffset = kOpOffset + kNO * kOpStage;
  static constexpr int kTotal = kBarOffset + 512 + 1024;        // barriers + alignment slack
  static constexpr uint32_t kTmemCols = (2 * S * CP <= 32) ? 32
                                        : (2 * S * CP <= 64) ? 64
                                        : (2 * S * CP <= 128) ? 128
                                        : (2 * S * CP <= 256) ? 256 : 512;
};

template <int S, int CP>
__global__ void __launch_bounds__(kThreads, 1)
    sketch_tc_kernel(const __grid_constant__ CUtensorMap mapA,
                     const __grid_constant__ CUtensorMap mapG, TcArgs g) {
  using L = Layout<S, CP>;
  constexpr int NA = L::kNA, NO = L::kNO;
  static_assert(2 * S * CP <= 512, "accumulators exceed tensor memory");
  static_assert(CP % 16 == 0 && CP >= 16 && CP <= 128, "N must be a multiple of 16, <= 128");
  static_assert(L::kTotal <= 227 * 1024, "shared memory");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOffset);
  uint64_t* fullA = bars;                 // [NA] A tile landed (TMA)
  uint64_t* emptyA = fullA + NA;          // [NA] A tile converted
  uint64_t* fullG = emptyA + NA;          // [NO] G_q tile landed (TMA)
  uint64_t* conv = fullG + NO;            // [NO] digit tiles written
  uint64_t* emptyO = conv + NO;           // [NO] MMAs done with the operand stage
  uint64_t* accf = emptyO + NO;           // [2] chunk accumulators complete
  uint64_t* acce = accf + 2;              // [2] chunk accumulators drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  int* s_abort = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NA; ++s) {
      mbar_init(&fullA[s], 1);
      mbar_init(&emptyA[s], kConvWarps * 32);
    }
    for (int s = 0; s < NO; ++s) {
      mbar_init(&fullG[s], 1);
      mbar_init(&conv[s], kConvWarps * 32);
      mbar_init(&emptyO[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], kConvWarps * 32);
    }
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(L::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t nunits = g.nstrips * g.ks;
  auto unit_tiles = [&](int64_t u) -> int {
    int64_t z = u / g.nstrips;
    int64_t k0 = z * g.kunit, k1 = min(g.m, k0 + g.kunit);
    return (int)((k1 - k0 + kTileK - 1) / kTileK);
  };

  if (warp == 0) {
    // ---------------- TMA producer of the FP32 A tiles ----------------
    if (lane == 0) {
      uint32_t t = 0;
      for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int64_t strip = u % g.nstrips, z = u / g.nstrips;
        const int nt = unit_tiles(u);
        for (int i = 0; i < nt; ++i, ++t) {
          const uint32_t s = t % NA;
          if (t >= (uint32_t)NA && !mbar_wait(&emptyA[s], ((t / NA) - 1) & 1)) {
            atomicCAS(g.err, 0, kDevTimeout);
            *((volatile int*)s_abort) = 1;
            break;
          }
          if (*((volatile int*)s_abort)) break;
          mbar_expect_tx(&fullA[s], (uint32_t)L::kABytes);
          tma_load_2d(smem + s * L::kABytes, &mapA, &fullA[s], (int)(strip * kTileN),
                      (int)(z * g.kunit) + i * kTileK);
        }
        if (*((volatile int*)s_abort)) break;
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CP >> 3) << 17) |
                             ((uint32_t)(kTileN >> 4) << 24);
      uint32_t t = 0, chunk = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const int nt = unit_tiles(u);
        for (int i = 0; i < nt && ok; ++i, ++t) {
          const uint32_t so = t % NO;
          const bool first = (i % kChunkTiles) == 0;
          const bool last = (i % kChunkTiles) == kChunkTiles - 1 || i == nt - 1;
          const uint32_t buf = chunk & 1;
          if (first && chunk >= 2 && !mbar_wait(&acce[buf], ((chunk >> 1) - 1) & 1)) { ok = false; break; }
          if (!mbar_wait(&conv[so], (t / NO) & 1)) { ok = false; break; }
          if (!mbar_wait(&fullG[so], (t / NO) & 1)) { ok = false; break; }
          tc_fence_after();
          uint8_t* st = smem + L::kOpOffset + so * L::kOpStage;
          const uint32_t gaddr = smem_u32(st + S * L::kOpBytes);
#pragma unroll
          for (int sl = 0; sl < S; ++sl) {
            const uint32_t aaddr = smem_u32(st + sl * L::kOpBytes);
            const uint32_t dcol = tmem + (uint32_t)((buf * S + sl) * CP);
#pragma unroll
            for (int kk = 0; kk < kTileK / 16; ++kk)
              mma_bf16(dcol, desc_sw128(aaddr + kk * 32), desc_sw128(gaddr + kk * 32), idesc,
                       (first && kk == 0) ? 0u : 1u);
          }
          mma_commit(&emptyO[so]);
          if (last) {
            mma_commit(&accf[buf]);
            ++chunk;
          }
        }
      }
      if (!ok) { atomicCAS(g.err, 0, kDevTimeout); *((volatile int*)s_abort) = 1; }
    }
  } else {
    // ---------------- converters (+ G_q tile loads) + drain ----------------
    const int ct = threadIdx.x - 64;           // 0..255
    const int jl = ct & (kTileN - 1);          // this thread's column in the tile
    const int half = ct >> 7;                  // k-group parity
    const int q = warp & 3;                    // TMEM lane quarter of this warp
    const int dh = (warp - 2) >> 2;            // 0: warps 2-5, 1: warps 6-9
    constexpr int HALF = CP / 2;               // sketch rows per drain thread
    long long acc[HALF];
#pragma unroll
    for (int r = 0; r < HALF; ++r) acc[r] = 0;
    uint32_t t = 0, chunk = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      const int64_t strip = u % g.nstrips, z = u / g.nstrips;
      const int nt = unit_tiles(u);
      const int64_t jg = strip * kTileN + jl;
      const int E = jg < g.n ? g.colexp[jg] : 0;
      const float sc = ldexpf(1.0f, min(8 - E, 126));  // columns below 2^-118: digits lose range
      const uint64_t sc2 = f2_pack(sc, sc);
      for (int i = 0; i < nt && ok; ++i, ++t) {
        const uint32_t sa = t % NA, so = t % NO;
        // the operand stage must be free of the MMAs that read it last time
        if (t >= (uint32_t)NO && !mbar_wait(&emptyO[so], ((t / NO) - 1) & 1)) { ok = false; break; }
        uint8_t* st = smem + L::kOpOffset + so * L::kOpStage;
        if (ct == 0) {
          mbar_expect_tx(&fullG[so], (uint32_t)L::kGBytes);
          tma_load_2d(st + S * L::kOpBytes, &mapG, &fullG[so], (int)(z * g.kunit) + i * kTileK, 0);
        }
        if (!mbar_wait(&fullA[sa], (t / NA) & 1)) { ok = false; break; }
        const float* At = reinterpret_cast<const float*>(smem + sa * L::kABytes);
#pragma unroll
        for (int it = 0; it < 4; ++it) {
          const int kg = half + 2 * it;
          uint32_t packed[S][4];
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            // rows k, k+1 of column jl as one f32x2 pair, scaled by 2^(8 - E_j) (exact)
            uint64_t y = f2_mul(f2_pack(At[(kg * 8 + e) * kTileN + jl],
                                        At[(kg * 8 + e + 1) * kTileN + jl]), sc2);
#pragma unroll
            for (int sl = S - 1; sl >= 0; --sl) {
              const uint64_t d = f2_sub(f2_add(y, kMagic2), kMagic2);
              // the two digits are integers |d| <= 256: their top halves are exact BF16
              packed[sl][e >> 1] = __byte_perm((uint32_t)d, (uint32_t)(d >> 32), 0x7632);
              if (sl > 0) y = f2_mul(f2_sub(y, d), k256x2);
            }
          }
          // K-major SW128: row jl, 16-byte chunk kg at (kg ^ (jl & 7))
          const uint32_t off = (uint32_t)((jl >> 3) * 1024 + (jl & 7) * 128 + ((kg ^ (jl & 7)) << 4));
#pragma unroll
          for (int sl = 0; sl < S; ++sl) {
            uint4 v = make_uint4(packed[sl][0], packed[sl][1], packed[sl][2], packed[sl][3]);
            *reinterpret_cast<uint4*>(st + sl * L::kOpBytes + off) = v;
          }
        }
        mbar_arrive(&emptyA[sa]);   // the FP32 tile may be refilled
        fence_async_smem();
        mbar_arrive(&conv[so]);
        const bool last = (i % kChunkTiles) == kChunkTiles - 1 || i == nt - 1;
        if (last) {
          // drain: accumulators of this chunk -> int64
          const uint32_t buf = chunk & 1;
          if (!mbar_wait(&accf[buf], (chunk >> 1) & 1)) { ok = false; break; }
          tc_fence_after();
#pragma unroll
          for (int gcol = 0; gcol < HALF; gcol += 8) {
            uint32_t r[S][8];
#pragma unroll
            for (int sl = 0; sl < S; ++sl)
              tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) +
                           (uint32_t)((buf * S + sl) * CP + dh * HALF + gcol),
                       r[sl]);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              long long v = 0;
#pragma unroll
              for (int sl = S - 1; sl >= 0; --sl) v = v * 256 + (long long)f2i_exact(r[sl][e]);
              acc[gcol + e] += v;
            }
          }
          tc_fence_before();
          mbar_arrive(&acce[buf]);
          ++chunk;
        }
      }
      if (!ok) break;
      // unit done: add this thread's (rows, column) sums into the global int64 sums
      const int jt = q * 32 + lane;   // the column this thread drained (TMEM lane)
      const int64_t jw = strip * kTileN + jt;
#pragma unroll
      for (int r = 0; r < HALF; ++r) {
        const int row = dh * HALF + r;
        if (row < g.c && jw < g.n && acc[r] != 0)
          atomicAdd(&g.acc[(int64_t)row * g.n + jw], (unsigned long long)acc[r]);
        acc[r] = 0;
      }
    }
    if (!ok) { atomicCAS(g.err, 0, kDevTimeout); *((volatile int*)s_abort) = 1; }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(L::kTmemCols));
  }
}

// ---- column scales: E_j with max_k |A(k,j)| < 2^E_j --------------------------
__global__ void colmax_kernel(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                              int64_t rows_per_cta, unsigned* __restrict__ colmax_bits) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta, r1 = min(m, r0 + rows_per_cta);
  unsigned mx = 0;
  for (int64_t k = r0; k < r1; ++k) {
    unsigned b = __float_as_uint(A[k * lda + j]) & 0x7FFFFFFFu;
    mx = b > mx ? b : mx;  // |x| compares as an unsigned integer (NaN sorts above Inf)
  }
  atomicMax(&colmax_bits[j], mx);
}

// E_j, and the scale 2^(E_j - 8S) that turns column j's integer sums into Y
// (NaN for a column holding Inf/NaN).
__global__ void colexp_kernel(const unsigned* __restrict__ colmax_bits, int64_t n, int S,
                              int* __restrict__ colexp, double* __restrict__ colscale) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const unsigned b = colmax_bits[j];
  int E = 0;
  if (b >= 0x7F800000u) E = 1 << 20;          // Inf/NaN: flagged by the reduction
  else if (b != 0) frexpf(__uint_as_float(b), &E);
  colexp[j] = E;
  colscale[j] = (E >= (1 << 20)) ? __longlong_as_double(0x7FF8000000000000LL)
                                 : ldexp(1.0, E - 8 * S);
}

// Y[i, j] = 2^(E_j - 8S) acc[i][j] (exact for S <= 3: |acc| < 2^53 and the
// scale is a power of two; one rounding to FP64 for S = 4): one thread per column of a 256-column block and a group of
// kReduceRows rows (blockIdx.y), plus per-CTA sums of squares.
constexpr int kReduceRows = 16;

__global__ void tc_reduce_kernel(const long long* __restrict__ acc, int64_t c, int64_t n,
                                 const double* __restrict__ colscale, double* __restrict__ Y,
                                 double* __restrict__ sumsq_part) {
  __shared__ double red[8];
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * kReduceRows, i1 = min(c, i0 + kReduceRows);
  double ss = 0.0;
  if (j < n) {
    const double sc = colscale[j];
    for (int64_t i = i0; i < i1; ++i) {
      const double y = (double)acc[i * n + j] * sc;
      Y[i * n + j] = y;
      ss = fma(y, y, ss);
    }
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    sumsq_part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// ---- G_q: 8-bit Gaussian sketch as BF16 (row stride ldq, zero padded) --------
__global__ void gaussian_q8_kernel(const double* __restrict__ G, int64_t c, int64_t m,
                                   int64_t ldq, uint16_t* __restrict__ Gq) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= c * ldq) return;
  const int64_t i = e / ldq, k = e - i * ldq;
  float q = 0.0f;
  if (k < m) {
    double v = rint(16.0 * G[i * m + k]);
    v = v > 127.0 ? 127.0 : (v < -127.0 ? -127.0 : v);
    q = (float)v;
  }
  Gq[e] = (uint16_t)(__float_as_uint(q) >> 16);  // exact: |q| <= 127
}

template <int S, int CP>
cudaError_t launch_tc(const LaunchEnv& env, const CUtensorMap& mA, const CUtensorMap& mG,
                      const TcArgs& a, int grid) {
  using L = Layout<S, CP>;
  cudaError_t e = cudaFuncSetAttribute((const void*)sketch_tc_kernel<S, CP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, L::kTotal);
  if (e != cudaSuccess) return e;
  sketch_tc_kernel<S, CP><<<grid, kThreads, L::kTotal, env.stream>>>(mA, mG, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gaussian_q8(const LaunchEnv& env, const double* G, int64_t c, int64_t m,
                               int64_t ldq, uint16_t* Gq) {
  const int64_t tot = c * ldq;
  gaussian_q8_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, env.stream>>>(G, c, m, ldq, Gq);
  return cudaGetLastError();
}

int sketch_tc_cpad(int c, int S) {
  int cp = (c + 15) / 16 * 16;
  if (cp < 16) cp = 16;
  // instantiated widths
  const int widths[] = {16, 32, 48, 64, 80, 96, 112, 128};
  for (int w : widths)
    if (w >= cp && 2 * S * w <= 512) return w;
  return -1;
}

size_t sketch_tc_scratch_bytes(int64_t c, int64_t m, int64_t n, int ks) {
  const int64_t ldq = (m + 63) / 64 * 64;
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) / 256 * 256; };
  add(sizeof(uint16_t) * (size_t)(c * ldq));     // G_q
  add(sizeof(unsigned) * (size_t)n);             // column max bits
  add(sizeof(int) * (size_t)n);                  // column exponents
  add(sizeof(double) * (size_t)n);               // column scales
  add(sizeof(long long) * (size_t)c * n);        // int64 sums
  return b;
}

int sketch_tc_plan_ks(const LaunchEnv& env, int64_t m, int64_t n) {
  const int64_t strips = (n + kTileN - 1) / kTileN;
  const int64_t chunks = (m + kTileK * kChunkTiles - 1) / (kTileK * kChunkTiles);
  // about 8 work units per SM (balance), each at least 2 chunks of rows
  int64_t ks = (8LL * env.num_sms + strips - 1) / strips;
  int64_t ks_max = (chunks + 1) / 2;
  if (ks > ks_max) ks = ks_max;
  return ks < 1 ? 1 : (int)ks;
}

cudaError_t launch_sketch_tc(const LaunchEnv& env, int S, const double* G, int64_t c,
                             const float* A, int64_t lda, int64_t m, int64_t n, void* scratch,
                             int ks, double* Y, double* sumsq_part, int64_t* nparts, int* err) {
  const int CP = sketch_tc_cpad((int)c, S);
  if (CP < 0) return cudaErrorInvalidValue;
  const int64_t ldq = (m + 63) / 64 * 64;
  char* p = static_cast<char*>(scratch);
  auto take = [&](size_t x) { char* r = p; p += (x + 255) / 256 * 256; return r; };
  uint16_t* Gq = (uint16_t*)take(sizeof(uint16_t) * (size_t)(c * ldq));
  unsigned* cmax = (unsigned*)take(sizeof(unsigned) * (size_t)n);
  int* cexp = (int*)take(sizeof(int) * (size_t)n);
  double* cscale = (double*)take(sizeof(double) * (size_t)n);
  long long* acc64 = (long long*)take(sizeof(long long) * (size_t)c * n);

  // G_q (BF16, rows padded to a multiple of 64 so TMA strides are 16-byte multiples)
  cudaError_t e = launch_gaussian_q8(env, G, c, m, ldq, Gq);
  if (e != cudaSuccess) return e;
  // column scales
  e = cudaMemsetAsync(cmax, 0, sizeof(unsigned) * (size_t)n, env.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc64, 0, sizeof(long long) * (size_t)(c * n), env.stream);
  if (e != cudaSuccess) return e;
  {
    int64_t rows_per = 512;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)((m + rows_per - 1) / rows_per));
    colmax_kernel<<<grid, 256, 0, env.stream>>>(A, lda, m, n, rows_per, cmax);
    colexp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, env.stream>>>(cmax, n, S, cexp, cscale);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap mA, mG;
  {
    cuuint64_t gdim[2] = {(cuuint64_t)n, (cuuint64_t)m};
    cuuint64_t gstride[1] = {(cuuint64_t)lda * 4};
    cuuint32_t box[2] = {kTileN, kTileK};
    cuuint32_t es[2] = {1, 1};
    if (enc(&mA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)A, gdim, gstride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    cuuint64_t gdim[2] = {(cuuint64_t)ldq, (cuuint64_t)c};
    cuuint64_t gstride[1] = {(cuuint64_t)ldq * 2};
    cuuint32_t box[2] = {kTileK, (cuuint32_t)CP};
    cuuint32_t es[2] = {1, 1};
    if (enc(&mG, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)Gq, gdim, gstride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  TcArgs a;
  a.m = m; a.n = n; a.c = (int)c; a.c_pad = CP; a.colexp = cexp;
  a.acc = reinterpret_cast<unsigned long long*>(acc64);
  const int64_t chunks = (m + kTileK * kChunkTiles - 1) / (kTileK * kChunkTiles);
  const int64_t chunks_per = (chunks + ks - 1) / ks;
  a.kunit = chunks_per * kTileK * kChunkTiles;
  a.ks = (int)((m + a.kunit - 1) / a.kunit);
  a.nstrips = (n + kTileN - 1) / kTileN;
  a.err = err;
  int64_t units = a.nstrips * a.ks;
  int grid = (int)(units < env.num_sms ? units : env.num_sms);

#define CUR_TC_CASE(SS, CC)                                    \
  if (S == SS && CP == CC) e = launch_tc<SS, CC>(env, mA, mG, a, grid); \
  else
  CUR_TC_CASE(1, 16) CUR_TC_CASE(1, 32) CUR_TC_CASE(1, 48) CUR_TC_CASE(1, 64)
  CUR_TC_CASE(1, 80) CUR_TC_CASE(1, 96) CUR_TC_CASE(1, 112) CUR_TC_CASE(1, 128)
  CUR_TC_CASE(2, 16) CUR_TC_CASE(2, 32) CUR_TC_CASE(2, 48) CUR_TC_CASE(2, 64)
  CUR_TC_CASE(2, 80) CUR_TC_CASE(2, 96) CUR_TC_CASE(2, 112) CUR_TC_CASE(2, 128)
  CUR_TC_CASE(3, 16) CUR_TC_CASE(3, 32) CUR_TC_CASE(3, 48) CUR_TC_CASE(3, 64)
  CUR_TC_CASE(3, 80)
  CUR_TC_CASE(4, 16) CUR_TC_CASE(4, 32) CUR_TC_CASE(4, 48) CUR_TC_CASE(4, 64)
  e = cudaErrorInvalidValue;
#undef CUR_TC_CASE
  if (e != cudaSuccess) return e;

  const dim3 rgrid((unsigned)((n + 255) / 256), (unsigned)((c + kReduceRows - 1) / kReduceRows));
  tc_reduce_kernel<<<rgrid, 256, 0, env.stream>>>(acc64, c, n, cscale, Y, sumsq_part);
  *nparts = (int64_t)rgrid.x * rgrid.y;
  return cudaGetLastError();
}

}  // namespace cur
