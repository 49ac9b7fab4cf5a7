// sketch_fx.cu -- FP64 form of the initial sketch Y = G A of IterativeCUR
// (arXiv 2509.21963, Algorithm 1; Sec. 3.4 counts the sketch among the primary
// costs) on the 5th-generation tensor cores, exact by construction.
//
// GB300 has no fast FP64 arithmetic (about 2 DFMA per clock per SM), so an FP64
// sketch on the FP64 pipe runs ~30x below the HBM rate.  Here the products
// run on tcgen05 with BF16 operands holding small integers:
//   * G_q = clamp(rint(16 Z), -127, 127): the Gaussian sketch rounded to 8-bit
//     integers (exact in BF16).
//   * column j of A gets E_j with max |A(:,j)| < 2^E_j (a column-max pass);
//     every entry x becomes the integer X = trunc(x 2^(52 - E_j)), |X| < 2^52,
//     written with six balanced base-512 digits d_k in [-256, 255] (exact in
//     BF16): with K = 256 sum_k 512^k, X + K lies in [0, 2^54) and its 9-bit
//     fields f_k give d_k = f_k - 256, X = sum_k d_k 512^k.
//   * per digit an M = 128 (columns of A) x N = c_pad (rows of G_q) x K = 16
//     (rows of A) MMA accumulates in FP32 in tensor memory: |G_q d| <= 32512
//     and a chunk of 512 rows sums to at most 16646144 < 2^24, so every
//     accumulator is an exact integer.
//   * at the end of a chunk the six digit sums s_k are drained (exact int32)
//     and combined into lo = s_0 + 2^9 s_1 + 2^18 s_2 and hi = s_3 + 2^9 s_4 +
//     2^18 s_5 (int64, per CTA in shared memory), added into global int64 sums
//     when the CTA leaves a column strip; the reduction forms V = 2^27 hi + lo
//     exactly (128 bits), rounds it once to FP64 and scales by 2^(E_j - 52).
// So Y = RN(G_q trunc(A 2^(52-E))) 2^(E-52): the exact sketch of A's 52-bit
// fixed point, rounded once.
//
// Kernel structure (one persistent CTA per SM, 18 warps):
//   warp 0     TMA producer: A tiles (16 rows x 128 columns FP64 = 16 KB, no
//              swizzle) into a 4-stage ring, with an L2 prefetch running ahead;
//              G_q tiles (c_pad rows x 64 rows of A, BF16, 128-byte swizzle =
//              the K-major SW128 operand layout) into a 2-slot ring.
//   warp 1     allocates and frees tensor memory.
//   warps 2-17 converters in two groups of eight (two warps per 32-lane
//              quarter of tensor memory, eight rows each): group g converts
//              the stages i with i % 2 == g into its digit buffer (tcgen05.st:
//              lane = column of A, two rows of A per 32-bit column), and the
//              group's first thread issues that stage's six MMAs (one per
//              digit) with the digit tile as the A operand; all sixteen warps
//              drain and zero the accumulators at the end of each chunk.
// Tensor memory: six accumulators of c_pad columns, then two digit buffers of
// 6 x 8 columns.  Digits going to tensor memory instead of shared memory keep
// the shared-memory traffic at ~22 bytes per entry of A.  Every wait is
// bounded: on timeout the CTA records an error and leaves its loops.
#include <cuda.h>

#include "cur_internal.cuh"
#include "tc_ptx.cuh"

namespace cur {
namespace {

using namespace tc;

constexpr int kRows = 16;          // rows of A per stage = K of one MMA
constexpr int kCols = 128;         // columns of A per tile = MMA M
constexpr int kChunkRows = 512;    // rows per exact accumulation chunk (= work unit)
constexpr int kGRows = 64;         // rows of A per G_q tile (128-byte rows of BF16)
constexpr int kNA = 4;             // A ring depth
constexpr int kPrefetch = 12;      // tiles of A prefetched into L2 ahead of the ring
constexpr int kDigits = 6;
constexpr int kConvWarps = 16;     // two groups of 8: two warps per lane quarter each
constexpr int kThreads = (2 + kConvWarps) * 32;
constexpr int kOpCols = kDigits * (kRows / 2);   // tensor-memory columns of one digit buffer
// 256 * sum_{k<6} 512^k: adding it makes every 9-bit field of X + K equal d_k + 256.
constexpr uint64_t kBias = 0x0020100804020100ull;
constexpr uint32_t kBiasLo = (uint32_t)kBias, kBiasHi = (uint32_t)(kBias >> 32);
// Columns whose scale is at least 2^-970 hold every subnormal entry below the
// grid 2^(E-52) (X = 0); the fast digit path relies on it.
constexpr int kFastMinExp = -970;

static_assert(kBias == 256ull * (1ull + (1ull << 9) + (1ull << 18) + (1ull << 27) +
                                 (1ull << 36) + (1ull << 45)), "bias");

template <int CP>
struct FxLayout {
  static constexpr int kABytes = kRows * kCols * 8;             // 16384
  static constexpr int kGBytes = CP * kGRows * 2;               // CP * 128
  static constexpr int kAccBytes = 2 * CP * kCols * 8;          // lo and hi, int64
  static constexpr int kGOffset = kNA * kABytes;
  static constexpr int kAccOffset = kGOffset + 2 * kGBytes;
  static constexpr int kBarOffset = kAccOffset + kAccBytes;
  static constexpr int kTotal = kBarOffset + 256 + 1024;        // barriers + alignment slack
  static constexpr int kOpCol = kDigits * CP;                   // first digit-buffer column
  static constexpr int kUsed = kOpCol + 2 * kOpCols;
  static constexpr uint32_t kTmemCols = kUsed <= 32 ? 32 : kUsed <= 64 ? 64 : kUsed <= 128 ? 128
                                        : kUsed <= 256 ? 256 : 512;
};

struct FxArgs {
  int64_t m, n;
  int c;                   // rows of Y in this row group
  int64_t row0;            // first row of this group in Y / the global sums
  int64_t ldy;             // row stride of the global sums (n)
  const int* colexp;       // E_j per column
  unsigned long long* acc_lo;  // int64 sums (two's complement), zeroed by the host
  unsigned long long* acc_hi;
  int64_t nstrips, nchunks;    // units: strip-major (strip, chunk)
  int* err;
};

// Balanced base-512 digits of X = trunc(x 2^(52-E)) as FP32 values (exact
// integers in [-256, 255]), any finite column: rshift_base = 1023 + E.
__device__ __forceinline__ void fx_digits(uint64_t bits, int rshift_base, float (&f)[kDigits]) {
  const uint32_t hi = (uint32_t)(bits >> 32);
  const uint32_t e = (hi >> 20) & 0x7FFu;
  // |x| = M 2^(max(e,1) - 1075) with the implicit bit only for normal numbers
  const uint64_t M = (bits & 0x000FFFFFFFFFFFFFull) | ((uint64_t)(e != 0) << 52);
  // X = M 2^-r: a right shift (r >= 1) unless the column's largest entry is
  // itself subnormal (E < -1021), where the subnormal mantissas move left
  const int r = rshift_base - (int)(e != 0 ? e : 1u);
  const uint64_t T = (r >= 64) ? 0ull : (r >= 0 ? (M >> r) : (M << (-r)));
  const uint64_t sm = (uint64_t)((int64_t)(int32_t)hi >> 31);  // all ones for x < 0
  const uint64_t Yb = (T ^ sm) + (kBias - sm);                 // X + K, X = -T for x < 0
#pragma unroll
  for (int k = 0; k < kDigits; ++k) {
    const uint32_t fld = (uint32_t)(Yb >> (9 * k)) & 0x1FFu;
    // (2^23 + fld) - (2^23 + 256) = fld - 256, exact
    f[k] = __uint_as_float(0x4B000000u | fld) - 8388864.0f;
  }
}

// The same digits for columns with E >= kFastMinExp, branch-free: the implicit
// bit is always set (an exponent field of 0 gives a shift >= 53, X = 0), the
// 64-bit shift is one clamped shr.b64, and each 9-bit field goes
// straight into an FP32 mantissa whose exponent gives that field weight one
// (2^23 + f for bits 0-8, 2^14 + f for bits 9-17 left in place), so one
// subtraction yields the digit.  f[0..5] hold FP32 bit patterns.
__device__ __forceinline__ void fx_digits_fast(uint32_t lo, uint32_t hi, int rshift_base,
                                               uint32_t (&f)[kDigits]) {
  const uint32_t r = (uint32_t)(rshift_base - (int)((hi >> 20) & 0x7FFu));   // >= 1
  const uint32_t mh = (hi & 0x000FFFFFu) | 0x00100000u;
  uint64_t T64;   // PTX clamps the shift at 64: X = 0 for r >= 64
  asm("shr.b64 %0, %1, %2;" : "=l"(T64) : "l"(((uint64_t)mh << 32) | lo), "r"(r));
  const uint32_t th = (uint32_t)(T64 >> 32), tl = (uint32_t)T64;
  const uint32_t sm = (uint32_t)((int32_t)hi >> 31);           // all ones for x < 0
  uint32_t yl, yh;                                             // X + K, X = -T for x < 0
  asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, %5;"
      : "=r"(yl), "=r"(yh)
      : "r"(tl ^ sm), "r"(kBiasLo - sm), "r"(th ^ sm), "r"(kBiasHi));
  const uint32_t t = __funnelshift_r(yl, yh, 18);              // bits 18..49
  const uint32_t u = yh >> 4;                                  // bits 36..63
  f[0] = 0x4B000000u | (yl & 0x1FFu);
  f[1] = 0x46800000u | (yl & 0x3FE00u);
  f[2] = 0x4B000000u | (t & 0x1FFu);
  f[3] = 0x46800000u | (t & 0x3FE00u);
  f[4] = 0x4B000000u | (u & 0x1FFu);
  f[5] = 0x46800000u | (u & 0x3FE00u);
  // (2^23 + f) - (2^23 + 256) and (2^14 + f) - (2^14 + 256), two lanes at a time
  constexpr uint64_t kSub = ((uint64_t)0xC6820000u << 32) | 0xCB000100u;   // (-16640, -8388864)
#pragma unroll
  for (int k = 0; k < kDigits; k += 2) {
    uint64_t v = (uint64_t)f[k] | ((uint64_t)f[k + 1] << 32), d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(v), "l"(kSub));
    f[k] = (uint32_t)d;
    f[k + 1] = (uint32_t)(d >> 32);
  }
}

template <int CP>
__global__ void __launch_bounds__(kThreads, 1)
    sketch_fx_kernel(const __grid_constant__ CUtensorMap mapA,
                     const __grid_constant__ CUtensorMap mapG, FxArgs g) {
  using L = FxLayout<CP>;
  static_assert(CP % 16 == 0 && CP >= 16 && CP <= 64, "N must be a multiple of 16, <= 64");
  static_assert(L::kUsed <= 512, "tensor memory");
  static_assert(L::kTotal <= 227 * 1024, "shared memory");
  constexpr int QROWS = CP / 4;            // rows of Y drained per converter warp
  constexpr int kSuper = kGRows / kRows;   // stages per G_q tile
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  long long* acc_lo = reinterpret_cast<long long*>(smem + L::kAccOffset);   // [CP][128]
  long long* acc_hi = acc_lo + CP * kCols;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOffset);
  uint64_t* fullA = bars;            // [kNA] A tile landed (TMA)
  uint64_t* emptyA = fullA + kNA;    // [kNA] A tile read by its converter group
  uint64_t* fullG = emptyA + kNA;    // [2]   G_q tile landed (TMA)
  uint64_t* emptyG = fullG + 2;      // [2]   both groups' MMAs done with the G_q tile
  uint64_t* opfull = emptyG + 2;     // [2]   group's digit buffer written
  uint64_t* opempty = opfull + 2;    // [2]   MMAs done with the group's digit buffer
  uint64_t* accf = opempty + 2;      // both groups' MMAs of the chunk complete
  uint64_t* drained = accf + 1;      // accumulators read and zeroed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drained + 1);
  int* s_abort = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kNA; ++s) {
      mbar_init(&fullA[s], 1);
      mbar_init(&emptyA[s], kConvWarps / 2);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&fullG[s], 1);
      mbar_init(&emptyG[s], 2);
      mbar_init(&opfull[s], kConvWarps / 2);
      mbar_init(&opempty[s], 1);
    }
    mbar_init(accf, 2);
    mbar_init(drained, kConvWarps);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, L::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // this CTA's units: a contiguous range of the strip-major (strip, chunk) list;
  // every unit has an even number of stages (a zero stage past the last row
  // pads an odd count), so stage i of every unit goes to converter group i % 2
  // (units are walked with incremental (strip, chunk) counters: 64-bit
  // divisions on the single-thread producer path cost hundreds of cycles)
  const int64_t nunits = g.nstrips * g.nchunks;
  const int64_t u0 = nunits * blockIdx.x / gridDim.x;
  const int64_t u1 = nunits * (blockIdx.x + 1) / gridDim.x;
  const int nch = (int)g.nchunks;
  const int strip0 = (int)(u0 / nch), z0 = (int)(u0 % nch);
  const int last_rows = (int)(g.m - (int64_t)(nch - 1) * kChunkRows);     // rows of the last chunk
  const int last_nt = (((last_rows + kRows - 1) / kRows) + 1) & ~1;
  auto unit_stages = [&](int z) -> int { return z == nch - 1 ? last_nt : kChunkRows / kRows; };
  auto abort_now = [&]() {
    atomicCAS(g.err, 0, kDevTimeout);
    *((volatile int*)s_abort) = 1;
  };
  auto aborted = [&]() { return *((volatile int*)s_abort) != 0; };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t t = 0, gs = 0;
      bool ok = true;
      // L2 prefetch cursor, kPrefetch tiles ahead of the loads
      int64_t pu = u0;
      int pstrip = strip0, pz = z0, pi = 0;
      auto prefetch_next = [&]() {
        if (pu >= u1) return;
        tma_prefetch_2d(&mapA, pstrip * kCols, pz * kChunkRows + pi * kRows);
        if (++pi == unit_stages(pz)) {
          pi = 0;
          ++pu;
          if (++pz == nch) { pz = 0; ++pstrip; }
        }
      };
      for (int k = 0; k < kPrefetch; ++k) prefetch_next();
      int strip = strip0, z = z0;
      for (int64_t u = u0; u < u1 && ok; ++u, (++z == nch ? (z = 0, ++strip) : 0)) {
        const int nt = unit_stages(z);
        for (int i = 0; i < nt; ++i, ++t) {
          if (aborted()) { ok = false; break; }
          prefetch_next();
          if (i % kSuper == 0) {
            const uint32_t sl = gs & 1;
            if (gs >= 2 && !mbar_wait(&emptyG[sl], ((gs >> 1) - 1) & 1)) { abort_now(); ok = false; break; }
            mbar_expect_tx(&fullG[sl], (uint32_t)L::kGBytes);
            tma_load_2d(smem + L::kGOffset + sl * L::kGBytes, &mapG, &fullG[sl],
                        z * kChunkRows + i * kRows, 0);
            ++gs;
          }
          const uint32_t s = t % kNA;
          if (t >= (uint32_t)kNA && !mbar_wait(&emptyA[s], ((t / kNA) - 1) & 1)) { abort_now(); ok = false; break; }
          mbar_expect_tx(&fullA[s], (uint32_t)L::kABytes);
          tma_load_2d(smem + s * L::kABytes, &mapA, &fullA[s], strip * kCols,
                      z * kChunkRows + i * kRows);
        }
      }
    }
  } else if (warp >= 2) {
    // ------- converters; the first thread of each group issues its MMAs -------
    const int cw = warp - 2;                 // 0..15
    const int grp = cw >> 3;                 // converter group: stages i % 2 == grp
    const int q = warp & 3;                  // tensor-memory lane quarter of this warp
    const int hk = (cw >> 2) & 1;            // which 8 of the stage's 16 rows
    const int jl = q * 32 + lane;            // this thread's column of the tile (= TMEM lane)
    const int rb = (cw >> 2) * QROWS;        // rows of Y this thread drains: [rb, rb + QROWS)
    const bool issuer = (cw & 7) == 0 && lane == 0;
    const uint32_t tlane = (uint32_t)(q * 32) << 16;
    constexpr uint32_t idesc = idesc_bf16(kCols, CP);
    const uint32_t zero4[4] = {0u, 0u, 0u, 0u};
    // every MMA accumulates: the accumulators start at zero and every drain
    // zeroes what it read, so the two groups' MMAs need no ordering
    for (int r = rb; r < rb + QROWS; ++r) acc_lo[r * kCols + jl] = acc_hi[r * kCols + jl] = 0;
#pragma unroll 1
    for (int g4 = 0; g4 < QROWS; g4 += 4)
      for (int d = 0; d < kDigits; ++d) tmem_st4(tmem + tlane + (uint32_t)(d * CP + rb + g4), zero4);
    tmem_wait_st();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(drained);
    uint32_t t = 0, ch = 0, gs = 0;
    int cur_strip = -1;
    int base = 0;
    bool fast = true;
    bool ok = true;
    int strip = strip0, z = z0;
    for (int64_t u = u0; u < u1 && ok; ++u, (++z == nch ? (z = 0, ++strip) : 0)) {
      const int nt = unit_stages(z);
      if (strip != cur_strip) {
        const int64_t jg = (int64_t)strip * kCols + jl;
        const int E = jg < g.n ? g.colexp[jg] : 0;
        base = 1023 + E;
        fast = __all_sync(0xffffffffu, E >= kFastMinExp);
        cur_strip = strip;
      }
      for (int i = 0; i < nt; ++i, ++t) {
        if ((i & 1) != grp) continue;
        const uint32_t s = t % kNA;
        if (!mbar_wait(&fullA[s], (t / kNA) & 1)) { ok = false; break; }
        const uint2* At = reinterpret_cast<const uint2*>(smem + s * L::kABytes) + hk * 8 * kCols;
        uint32_t w[kDigits][4];
        if (fast) {
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            uint32_t f0[kDigits], f1[kDigits];
            const uint2 x0 = At[(2 * p) * kCols + jl], x1 = At[(2 * p + 1) * kCols + jl];
            fx_digits_fast(x0.x, x0.y, base, f0);
            fx_digits_fast(x1.x, x1.y, base, f1);
#pragma unroll
            for (int d = 0; d < kDigits; ++d)   // two BF16 digits (rows 2p, 2p+1) per column
              asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w[d][p])
                  : "f"(__uint_as_float(f1[d])), "f"(__uint_as_float(f0[d])));
          }
        } else {
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            float f0[kDigits], f1[kDigits];
            const uint2 x0 = At[(2 * p) * kCols + jl], x1 = At[(2 * p + 1) * kCols + jl];
            fx_digits(((uint64_t)x0.y << 32) | x0.x, base, f0);
            fx_digits(((uint64_t)x1.y << 32) | x1.x, base, f1);
#pragma unroll
            for (int d = 0; d < kDigits; ++d)
              w[d][p] = __byte_perm(__float_as_uint(f0[d]), __float_as_uint(f1[d]), 0x7632);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&emptyA[s]);   // the FP64 rows may be refilled
        // the digits are in registers: only now wait for the MMAs that read this
        // group's buffer last (the conversion overlapped them)
        if (t >= 2 && !mbar_wait(&opempty[grp], ((t >> 1) - 1) & 1)) { ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int d = 0; d < kDigits; ++d)
          tmem_st4(tmem + tlane +
                       (uint32_t)(L::kOpCol + grp * kOpCols + d * (kRows / 2) + hk * 4),
                   w[d]);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&opfull[grp]);
        if (issuer) {
          const uint32_t sl = gs & 1;
          const int kk = i % kSuper;
          if (i == grp && !mbar_wait(drained, ch & 1)) { ok = false; break; }
          if (!mbar_wait(&opfull[grp], (t >> 1) & 1)) { ok = false; break; }
          if (kk == grp && !mbar_wait(&fullG[sl], (gs >> 1) & 1)) { ok = false; break; }
          tc_fence_after();
          const uint32_t gaddr = smem_u32(smem + L::kGOffset + sl * L::kGBytes) + kk * 32;
#pragma unroll
          for (int d = 0; d < kDigits; ++d)
            mma_bf16_tmem_a(tmem + (uint32_t)(d * CP),
                            tmem + (uint32_t)(L::kOpCol + grp * kOpCols + d * (kRows / 2)),
                            desc_sw128(gaddr), idesc, 1u);
          mma_commit(&opempty[grp]);
          if (kk >= kSuper - 2 || i + 2 >= nt) {   // this group's last stage on the G_q tile
            mma_commit(&emptyG[sl]);
            ++gs;
          }
          if (i + 2 >= nt) mma_commit(accf);       // this group's last stage of the chunk
        }
      }
      if (!ok) break;
      // chunk drain: six digit sums per (row of Y, column of A) -> lo, hi; zero them
      if (!mbar_wait(accf, ch & 1)) { ok = false; break; }
      tc_fence_after();
#pragma unroll 1
      for (int g4 = 0; g4 < QROWS; g4 += 4) {
        uint32_t v[kDigits][4];
#pragma unroll
        for (int d = 0; d < kDigits; ++d) tmem_ld4(tmem + tlane + (uint32_t)(d * CP + rb + g4), v[d]);
        tmem_wait_ld();
#pragma unroll
        for (int d = 0; d < kDigits; ++d) tmem_st4(tmem + tlane + (uint32_t)(d * CP + rb + g4), zero4);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const long long lo = (long long)f2i_exact(v[0][e]) +
                               ((long long)f2i_exact(v[1][e]) << 9) +
                               ((long long)f2i_exact(v[2][e]) << 18);
          const long long hi = (long long)f2i_exact(v[3][e]) +
                               ((long long)f2i_exact(v[4][e]) << 9) +
                               ((long long)f2i_exact(v[5][e]) << 18);
          const int r = rb + g4 + e;
          acc_lo[r * kCols + jl] += lo;
          acc_hi[r * kCols + jl] += hi;
        }
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(drained);
      ++ch;
      // leaving the strip: add this thread's sums into the global ones
      if (u + 1 == u1 || z + 1 == nch) {
        const int64_t jg = (int64_t)strip * kCols + jl;
        for (int r = rb; r < rb + QROWS; ++r) {
          const long long lo = acc_lo[r * kCols + jl], hi = acc_hi[r * kCols + jl];
          if (r < g.c && jg < g.n) {
            const int64_t o = (g.row0 + r) * g.ldy + jg;
            if (lo) atomicAdd(&g.acc_lo[o], (unsigned long long)lo);
            if (hi) atomicAdd(&g.acc_hi[o], (unsigned long long)hi);
          }
          acc_lo[r * kCols + jl] = acc_hi[r * kCols + jl] = 0;
        }
      }
    }
    if (!ok) abort_now();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, L::kTmemCols);
  }
}

// ---- column scales: E_j with max_k |A(k,j)| < 2^E_j ------------------------
// |x| compares as an unsigned integer of its bit pattern (NaN above Inf).
__global__ void colmax_f64_kernel(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                  int64_t rows_per_cta, unsigned long long* __restrict__ cmax) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta, r1 = min(m, r0 + rows_per_cta);
  const unsigned long long* p = reinterpret_cast<const unsigned long long*>(A) + j;
  unsigned long long mx[4] = {0, 0, 0, 0};
  int64_t k = r0;
  for (; k + 4 <= r1; k += 4) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const unsigned long long b = __ldg(p + (k + e) * lda) & 0x7FFFFFFFFFFFFFFFull;
      mx[e] = b > mx[e] ? b : mx[e];
    }
  }
  for (; k < r1; ++k) {
    const unsigned long long b = __ldg(p + k * lda) & 0x7FFFFFFFFFFFFFFFull;
    mx[0] = b > mx[0] ? b : mx[0];
  }
  unsigned long long v = mx[0] > mx[1] ? mx[0] : mx[1];
  const unsigned long long w = mx[2] > mx[3] ? mx[2] : mx[3];
  v = v > w ? v : w;
  if (v) atomicMax(&cmax[j], v);
}

// E_j (frexp of the column max; 0 for a zero column), 1 << 20 for Inf/NaN.
__global__ void colexp_f64_kernel(const unsigned long long* __restrict__ cmax, int64_t n,
                                  int* __restrict__ colexp) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const unsigned long long b = cmax[j];
  int E = 0;
  if (b >= 0x7FF0000000000000ull) E = 1 << 20;
  else if (b != 0) frexp(__longlong_as_double((long long)b), &E);
  colexp[j] = E;
}

// Round the 128-bit integer 2^27 hi + lo once to FP64 (to nearest, ties to
// even): the magnitude's leading 64 bits with a sticky bit for the rest, then
// one conversion (the 11 extra bits and the sticky bit make it exact RN).
__device__ double fx_round(long long hi, long long lo) {
  // v = hi * 2^27 + lo as (vh, vl), two's complement
  unsigned long long vl = (unsigned long long)hi << 27;
  long long vh = hi >> 37;
  const unsigned long long s = vl + (unsigned long long)lo;
  vh += (lo < 0 ? -1 : 0) + (s < vl ? 1 : 0);
  vl = s;
  const bool neg = vh < 0;
  unsigned long long uh = (unsigned long long)vh, ul = vl;
  if (neg) {  // magnitude
    ul = ~ul + 1ull;
    uh = ~uh + (ul == 0 ? 1ull : 0ull);
  }
  double d;
  if (uh == 0) {
    d = __ull2double_rn(ul);
  } else {
    const int sh = 64 - __clzll((long long)uh);               // 1..64 bits above the low word
    unsigned long long top = sh == 64 ? uh : ((uh << (64 - sh)) | (ul >> sh));
    const unsigned long long rest = sh == 64 ? ul : (ul << (64 - sh));
    top |= (rest != 0) ? 1ull : 0ull;
    d = __ull2double_rn(top) * __longlong_as_double((long long)(1023 + sh) << 52);  // exact 2^sh
  }
  return neg ? -d : d;
}

// y 2^e with one rounding (the first factor keeps y normal and exact).
__device__ double fx_scale(double y, int e) {
  const int e1 = e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
  const int e2 = e - e1;                                      // in [-126, 100] for our exponents
  y *= __longlong_as_double((long long)(1023 + e1) << 52);
  if (e2 != 0) {
    y *= e2 >= -1022 ? __longlong_as_double((long long)(1023 + e2) << 52)
                     : __longlong_as_double(1ll << (e2 + 1074));   // subnormal power of two
  }
  return y;
}

constexpr int kReduceRows = 16;

// Y[i, j] = RN(2^27 hi + lo) 2^(E_j - 52) (NaN for a non-finite column), one
// thread per column of a 256-column block and kReduceRows rows, plus per-CTA
// sums of squares.
__global__ void fx_reduce_kernel(const long long* __restrict__ acc_lo,
                                 const long long* __restrict__ acc_hi, int64_t c, int64_t n,
                                 const int* __restrict__ colexp, double* __restrict__ Y,
                                 double* __restrict__ sumsq_part) {
  __shared__ double red[8];
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * kReduceRows, i1 = min(c, i0 + kReduceRows);
  double ss = 0.0;
  if (j < n) {
    const int E = colexp[j];
    for (int64_t i = i0; i < i1; ++i) {
      const int64_t o = i * n + j;
      const double y = E >= (1 << 20) ? __longlong_as_double(0x7FF8000000000000LL)
                                      : fx_scale(fx_round(acc_hi[o], acc_lo[o]), E - 52);
      Y[o] = y;
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

template <int CP>
cudaError_t launch_fx(const LaunchEnv& env, const CUtensorMap& mA, const CUtensorMap& mG,
                      const FxArgs& a, int grid) {
  using L = FxLayout<CP>;
  cudaError_t e = smem_opt_in((const void*)sketch_fx_kernel<CP>, L::kTotal);
  if (e != cudaSuccess) return e;
  sketch_fx_kernel<CP><<<grid, kThreads, L::kTotal, env.stream>>>(mA, mG, a);
  return cudaGetLastError();
}

int64_t ldq_of(int64_t m) { return (m + kGRows - 1) / kGRows * kGRows; }

}  // namespace

size_t sketch_fx_scratch_bytes(int64_t c, int64_t m, int64_t n) {
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) / 256 * 256; };
  add(sizeof(uint16_t) * (size_t)(c * ldq_of(m)));   // G_q
  add(sizeof(unsigned long long) * (size_t)n);        // column max bits
  add(sizeof(int) * (size_t)n);                       // column exponents
  add(2 * sizeof(long long) * (size_t)(c * n));       // lo and hi sums
  return b;
}

int64_t sketch_fx_max_parts(int64_t c, int64_t n) {
  return ((n + 255) / 256) * ((c + kReduceRows - 1) / kReduceRows);
}

namespace {
struct FxScratch {
  uint16_t* Gq;
  unsigned long long* cmax;
  int* cexp;
  long long* acc_lo;
  long long* acc_hi;
};

FxScratch carve_fx(void* scratch, int64_t c, int64_t m, int64_t n) {
  const int64_t ldq = ldq_of(m);
  char* p = static_cast<char*>(scratch);
  auto take = [&](size_t x) { char* r = p; p += (x + 255) / 256 * 256; return r; };
  FxScratch f;
  f.Gq = (uint16_t*)take(sizeof(uint16_t) * (size_t)(c * ldq));
  f.cmax = (unsigned long long*)take(sizeof(unsigned long long) * (size_t)n);
  f.cexp = (int*)take(sizeof(int) * (size_t)n);
  long long* acc = (long long*)take(2 * sizeof(long long) * (size_t)(c * n));
  f.acc_lo = acc;
  f.acc_hi = acc + c * n;
  return f;
}

bool fx_args_ok(int64_t c, const double* A, int64_t lda, int64_t m, int64_t n) {
  return c >= 1 && m >= 1 && n >= 1 && lda >= n && !(lda & 1) &&
         !(reinterpret_cast<uintptr_t>(A) & 15);
}
}  // namespace

cudaError_t launch_sketch_fx_scales(const LaunchEnv& env, const double* G, int64_t c,
                                    const double* A, int64_t lda, int64_t m, int64_t n,
                                    void* scratch) {
  if (!fx_args_ok(c, A, lda, m, n)) return cudaErrorInvalidValue;
  const int64_t ldq = ldq_of(m);
  const FxScratch f = carve_fx(scratch, c, m, n);
  cudaError_t e = launch_gaussian_q8(env, G, c, m, ldq, f.Gq);
  if (e == cudaSuccess) e = launch_sketch_fx_colscales(env, c, A, lda, m, n, scratch);
  return e;
}

cudaError_t launch_sketch_fx_q8(const LaunchEnv& env, const double* G, int64_t c, int64_t m,
                                int64_t n, void* scratch) {
  const FxScratch f = carve_fx(scratch, c, m, n);
  return launch_gaussian_q8(env, G, c, m, ldq_of(m), f.Gq);
}

cudaError_t launch_sketch_fx_colscales(const LaunchEnv& env, int64_t c, const double* A,
                                       int64_t lda, int64_t m, int64_t n, void* scratch) {
  cudaError_t e = launch_sketch_fx_zero(env, c, A, lda, m, n, scratch);
  if (e == cudaSuccess) e = launch_sketch_fx_colscales_range(env, c, A, lda, m, n, scratch, 0, n);
  return e;
}

cudaError_t launch_sketch_fx_zero(const LaunchEnv& env, int64_t c, const double* A, int64_t lda,
                                  int64_t m, int64_t n, void* scratch) {
  if (!fx_args_ok(c, A, lda, m, n)) return cudaErrorInvalidValue;
  const FxScratch f = carve_fx(scratch, c, m, n);
  cudaError_t e = cudaMemsetAsync(f.cmax, 0, sizeof(unsigned long long) * (size_t)n, env.stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(f.acc_lo, 0, 2 * sizeof(long long) * (size_t)(c * n), env.stream);
  return e;
}

cudaError_t launch_sketch_fx_colscales_range(const LaunchEnv& env, int64_t c, const double* A,
                                             int64_t lda, int64_t m, int64_t n, void* scratch,
                                             int64_t c0, int64_t c1) {
  cudaError_t e = launch_sketch_fx_colmax_block(env, c, A, lda, m, n, scratch, 0, m, c0, c1);
  if (e == cudaSuccess) e = launch_sketch_fx_colexp_range(env, c, A, lda, m, n, scratch, c0, c1);
  return e;
}

cudaError_t launch_sketch_fx_colmax_block(const LaunchEnv& env, int64_t c, const double* A,
                                          int64_t lda, int64_t m, int64_t n, void* scratch,
                                          int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
  if (!fx_args_ok(c, A, lda, m, n) || c0 < 0 || c1 > n || c0 >= c1 || r0 < 0 || r1 > m ||
      r0 >= r1)
    return cudaErrorInvalidValue;
  const FxScratch f = carve_fx(scratch, c, m, n);
  const int64_t nb = c1 - c0, mb = r1 - r0;
  const int64_t rows_per = 512;
  dim3 grid((unsigned)((nb + 255) / 256), (unsigned)((mb + rows_per - 1) / rows_per));
  colmax_f64_kernel<<<grid, 256, 0, env.stream>>>(A + r0 * lda + c0, lda, mb, nb, rows_per,
                                                  f.cmax + c0);
  return cudaGetLastError();
}

cudaError_t launch_sketch_fx_colexp_range(const LaunchEnv& env, int64_t c, const double* A,
                                          int64_t lda, int64_t m, int64_t n, void* scratch,
                                          int64_t c0, int64_t c1) {
  if (!fx_args_ok(c, A, lda, m, n) || c0 < 0 || c1 > n || c0 >= c1) return cudaErrorInvalidValue;
  const FxScratch f = carve_fx(scratch, c, m, n);
  const int64_t nb = c1 - c0;
  colexp_f64_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, env.stream>>>(f.cmax + c0, nb,
                                                                         f.cexp + c0);
  return cudaGetLastError();
}

cudaError_t launch_sketch_fx_main(const LaunchEnv& env, int64_t c, const double* A, int64_t lda,
                                  int64_t m, int64_t n, void* scratch, double* Y,
                                  double* sumsq_part, int64_t* nparts, int* err) {
  cudaError_t e = launch_sketch_fx_main_range(env, c, A, lda, m, n, scratch, 0, n, err);
  if (e == cudaSuccess) e = launch_sketch_fx_reduce(env, c, A, lda, m, n, scratch, Y, sumsq_part, nparts);
  return e;
}

cudaError_t launch_sketch_fx_main_range(const LaunchEnv& env, int64_t c, const double* A,
                                        int64_t lda, int64_t m, int64_t n, void* scratch,
                                        int64_t c0, int64_t c1, int* err) {
  if (!fx_args_ok(c, A, lda, m, n) || c0 < 0 || c1 > n || c0 >= c1 || (c0 & 1))
    return cudaErrorInvalidValue;
  const int64_t ldq = ldq_of(m);
  const FxScratch f = carve_fx(scratch, c, m, n);
  const int64_t nb = c1 - c0;
  cudaError_t e = cudaSuccess;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap mA;
  {
    cuuint64_t gdim[2] = {(cuuint64_t)nb, (cuuint64_t)m};
    cuuint64_t gstride[1] = {(cuuint64_t)lda * 8};
    cuuint32_t box[2] = {kCols, kRows};
    cuuint32_t es[2] = {1, 1};
    if (enc(&mA, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)(A + c0), gdim, gstride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  FxArgs a;
  a.m = m; a.n = nb; a.ldy = n; a.colexp = f.cexp + c0;   // the block's columns, the full sums' pitch
  a.acc_lo = reinterpret_cast<unsigned long long*>(f.acc_lo + c0);
  a.acc_hi = reinterpret_cast<unsigned long long*>(f.acc_hi + c0);
  a.nstrips = (nb + kCols - 1) / kCols;
  a.nchunks = (m + kChunkRows - 1) / kChunkRows;
  a.err = err;
  const int64_t units = a.nstrips * a.nchunks;
  const int grid = (int)(units < env.num_sms ? units : env.num_sms);
  // row groups of at most 64 rows of G_q: one pass of the block's columns each
  for (int64_t g0 = 0; g0 < c; g0 += 64) {
    const int64_t cg = c - g0 < 64 ? c - g0 : 64;
    const int CP = (int)((cg + 15) / 16 * 16);
    CUtensorMap mG;
    cuuint64_t gdim[2] = {(cuuint64_t)ldq, (cuuint64_t)(c - g0)};
    cuuint64_t gstride[1] = {(cuuint64_t)ldq * 2};
    cuuint32_t box[2] = {kGRows, (cuuint32_t)CP};
    cuuint32_t es[2] = {1, 1};
    if (enc(&mG, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)(f.Gq + g0 * ldq), gdim, gstride, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
    a.c = (int)cg;
    a.row0 = g0;
    switch (CP) {
      case 16: e = launch_fx<16>(env, mA, mG, a, grid); break;
      case 32: e = launch_fx<32>(env, mA, mG, a, grid); break;
      case 48: e = launch_fx<48>(env, mA, mG, a, grid); break;
      default: e = launch_fx<64>(env, mA, mG, a, grid); break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_sketch_fx_reduce(const LaunchEnv& env, int64_t c, const double* A, int64_t lda,
                                    int64_t m, int64_t n, void* scratch, double* Y,
                                    double* sumsq_part, int64_t* nparts) {
  if (!fx_args_ok(c, A, lda, m, n)) return cudaErrorInvalidValue;
  const FxScratch f = carve_fx(scratch, c, m, n);
  const dim3 rgrid((unsigned)((n + 255) / 256), (unsigned)((c + kReduceRows - 1) / kReduceRows));
  fx_reduce_kernel<<<rgrid, 256, 0, env.stream>>>(f.acc_lo, f.acc_hi, c, n, f.cexp, Y, sumsq_part);
  *nparts = (int64_t)rgrid.x * rgrid.y;
  return cudaGetLastError();
}

}  // namespace cur
