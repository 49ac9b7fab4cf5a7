// rng.cuh -- device side of the Gaussian sketching matrix G of Algorithm 1
// (arXiv 2509.21963, N(0,1) entries per Sec. 3.2.1), shared by the kernels
// that draw G.  Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by
// {seed, 0x43555200}, counter {q, i, 0, 0} for the four entries 4q..4q+3 of
// row i; Box-Muller (1958) turns pairs of 53-bit uniforms into normals.
#pragma once

#include <stdint.h>

namespace cur {

__device__ __forceinline__ void philox_round(uint64_t x[4], uint64_t k0, uint64_t k1) {
  const uint64_t m0 = 0xD2E7470EE14C6C93ULL, m1 = 0xCA5A826395121157ULL;
  uint64_t hi0 = __umul64hi(m0, x[0]), lo0 = m0 * x[0];
  uint64_t hi1 = __umul64hi(m1, x[2]), lo1 = m1 * x[2];
  uint64_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
  x[0] = y0; x[1] = lo1; x[2] = y2; x[3] = lo0;
}

__device__ __forceinline__ void philox4x64_10(uint64_t x[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B97F4A7C15ULL; k1 += 0xBB67AE8584CAA73BULL; }
    philox_round(x, k0, k1);
  }
}

__device__ __forceinline__ double open01(uint64_t x) {
  // 53 random bits, offset by half a step: in (0, 1), exact in FP64.
  return __dmul_rn(__dadd_rn((double)(x >> 11), 0.5), 0x1.0p-53);
}

// The four normals G[i][4q .. 4q+3] of the sketch with this seed.
__device__ __forceinline__ void gaussian_block(uint64_t seed, int64_t i, int64_t q, double z[4]) {
  const double two_pi = 6.283185307179586476925286766559;
  uint64_t x[4] = {(uint64_t)q, (uint64_t)i, 0ULL, 0ULL};
  philox4x64_10(x, seed, 0x43555200ULL);
  double u0 = open01(x[0]), u1 = open01(x[1]), u2 = open01(x[2]), u3 = open01(x[3]);
  double r01 = sqrt(__dmul_rn(-2.0, log(u0)));
  double r23 = sqrt(__dmul_rn(-2.0, log(u2)));
  double s1, c1, s3, c3;
  sincos(__dmul_rn(two_pi, u1), &s1, &c1);
  sincos(__dmul_rn(two_pi, u3), &s3, &c3);
  z[0] = __dmul_rn(r01, c1); z[1] = __dmul_rn(r01, s1);
  z[2] = __dmul_rn(r23, c3); z[3] = __dmul_rn(r23, s3);
}

}  // namespace cur
