// rng.cu -- the Gaussian sketching matrix G of Algorithm 1 (arXiv 2509.21963,
// "Generate a sketch matrix", N(0,1) entries per Sec. 3.2.1), drawn on the
// device from a counter-based generator so that G never has to be stored on
// the host.  Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by the
// seed; Box-Muller (1958) turns pairs of 53-bit uniforms into normals.
#include "cur_internal.cuh"

namespace cur {
namespace {

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

// One thread per Philox block: four consecutive entries of row i.
__global__ void gaussian_kernel(uint64_t seed, int64_t c, int64_t m, int64_t blocks_per_row,
                                double* __restrict__ G, int64_t ldg) {
  const double two_pi = 6.283185307179586476925286766559;
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= c * blocks_per_row) return;
  int64_t i = gid / blocks_per_row, q = gid - i * blocks_per_row;
  uint64_t x[4] = {(uint64_t)q, (uint64_t)i, 0ULL, 0ULL};
  philox4x64_10(x, seed, 0x43555200ULL);
  double u0 = open01(x[0]), u1 = open01(x[1]), u2 = open01(x[2]), u3 = open01(x[3]);
  double r01 = sqrt(__dmul_rn(-2.0, log(u0)));
  double r23 = sqrt(__dmul_rn(-2.0, log(u2)));
  double s1, c1, s3, c3;
  sincos(__dmul_rn(two_pi, u1), &s1, &c1);
  sincos(__dmul_rn(two_pi, u3), &s3, &c3);
  double z[4] = {__dmul_rn(r01, c1), __dmul_rn(r01, s1), __dmul_rn(r23, c3), __dmul_rn(r23, s3)};
  double* row = G + i * ldg;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    int64_t k = 4 * q + t;
    if (k < m) row[k] = z[t];
  }
}

}  // namespace

cudaError_t launch_gaussian(const LaunchEnv& env, uint64_t seed, int64_t c, int64_t m,
                            double* G, int64_t ldg) {
  int64_t bpr = (m + 3) / 4;
  int64_t total = c * bpr;
  if (total == 0) return cudaSuccess;
  int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  gaussian_kernel<<<(unsigned)blocks, threads, 0, env.stream>>>(seed, c, m, bpr, G, ldg);
  return cudaGetLastError();
}

}  // namespace cur
