// rng.cu -- the Gaussian sketching matrix G of Algorithm 1 (arXiv 2509.21963,
// "Generate a sketch matrix", N(0,1) entries per Sec. 3.2.1), drawn on the
// device from a counter-based generator so that G never has to be stored on
// the host.  Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by the
// seed; Box-Muller (1958) turns pairs of 53-bit uniforms into normals.
#include "cur_internal.cuh"
#include "rng.cuh"

namespace cur {
namespace {

// One thread per Philox block: four consecutive entries of row i.
__global__ void gaussian_kernel(uint64_t seed, int64_t c, int64_t m, int64_t blocks_per_row,
                                double* __restrict__ G, int64_t ldg) {
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= c * blocks_per_row) return;
  int64_t i = gid / blocks_per_row, q = gid - i * blocks_per_row;
  double z[4];
  gaussian_block(seed, i, q, z);
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
