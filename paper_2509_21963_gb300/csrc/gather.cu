// gather.cu -- index gathers of IterativeCUR (arXiv 2509.21963): C_k = A(:,J_k)
// and R_k = A(I_k,:) (Algorithm 1's column residual), the residual entries
// S(:,J_k), S(I_k,:), N_k = S(I_k,J_k) of Lemma 1, and the core A(I,J).
//
// One kernel covers every case: out[a, t] = X(r(a), c(t)) with optional row /
// column index lists and an optional transpose, converting FP32 sources to
// FP64.  The thread layout keeps the source reads coalesced whenever the
// source's fast axis is the gathered output's fast axis: rows of A (R_k) are
// contiguous 128-bit-friendly runs; column gathers of a row-major A touch one
// 32-byte sector per element, which is the minimum for that layout.
#include "cur_internal.cuh"

namespace cur {
namespace {

template <bool F32>
__global__ void gather2d_kernel(const void* __restrict__ X, int64_t ldx, bool trans,
                                const int64_t* __restrict__ ridx, const int64_t* __restrict__ cidx,
                                int64_t rows, int64_t cols, int64_t rlim, int64_t clim,
                                double* __restrict__ out, int64_t ldo) {
  // x: the output's fast axis (t), y: the output's rows (a); grid-stride both.
  for (int64_t a = blockIdx.y; a < rows; a += gridDim.y) {
    int64_t r = ridx ? ridx[a] : a;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cols;
         t += (int64_t)gridDim.x * blockDim.x) {
      int64_t c = cidx ? cidx[t] : t;
      if (r < 0 || r >= rlim || c < 0 || c >= clim) {  // never read outside the source
        out[a * ldo + t] = 0.0;
        continue;
      }
      int64_t off = trans ? c * ldx + r : r * ldx + c;
      double v = F32 ? (double)static_cast<const float*>(X)[off]
                     : static_cast<const double*>(X)[off];
      out[a * ldo + t] = v;
    }
  }
}

}  // namespace

cudaError_t launch_gather2d(const LaunchEnv& env, const void* X, bool x_is_f32, int64_t ldx,
                            bool trans, const int64_t* ridx, const int64_t* cidx,
                            int64_t rows, int64_t cols, int64_t rlim, int64_t clim,
                            double* out, int64_t ldo) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  int threads = 256;
  int64_t gx = (cols + threads - 1) / threads;
  if (gx > 1024) gx = 1024;
  int64_t gy = rows < 65535 ? rows : 65535;
  dim3 grid((unsigned)gx, (unsigned)gy);
  if (x_is_f32)
    gather2d_kernel<true><<<grid, threads, 0, env.stream>>>(X, ldx, trans, ridx, cidx, rows, cols, rlim, clim, out, ldo);
  else
    gather2d_kernel<false><<<grid, threads, 0, env.stream>>>(X, ldx, trans, ridx, cidx, rows, cols, rlim, clim, out, ldo);
  return cudaGetLastError();
}

}  // namespace cur
