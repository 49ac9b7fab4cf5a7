// cur_internal.cuh -- declarations shared by the CUDA translation units of the
// IterativeCUR library (arXiv 2509.21963).  Each kernel file exposes host-side
// launch functions; the orchestrator (cur_api.cu) chains them on one stream.
#pragma once

#include <cuda_bf16.h>

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

namespace cur {

// Error codes written by kernels into a device status word (never __trap()).
enum DevErr : int {
  kDevOk = 0,
  kDevTimeout = 1,      // a grid barrier waited past its cycle budget
  kDevNoCandidate = 2,  // LUPP ran out of eligible candidates
};

// Device-side status block: kernels set `err` with atomicCAS(0 -> code).
struct DevStatus {
  int err;
  int pad;
  double scalar[6];  // [0] sumsq of Y, [1] sumsq of S, [2] pinv rank-scale, ...
};

// Bounded software barrier for co-resident CTAs (cooperative launches, software
// teams): one 64-bit arrival counter that only grows (gridbar.cuh).  Zeroed
// before a launch; a completed barrier leaves it at a multiple of its CTA count.
struct alignas(8) GridBar {
  unsigned long long count;
};

// Cycle budget of one barrier wait (~2 s at 2 GHz): far above any legitimate
// wait, short enough that a lost block surfaces as CUR_ETIMEOUT.
constexpr long long kBarrierBudget = 4000000000LL;

struct LaunchEnv {
  cudaStream_t stream;
  int num_sms;
  int device;
};

// Opt a kernel in to `need` bytes of dynamic shared memory.  The ceiling is a
// process-wide attribute of the kernel, so it is only ever set to one value
// (all the opt-in shared memory the kernel's static part leaves): host threads
// launching the kernel at once with different sizes never see another thread
// lower it between its own set and launch.  It is set once per kernel and
// device, then remembered.  cudaErrorInvalidValue if `need` exceeds it.
inline cudaError_t smem_opt_in(const void* fn, size_t need) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> caps;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  auto it = caps.find({fn, dev});
  if (it == caps.end()) {
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    const int cap = optin - (int)fa.sharedSizeBytes;
    if (cap < 0) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e != cudaSuccess) return e;
    it = caps.emplace(std::make_pair(fn, dev), cap).first;
  }
  return need > (size_t)it->second ? cudaErrorInvalidValue : cudaSuccess;
}

// ---- rng.cu ---------------------------------------------------------------
cudaError_t launch_gaussian(const LaunchEnv& env, uint64_t seed, int64_t c, int64_t m,
                            double* G, int64_t ldg);

// ---- gemm.cu --------------------------------------------------------------
// D = alpha * op(A) op(B) + beta * Cin (row-major; op(X) = X or X^T).
// A is FP64; B is FP64 or FP32 (b_is_f32).  Cin may alias D.  If sumsq_part
// is non-null, each CTA writes the sum of squares of its D tile into
// sumsq_part[cta] and the number of CTAs into *nparts.  ksplit > 1 splits the
// K range across gridDim.z, accumulating partial tiles in `partial`
// (ksplit * M * N doubles) and finishing in a reduction kernel.
struct GemmArgs {
  int64_t M, N, K;
  double alpha;
  const double* A; int64_t lda; bool transA;
  const void* B; int64_t ldb; bool transB; bool b_is_f32;
  double beta;
  const double* Cin; int64_t ldcin;
  double* D; int64_t ldd;
  double* sumsq_part;   // optional
  double* partial;      // required when ksplit > 1
  int ksplit;
};
// Returns the number of sum-of-squares partials written (0 if none).
int64_t gemm_num_sumsq_parts(const GemmArgs& g);
cudaError_t launch_gemm(const LaunchEnv& env, const GemmArgs& g);
// out[0] = sum of parts[0..n) in a fixed order (one CTA).
cudaError_t launch_sum_parts(const LaunchEnv& env, const double* parts, int64_t n, double* out);

// ---- sketch_simt.cu --------------------------------------------------------
// Y = G A (c x n) in FP64 on the SIMT FP64 pipe, K split into ks balanced work
// units (partial buffer of ks * c * n doubles when ks > 1), fixed-order reduce.
struct SketchPlan {
  int64_t kunit = 0;          // rows of A per work unit
  int ks = 1;                 // number of work units along K
  size_t partial_doubles = 0; // scratch for the K split
  int64_t sumsq_parts = 0;    // number of sum-of-squares partials written
};
SketchPlan plan_sketch_simt(const LaunchEnv& env, int64_t c, int64_t m, int64_t n);
cudaError_t launch_sketch_simt(const LaunchEnv& env, const SketchPlan& p, const double* G,
                               int64_t ldg, int64_t c, const void* A, bool a_f32, int64_t lda,
                               int64_t m, int64_t n, double* Y, double* partial,
                               double* sumsq_part);
// Row-block form (for a sketch that overlaps the host-to-device copy of A):
// the plan's ks slices of G(:, rows) A(rows, :) into `slices`, unreduced;
// then Y = the fixed-order sum of all nslices slices, with sketch_reduce_parts
// sum-of-squares partials.
cudaError_t launch_sketch_simt_slices(const LaunchEnv& env, const SketchPlan& p, const double* G,
                                      int64_t ldg, int64_t c, const void* A, bool a_f32,
                                      int64_t lda, int64_t m, int64_t n, double* slices);
int64_t sketch_reduce_parts(int64_t c, int64_t n);
cudaError_t launch_sketch_reduce(const LaunchEnv& env, const double* slices, int nslices,
                                 int64_t c, int64_t n, double* Y, double* sumsq_part);

// ---- sketch_tc.cu ------------------------------------------------------------
// Precision form of Y = G A on tcgen05 (BF16 digit slices, exact FP32/int64
// accumulation): Y = G_q fix_S(A), G_q = clamp(rint(16 G), +-127), S in 1..4.
// A is FP32 with lda % 4 == 0 and a 16-byte aligned base.  Scratch layout is
// owned by the launch (sketch_tc_scratch_bytes).  c_pad = sketch_tc_cpad(c, S)
// must be > 0.  Writes *nparts sum-of-squares partials into sumsq_part.
int sketch_tc_cpad(int c, int S);
int sketch_tc_plan_ks(const LaunchEnv& env, int64_t m, int64_t n);
size_t sketch_tc_scratch_bytes(int64_t c, int64_t m, int64_t n, int ks);
cudaError_t launch_sketch_tc(const LaunchEnv& env, int S, const double* G, int64_t c,
                             const float* A, int64_t lda, int64_t m, int64_t n, void* scratch,
                             int ks, double* Y, double* sumsq_part, int64_t* nparts, int* err);

// G_q = clamp(rint(16 G), +-127) as BF16 (c x ldq, columns m..ldq-1 zero):
// the 8-bit sketch of both tensor-core forms.
cudaError_t launch_gaussian_q8(const LaunchEnv& env, const double* G, int64_t c, int64_t m,
                               int64_t ldq, uint16_t* Gq);

// ---- sketch_fx.cu ------------------------------------------------------------
// FP64 form of Y = G A on tcgen05: Y = RN(G_q trunc(A 2^(52-E_j))) 2^(E_j-52)
// with the integer sum exact (six balanced base-512 BF16 digits per entry,
// exact FP32 chunk sums, int64 combination).  A is FP64 with lda % 2 == 0 and a
// 16-byte aligned base.  Any c >= 1 (row groups of 64 rows of G, one pass of A
// each).  A column holding Inf/NaN gives NaN in Y (and so in the sum of
// squares).  Writes *nparts sum-of-squares partials into sumsq_part.
// Two launches on the same scratch: the scales (G_q, column exponents, zeroed
// sums), then the tensor-core pass and the reduction into Y.
size_t sketch_fx_scratch_bytes(int64_t c, int64_t m, int64_t n);
int64_t sketch_fx_max_parts(int64_t c, int64_t n);
cudaError_t launch_sketch_fx_scales(const LaunchEnv& env, const double* G, int64_t c,
                                    const double* A, int64_t lda, int64_t m, int64_t n,
                                    void* scratch);
// The two halves of launch_sketch_fx_scales, for running them on two streams:
// G_q from G, and the column exponents of A (with the zeroing of the sums).
cudaError_t launch_sketch_fx_q8(const LaunchEnv& env, const double* G, int64_t c, int64_t m,
                                int64_t n, void* scratch);
cudaError_t launch_sketch_fx_colscales(const LaunchEnv& env, int64_t c, const double* A,
                                       int64_t lda, int64_t m, int64_t n, void* scratch);
// The FP64 tensor-core sketch in pieces: zero the column maxima and the sums;
// column scales of columns [c0, c1); the tensor-core pass over those columns
// (c0 even); the final reduction.
cudaError_t launch_sketch_fx_zero(const LaunchEnv& env, int64_t c, const double* A, int64_t lda,
                                  int64_t m, int64_t n, void* scratch);
cudaError_t launch_sketch_fx_colscales_range(const LaunchEnv& env, int64_t c, const double* A,
                                             int64_t lda, int64_t m, int64_t n, void* scratch,
                                             int64_t c0, int64_t c1);
// The column scales in finer pieces: the maxima of rows [r0, r1) of columns
// [c0, c1) (atomic maxima into the zeroed column maxima), then E_j of columns
// [c0, c1) once all their rows are in.
cudaError_t launch_sketch_fx_colmax_block(const LaunchEnv& env, int64_t c, const double* A,
                                          int64_t lda, int64_t m, int64_t n, void* scratch,
                                          int64_t r0, int64_t r1, int64_t c0, int64_t c1);
cudaError_t launch_sketch_fx_colexp_range(const LaunchEnv& env, int64_t c, const double* A,
                                          int64_t lda, int64_t m, int64_t n, void* scratch,
                                          int64_t c0, int64_t c1);
cudaError_t launch_sketch_fx_main_range(const LaunchEnv& env, int64_t c, const double* A,
                                        int64_t lda, int64_t m, int64_t n, void* scratch,
                                        int64_t c0, int64_t c1, int* err);
cudaError_t launch_sketch_fx_reduce(const LaunchEnv& env, int64_t c, const double* A, int64_t lda,
                                    int64_t m, int64_t n, void* scratch, double* Y,
                                    double* sumsq_part, int64_t* nparts);
cudaError_t launch_sketch_fx_main(const LaunchEnv& env, int64_t c, const double* A, int64_t lda,
                                  int64_t m, int64_t n, void* scratch, double* Y,
                                  double* sumsq_part, int64_t* nparts, int* err);

// ---- faultcheck.cu -----------------------------------------------------------
// Drive a bounded device wait past `budget` cycles on purpose (which 0: the
// grid barrier, `nblocks` CTAs expecting one more; 1: an mbarrier wait); the
// wait records kDevTimeout in *st and the kernel returns.
cudaError_t launch_timeout_check(const LaunchEnv& env, int which, int nblocks, long long budget,
                                 GridBar* bar, DevStatus* st);

// ---- gather.cu ------------------------------------------------------------
// out[a * ldo + t] = src(r(a), c(t)) for a < rows, t < cols, where
// r(a) = ridx ? ridx[a] : a, c(t) = cidx ? cidx[t] : t and src(i, j) =
// X[i * ldx + j] (or X[j * ldx + i] if trans).  X is FP64 or FP32.  Index
// pairs outside [0, rlim) x [0, clim) are not read (out = 0).
cudaError_t launch_gather2d(const LaunchEnv& env, const void* X, bool x_is_f32, int64_t ldx,
                            bool trans, const int64_t* ridx, const int64_t* cidx,
                            int64_t rows, int64_t cols, int64_t rlim, int64_t clim,
                            double* out, int64_t ldo);

// ---- resid_tc.cu ------------------------------------------------------------
// Residual products on the tensor cores: D(n, i) -= sum_{k<K} P(i, k) Q(n, k)
// with P (M x K) and Q (N x K, N <= 128) held as np = 2 or 3 BF16 planes,
// K-major with pitches ldp, ldq (multiples of 64).
int64_t resid_plane_pitch(int64_t kmax);
// ||X||_F^2 of a rows x cols FP64 matrix as resid_sumsq_parts() per-CTA partial
// sums (fixed order; reduce with launch_sum_parts).
int64_t resid_sumsq_parts();
cudaError_t launch_sumsq_parts(const LaunchEnv& env, const double* X, int64_t rows, int64_t cols,
                               int64_t ld, double* parts);
cudaError_t launch_split_planes(const LaunchEnv& env, const double* src, int64_t st, int64_t si,
                                int64_t nt, int64_t M, __nv_bfloat16* const* planes, int np,
                                int64_t ldp, int64_t k0, bool negate = false);
cudaError_t launch_gather_plane_rows(const LaunchEnv& env, __nv_bfloat16* const* planes, int np,
                                     int64_t ldp, int64_t prows, const int64_t* idx, int N,
                                     int64_t kp, __nv_bfloat16* const* dst, int64_t ldq);
cudaError_t launch_resid_tc(const LaunchEnv& env, int np, __nv_bfloat16* const* P, int64_t ldp,
                            int64_t M, __nv_bfloat16* const* Q, int64_t ldq, int N, int64_t K,
                            double* D, int64_t ldd, int* err);

// ---- lupp.cu --------------------------------------------------------------
struct LuppWork {
  double* W;          // nr * ncand working copy
  double* slot_val;   // 2 * max_grid * lupp_slot_stride(nr)
  GridBar* bar;
  int max_grid;
};
size_t lupp_work_doubles(int64_t nr, int64_t ncand, int max_grid);
// Feature panel of the blocked selector; doubles per CTA and step parity in
// LuppWork::slot_val (2 * max_grid of them): the unblocked record (|value|,
// index, nr column values) or the blocked one (|value|, index, panel column,
// multipliers).
constexpr int kLuppPanel = 16;
__host__ __device__ inline int64_t lupp_slot_stride(int64_t nr) {
  return nr + 2 > 2 + 2 * kLuppPanel ? nr + 2 : 2 + 2 * kLuppPanel;
}
// The selector's barrier word is followed by its exchange words: 128 bytes
// from LuppWork::bar, all cleared by launch_lupp.
constexpr size_t kLuppBarBytes = 128;
__host__ __device__ inline unsigned long long* lupp_xchg(GridBar* bar) {
  return reinterpret_cast<unsigned long long*>(bar) + 8;
}
int lupp_grid(const LaunchEnv& env, int64_t nr, int64_t ncand);
cudaError_t launch_lupp(const LaunchEnv& env, const double* X, int64_t ldx, int64_t nr,
                        int64_t ncand, int64_t steps, uint8_t* mask, int64_t* piv,
                        const LuppWork& w, int grid, DevStatus* st);

// ---- qrcp.cu --------------------------------------------------------------
struct QrcpWork {
  double* Rc;       // q * p   (column-major copy of M: Rc[col * p + i])
  double* V;        // kmax * p Householder vectors
  double* tau;      // kmax
  double* rdiag;    // kmax
  int64_t* perm;    // q
  uint8_t* used;    // q
  double* slots;    // 2 * max_grid * 2
  GridBar* bar;
  int64_t* rank;    // 1 (device)
  double* Ysolve;   // p * p solve scratch
  int max_grid;
};
size_t qrcp_work_bytes(int64_t p, int64_t q, int max_grid);
void qrcp_carve(void* base, int64_t p, int64_t q, int max_grid, QrcpWork* w);
int qrcp_grid(const LaunchEnv& env, int64_t p, int64_t q);
// True when the factorisation keeps M in shared memory (one CTA, or each CTA of
// the cooperative grid holding its columns); false: the global-memory kernel.
bool qrcp_resident(const LaunchEnv& env, int64_t p, int64_t q);
// thr_mode: 0 relative (max(p,q) 2^-52 |R_00|); 1 absolute `thr`; 2 absolute
// thr * (*scale_dev), where *scale_dev (if *scale_dev < 0) is first set to
// 2^-52 |R_00| of this factorisation.
cudaError_t launch_qrcp_pinv(const LaunchEnv& env, const double* M, int64_t p, int64_t q,
                             int64_t ldm, int thr_mode, double thr, double* scale_dev,
                             double* X, int64_t ldx, const QrcpWork& w, int grid,
                             DevStatus* st);

}  // namespace cur
