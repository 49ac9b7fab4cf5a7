/*
 * cur_steps.h -- the individual steps of IterativeCUR (arXiv 2509.21963,
 * Algorithm 1) as C-ABI entry points on device buffers.  cur_run() chains the
 * same kernels; these calls exist so that each step can be checked and timed
 * on its own.  Same conventions as cur.h: row-major, 0-based int64 indices,
 * cur_status return codes, work enqueued on the context's stream.  All
 * pointers are device pointers unless named *_host.  Buffers are
 * caller-owned; the library keeps scratch inside the context.
 */
#ifndef CUR_STEPS_H
#define CUR_STEPS_H

#include "cur.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Gaussian sketching matrix G (c x m, FP64), Algorithm 1 "Generate a sketch
 * matrix" with N(0,1) entries (Sec. 3.2.1).  Definition (shared with nothing
 * but this comment):
 *   x = Philox4x64-10(counter = {q, i, 0, 0}, key = {seed, 0x43555200})
 *   u_t = ((x_t >> 11) + 0.5) 2^-53,  t = 0..3
 *   G[i,4q+0..1] = sqrt(-2 ln u_0) (cos, sin)(2 pi u_1)
 *   G[i,4q+2..3] = sqrt(-2 ln u_2) (cos, sin)(2 pi u_3)
 * G has row stride m.  Errors: CUR_EINVAL if c < 1 or m < 1. */
int cur_step_gaussian(cur_ctx *ctx, uint64_t seed, int64_t c, int64_t m, double *G);

/* Initial sketch S_0^col = Y = G A (Algorithm 1) in FP64 arithmetic.
 *   G  c x m FP64 (stride m); A m x n (stride lda, dtype FP64 or FP32);
 *   Y  c x n FP64 output (stride n);
 *   sumsq_host (may be NULL) receives ||Y||_F^2 (synchronises the stream). */
int cur_step_sketch(cur_ctx *ctx, const double *G, int64_t c, const void *A,
                    int64_t m, int64_t n, int64_t lda, int dtype, double *Y,
                    double *sumsq_host);

/* Precision form of the initial sketch on the tensor cores (see
 * cur_sketch_mode in cur.h): Y = G_q fix_S(A) exactly, with
 * G_q = clamp(rint(16 G), -127, 127) and S = digits in 1..4.
 *   G c x m FP64 (stride m); A m x n FP32 (stride lda, lda % 4 == 0, base
 *   16-byte aligned); Y c x n FP64; sumsq_host (may be NULL) receives ||Y||_F^2.
 *   Inf/NaN in a column of A turns that column of Y into NaN.
 * CUR_EINVAL for unsupported c / S / alignment. */
int cur_step_sketch_q(cur_ctx *ctx, const double *G, int64_t c, const float *A, int64_t m,
                      int64_t n, int64_t lda, int digits, double *Y, double *sumsq_host);

/* FP64 form of the initial sketch S_0^col = Y = G A (Algorithm 1) on the
 * tensor cores.  Sec. 3.4 counts this pass among the method's primary costs.
 * GB300's FP64 pipe cannot run it at the HBM rate; this form makes every
 * product exact on BF16 tensor cores instead:
 *   G_q = clamp(rint(16 G), -127, 127)   (8-bit integers; G c x m FP64, stride m)
 *   E_j: max_k |A(k,j)| < 2^E_j          (frexp of the column max, 0 for a zero column)
 *   X(k,j) = trunc(A(k,j) 2^(52-E_j))    (52-bit fixed point, |X| < 2^52)
 *   Y(i,j) = RN(sum_k G_q(i,k) X(k,j)) 2^(E_j-52)   (the integer sum exact,
 *                                        rounded once to nearest-even)
 * so |Y - G_q A| <= 2^(E_j-52) sum_k |G_q(i,k)| + ulp(Y)/2.
 *   A  m x n FP64, row stride lda (lda % 2 == 0), base 16-byte aligned;
 *   Y  c x n FP64 output (stride n), any c >= 1 (one pass of A per 64 rows of G);
 *   sumsq_host (may be NULL) receives ||Y||_F^2 (synchronises the stream).
 *   A column holding Inf or NaN turns that column of Y into NaN.
 * CUR_EINVAL for bad sizes, odd lda or a misaligned A. */
int cur_step_sketch_fx(cur_ctx *ctx, const double *G, int64_t c, const double *A, int64_t m,
                       int64_t n, int64_t lda, double *Y, double *sumsq_host);

/* D = alpha op(A) op(B) + beta C in FP64 (op = transpose when trans* != 0):
 * the products of the residual updates of Algorithm 1 in the Lemma 1 form,
 * S^row = A(:,J_k) - C U R(:,J_k) and S^col <- S^col - S^col(:,J_k) N^+ R_k
 * (Sec. 3.2).  D is M x N (stride ldd); op(A) is M x K (A stored K x M when
 * transA, stride lda); op(B) is K x N (B stored N x K when transB, stride
 * ldb); C (stride ldc) is read only when beta != 0 and may alias D.  All
 * pointers are device memory owned by the caller.  sumsq_host (may be NULL)
 * receives ||D||_F^2, summed in a fixed order (synchronises the stream): the
 * stopping test's norm.  CUR_EINVAL for negative sizes or short strides. */
int cur_step_gemm(cur_ctx *ctx, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
                  int64_t lda, int transA, const double *B, int64_t ldb, int transB, double beta,
                  const double *C, int64_t ldc, double *D, int64_t ldd, double *sumsq_host);

/* Index gather of Algorithm 1 (C = A(:,J), R = A(I,:), A(I,J), S(:,J_k)):
 * out[a * ldo + t] = X(r, c) with r = ridx ? ridx[a] : a and
 * c = cidx ? cidx[t] : t, where X(r, c) = X[r * ldx + c] (trans == 0) or
 * X[c * ldx + r] (trans != 0, the transposed gather); an index outside
 * [0, rlim) x [0, clim) writes 0.0 (so a rank that does not own an index
 * contributes zero to a sum over ranks).  out is rows x cols; X FP64; all
 * pointers device memory owned by the caller; asynchronous on the context's
 * stream.  CUR_EINVAL for negative sizes or short strides. */
int cur_step_gather(cur_ctx *ctx, const double *X, int64_t ldx, int trans, const int64_t *ridx,
                    const int64_t *cidx, int64_t rows, int64_t cols, int64_t rlim, int64_t clim,
                    double *out, int64_t ldo);

/* The residual product of cur_opts.residual_planes on its own:
 * D(n, i) -= sum_{k<K} P(i, k) Q(n, k) for n < N, i < M, with P (M x K, row
 * pitch ldp) and Q (N x K, pitch ldq) FP64, split into `planes` (2 or 3) BF16
 * planes and multiplied on the tensor cores with FP32 accumulation (the
 * products S^row = A(:,J_k) - L Rt(:,J_k) and R_k = A(I_k,:) - L(I_k,:) Rt of
 * Sec. 4.2 in this form).  D is N x M FP64 with pitch ldd.  All pointers are
 * device memory owned by the caller.  1 <= N <= 128.  CUR_EINVAL for bad sizes
 * or strides.  Synchronises the stream. */
int cur_step_resid_tc(cur_ctx *ctx, const double *P, int64_t ldp, const double *Q, int64_t ldq,
                      int64_t M, int64_t N, int64_t K, int planes, double *D, int64_t ldd);

/* LUPP index selection (Sec. 3.2.1, 3.2.2): the candidates are the ncand
 * columns of X (nr x ncand, stride ldx, FP64; read only).  Step t picks the
 * eligible candidate with the largest |W[t, i]| of the running Schur
 * complement (ties: smallest index; an all-zero row picks the smallest eligible
 * index and eliminates nothing) and eliminates every other eligible candidate
 * against it.  mask (ncand bytes, non-zero = not eligible) is updated with the
 * picks.  piv receives `steps` indices.  Requires steps <= nr and at least
 * `steps` eligible candidates (else CUR_EINVAL). */
int cur_step_lupp(cur_ctx *ctx, const double *X, int64_t ldx, int64_t nr,
                  int64_t ncand, int64_t steps, uint8_t *mask, int64_t *piv);

/* Generalised inverse X = M^+ (q x p, stride p) of M (p x q, stride ldm) by
 * Householder QR with column pivoting (Businger-Golub): M P = Q R,
 * k = #{|R_ii| > thr}, X = P [R_11^{-1} Q_1^T; 0].  This is the core solve
 * U = A(I,J)^+ of Algorithm 1 (the paper's default QR).  thr < 0 selects
 * thr = max(p,q) 2^-52 |R_00|.  rank_host (may be NULL) receives k
 * (synchronises the stream).  The kernels are those cur_run uses for a core
 * of this size: one CTA (p < 24), one thread-block cluster (24 <= p <= 512,
 * q <= 16 columns per CTA of the cluster), a cooperative grid holding M in
 * shared memory, or (square M too large for that, p <= 10240) the whole-GPU
 * team QR with a shared-memory solve panel.  When every remaining column norm
 * of a step is NaN the shared-memory variants return CUR_EINVAL; the team QR
 * carries the NaN through (its rank then counts no such column). */
int cur_step_pinv(cur_ctx *ctx, const double *M, int64_t p, int64_t q,
                  int64_t ldm, double thr, double *X, int64_t *rank_host);

/* cur_step_lupp without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc (code running
 * inside another framework's memory pool, allocation-free real-time loops,
 * allocators that must not be re-entered).  It needs no context: `device`
 * selects the GPU (made current by the call) and `cuda_stream` the stream
 * (NULL = legacy default stream).  X, mask and piv are as for cur_step_lupp
 * and stay caller-owned.
 *   Scratch: a fixed 16 MiB device array inside the library (held by every GPU
 *   that loads the library until the process exits) that must hold
 *   nr * ncand + 2 * G * max(nr + 2, 34) doubles plus 256 bytes, G <= the SM count
 *   (e.g. 55 x 20000 fits); larger problems return CUR_EINVAL with a
 *   message in err that states the bytes needed.  Device errors map as for
 *   cur_step_lupp: a timed-out barrier CUR_ETIMEOUT, too few eligible
 *   candidates CUR_EINVAL, any other device status CUR_ECUDA with its code in
 *   err.  The call allocates nothing (no cudaMalloc,
 *   cudaFree or allocating library routine).
 *   Set-up: the first call on a device resolves the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Concurrency: all calls share the one array, so calls that overlap on the
 *   GPU (different streams, threads or processes' streams on the same device)
 *   race; serialise them.  The call synchronises `cuda_stream`.
 *   err/err_len (may be NULL/0) receive a one-line message ("" on success). */
int cur_step_lupp_noalloc(int device, void *cuda_stream, const double *X, int64_t ldx,
                          int64_t nr, int64_t ncand, int64_t steps, uint8_t *mask,
                          int64_t *piv, char *err, size_t err_len);

/* Test hook for the failure path of the library's bounded device waits (the
 * paper has no counterpart): launches a kernel whose wait cannot complete and
 * gives up after budget_ms (0 < budget_ms <= 5000, converted to cycles at the
 * device's clock rate).  which = 0: `nblocks` CTAs (1 <= nblocks <= SM count)
 * arrive at the software grid barrier expecting nblocks + 1; which = 1: one
 * CTA waits on an mbarrier phase that gets one of its two arrivals.  The wait
 * records the timeout in the context's status word and the kernel returns,
 * so the call returns CUR_ETIMEOUT and the context stays usable.  Nothing
 * faults or waits without a limit.  Synchronises the context's stream. */
int cur_test_wait_timeout(cur_ctx *ctx, int which, int nblocks, double budget_ms);

/* Measured FP64 FMA rate of the context's device in TFLOP/s (*tflops): five
 * timed launches of independent FMA chains over all SMs.  The paper has no
 * counterpart; it is the denominator of the FP64-pipe roofline figures.  It
 * allocates 8 bytes of device memory for the duration of the call and
 * synchronises the context's stream. */
int cur_probe_fp64_tflops(cur_ctx *ctx, double *tflops);

/* Latency of dependent operations on the context's device, in SM cycles per
 * operation (one warp, a chain of 256), into cycles[0 .. n-1] in this order:
 * FP64 FMA, FP64 FMA with one active lane, FP64 add, FP64 shuffle + add,
 * FP64 divide, FP64 square root (+ add), FP64 compare-and-select, FP32 FMA,
 * 64-bit integer shuffle + max, dependent L2 load; entries past the tenth are
 * 0.  The paper has no counterpart: these figures decide which operations the
 * latency-bound steps (LUPP, the small QR) keep off their critical paths.
 * Allocates 33 KB of device memory for the call; synchronises the stream. */
int cur_probe_latency(cur_ctx *ctx, double *cycles, int n);

#ifdef __cplusplus
}
#endif
#endif /* CUR_STEPS_H */
