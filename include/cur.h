/*
 * cur.h -- C ABI of the GB300 (sm_103a) IterativeCUR library.
 *
 * IterativeCUR (Pritchard, Park, Nakatsukasa, Martinsson, arXiv 2509.21963,
 * Algorithm 1): given A (m x n) and a relative Frobenius tolerance eps, find
 * row indices I, column indices J and a core U = A(I,J)^+ such that
 * ||A - A(:,J) U A(I,:)||_F / ||A||_F is estimated below eps (Sec. 1.1, Sec. 3.1).
 * One Gaussian sketch Y = G A (c x n) is formed once; every iteration picks b
 * columns by LU with partial pivoting (LUPP) on the sketched residual, b rows by
 * LUPP on the residual at those columns, updates the residuals through Lemma 1
 * (Sec. 4.2) and stops when rho = ||S^col||_F / ||G A||_F <= eps (Sec. 3.3).
 *
 * Conventions for every entry point:
 *   - Matrices are row-major.  A has row stride lda >= n (elements).
 *   - "device" pointers live in the memory of the context's GPU; "host"
 *     pointers in ordinary (pageable or pinned) host memory.
 *   - Indices are 0-based (the paper is 1-based), int64.
 *   - Every call returns a cur_status; nothing aborts or throws across the
 *     ABI.  cur_last_error() holds a one-line description of the last failure.
 *   - A context is bound to one device and one CUDA stream; it is not
 *     thread-safe (use one context per host thread).  All work of a call is
 *     enqueued on that stream; calls that return results to the host
 *     synchronise it.
 */
#ifndef CUR_H
#define CUR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cur_ctx cur_ctx;       /* device, stream, workspace arena      */
typedef struct cur_result cur_result; /* outputs of one run (device + host)   */

typedef enum {
  CUR_OK = 0,
  CUR_EINVAL = 1,        /* invalid argument                                    */
  CUR_ENONFINITE = 2,    /* A contains Inf/NaN (found by the sketch pass)       */
  CUR_ENOMEM = 3,        /* device or host allocation failed                    */
  CUR_EBUDGET = 4,       /* workspace would exceed the context's HBM budget     */
  CUR_ECUDA = 5,         /* a CUDA call failed (code kept in cur_last_error)    */
  CUR_ETIMEOUT = 6,      /* a device-side wait ran out of its iteration limit   */
  CUR_TOL_UNREACHED = 7  /* stopped at max_rank with rho > eps (result valid)   */
} cur_status;

typedef enum { CUR_F64 = 0, CUR_F32 = 1 } cur_dtype;

/* Arithmetic of the sketch pass Y = G A (all later steps are FP64).
 * The precision forms run on the tensor cores (tcgen05, BF16 operands) and
 * need an FP32 A with lda % 4 == 0 and a 16-byte aligned base; they use the
 * 8-bit sketch G_q = clamp(rint(16 G), -127, 127) and the S-digit fixed point
 * of each column (digits of 8 bits relative to a power-of-two column scale
 * 2^E_j > max |A(:,j)|), and compute Y = G_q fix_S(A) exactly for S <= 3
 * (for S = 4: the exact value rounded once to FP64):
 *   |fix_S(A)(k,j) - A(k,j)| <= 2^(E_j - 8S - 1).
 * c (rounded up to 16) must be <= 128, <= 80 for S = 3 and <= 64 for S = 4. */
typedef enum {
  CUR_SKETCH_F64 = 0,   /* FP64 products and sums (the plain method)            */
  CUR_SKETCH_BF16 = 1,  /* S = 1: one BF16 digit per entry (2^-8 of column max)  */
  CUR_SKETCH_BF16X2 = 2,/* S = 2: hi + lo digits (2^-16)                         */
  CUR_SKETCH_BF16X3 = 3,/* S = 3: hi + mid + lo digits (2^-24)                   */
  CUR_SKETCH_BF16X4 = 4,/* S = 4: four digits (2^-32; exact for FP32 entries
                           within 2^-8 of their column's largest)               */
  CUR_SKETCH_F64_TC = 5 /* FP64 form on the tensor cores: FP64 A (lda % 2 == 0,
                           16-byte aligned base), the 8-bit sketch G_q above and
                           the 52-bit fixed point of each column:
                           Y = RN(G_q trunc(A 2^(52-E_j))) 2^(E_j-52), the
                           integer sum exact and rounded once to FP64, so
                           |Y - G_q A| <= 2^(E_j-52) sum_k |G_q| + ulp(Y)/2.
                           Any c.  See cur_step_sketch_fx.                      */
} cur_sketch_mode;

typedef struct cur_opts {
  int64_t max_rank;        /* 0: min(m, n).  The last block is clamped to it.   */
  const double *omega;     /* optional device G (c x m, row-major FP64), used
                              instead of the seeded Gaussian; NULL: generated.
                              The precision forms use clamp(rint(16 G), +-127). */
  int sketch_mode;         /* cur_sketch_mode                                   */
  double alpha;            /* risk-aware stopping (Sec. 3.3): 0 = off; else the
                              loop stops at eps (1+delta) sqrt(1-2 sqrt(-ln(alpha)/c))
                              and needs c > -4 ln(alpha) (CUR_EINVAL otherwise) */
  double delta;            /* see alpha                                         */
  int timing;              /* non-zero: record CUDA events around each phase
                              (cur_result_phase_ms); adds ~2 events per phase   */
  int residual_planes;     /* 0: the residual products of the loop (S^row =
                              A(:,J_k) - L Rt(:,J_k) and R_k = A(I_k,:) -
                              L(I_k,:) Rt, Sec. 4.2) in FP64.  2 or 3: on the
                              BF16 tensor cores, the factors L and Rt kept as
                              2 or 3 BF16 planes (x = x_0 + x_1 (+ x_2) + e),
                              plane pairs (a, b) with a + b < planes, FP32
                              accumulation: relative error ~2^-16 / ~2^-24 of
                              the product plus the FP32 sums; every other step
                              stays FP64.  Needs block_size <= 128.  Extra
                              device memory: planes * 2 (m + n) K bytes with
                              K = max_rank rounded up to 64.                    */
} cur_opts;

/* Phases of one run, for cur_result_phase_ms (device time, milliseconds). */
typedef enum {
  CUR_PHASE_GAUSSIAN = 0,  /* G from the seed (Algorithm 1's sketch matrix)     */
  CUR_PHASE_SKETCH = 1,    /* Y = G A and ||Y||_F: the pass over A              */
  CUR_PHASE_LUPP_COL = 2,  /* J_k, column selection                             */
  CUR_PHASE_ROW_RES = 3,   /* S^row, row residual                               */
  CUR_PHASE_LUPP_ROW = 4,  /* I_k, row selection                                */
  CUR_PHASE_FACTORS = 5,   /* Rt_k, N_k^+, L_k (Lemma 1 factors)                */
  CUR_PHASE_COL_RES = 6,   /* S^col update and ||S^col||_F (rho_k)              */
  CUR_PHASE_CORE = 7,      /* U = A(I,J)^+ at exit                              */
  CUR_PHASE_SCALES = 8,    /* FP64 tensor-core sketch only: G_q and the column
                              scales (a read of A); CUR_PHASE_SKETCH is then the
                              tensor-core pass and its reduction                */
  CUR_PHASE_COUNT = 9
} cur_phase;

/* Create a context on `device` that enqueues on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream).  hbm_budget_bytes caps the workspace the
 * context may hold (0 = no cap).  *out receives the context. */
int cur_create(cur_ctx **out, int device, void *cuda_stream, size_t hbm_budget_bytes);

/* Release the context and its workspace.  NULL is a no-op. */
void cur_free(cur_ctx *ctx);

/* Text of the last failure on this context ("" if none); owned by the ctx. */
const char *cur_last_error(const cur_ctx *ctx);

/* Run Algorithm 1 on a device matrix.
 *   A           device, m x n, row stride lda, FP64 or FP32 (dtype); borrowed:
 *               read only, must stay valid and unchanged until the call returns.
 *   tol         eps > 0 (NaN or <= 0: CUR_EINVAL).  eps >= 1 returns rank 0.
 *   block_size  b >= 1 indices per iteration (Algorithm 1 input b).
 *   sketch_size c rows of G; 0 selects floor(1.1 b) (Sec. 1.1); c < b: EINVAL.
 *   seed        key of the Gaussian sketch (see cur_step_gaussian).
 *   *out        a new result owned by the caller (free with cur_result_free);
 *               set on CUR_OK and on CUR_TOL_UNREACHED, NULL otherwise.
 * A = 0 (G A = 0) returns rank 0 with rho = 0. */
int cur_run(cur_ctx *ctx, const void *A, int64_t m, int64_t n, int64_t lda,
            int dtype, double tol, int block_size, int sketch_size,
            uint64_t seed, cur_result **out);

/* cur_run with options (opts may be NULL = defaults). */
int cur_run_opts(cur_ctx *ctx, const void *A, int64_t m, int64_t n,
                 int64_t lda, int dtype, double tol, int block_size,
                 int sketch_size, uint64_t seed, const cur_opts *opts,
                 cur_result **out);

/* End-to-end form: A is a HOST buffer (m x n, stride lda).  The call copies A
 * to the device (a context-owned buffer, grown as needed), runs, and copies
 * I, J, U and rho back into the result's host mirrors before returning.  With
 * the FP64 sketch the copy goes in row blocks on a second stream and the
 * sketch of each block starts when its copy lands (the copy overlaps the
 * sketch); the precision forms copy A whole first.  A_host is read until the
 * call returns (pinned memory makes the copies asynchronous). */
int cur_run_host(cur_ctx *ctx, const void *A_host, int64_t m, int64_t n,
                 int64_t lda, int dtype, double tol, int block_size,
                 int sketch_size, uint64_t seed, const cur_opts *opts,
                 cur_result **out);

/* Accessors.  Device arrays stay valid until cur_result_free. */
int64_t cur_result_rank(const cur_result *r);          /* |I| = |J|            */
int64_t cur_result_iterations(const cur_result *r);   /* loop iterations      */
int cur_result_status(const cur_result *r);            /* CUR_OK / TOL_UNREACHED */
double cur_result_err(const cur_result *r);            /* final rho            */
double cur_result_sketch_norm(const cur_result *r);    /* ||G A||_F            */
const int64_t *cur_result_I(const cur_result *r);      /* device, rank entries */
const int64_t *cur_result_J(const cur_result *r);      /* device, rank entries */
const double *cur_result_U(const cur_result *r);       /* device, rank x rank,
                                                          rows follow J, columns I */
/* Device milliseconds spent in `phase` (0 unless the run had opts->timing). */
double cur_result_phase_ms(const cur_result *r, int phase);
/* Number of kernel launches the run issued (all of them this library's). */
int64_t cur_result_kernel_launches(const cur_result *r);
/* rho after each iteration; host array of cur_result_iterations() entries. */
const double *cur_result_rho_history(const cur_result *r);

/* Copy I, J (rank entries each) and U (rank*rank) to host buffers; any of them
 * may be NULL.  Synchronises the context's stream. */
int cur_result_copy_to_host(const cur_result *r, int64_t *I, int64_t *J, double *U);

/* Release a result (device and host buffers).  NULL is a no-op. */
void cur_result_free(cur_result *r);

#ifdef __cplusplus
}
#endif
#endif /* CUR_H */
