/*
 * cur_oracle.h -- plain, slow, FP64 CPU restatement of IterativeCUR
 * (Pritchard, Park, Nakatsukasa, Martinsson, "Fast Rank Adaptive CUR via a
 * Recycled Small Sketch", arXiv 2509.21963, Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file: only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py use it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * Conventions: all matrices are row-major FP64; indices are 0-based (the paper
 * is 1-based); "u" below is the unit roundoff 2^-53.
 */
#ifndef CUR_ORACLE_H
#define CUR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x64-10 block function (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4):
 * ten rounds of the 4x64 S-box with the published multipliers and Weyl key
 * increments.  out may alias ctr. */
void cur_oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                              uint64_t out[4]);

/* Gaussian sketching matrix G (Algorithm 1, "Generate a sketch matrix";
 * entries N(0,1), Sec. 3.2 "random matrix with Gaussian entries").
 * Definition used on both sides of this project:
 *   block (i, q) = Philox4x64-10(ctr = {q, i, 0, 0}, key = {seed, 0x43555200})
 *   u_t = ((x_t >> 11) + 0.5) * 2^-53          t = 0..3, all in (0,1)
 *   G[i, 4q+0] = sqrt(-2 ln u_0) cos(2 pi u_1)  G[i, 4q+1] = ... sin(2 pi u_1)
 *   G[i, 4q+2] = sqrt(-2 ln u_2) cos(2 pi u_3)  G[i, 4q+3] = ... sin(2 pi u_3)
 * (Box & Muller 1958).  G is c x m, row-major. */
void cur_oracle_gaussian_sketch(uint64_t seed, int64_t c, int64_t m, double *G);

/* Y = G A (Algorithm 1, initial sketch S_0^col = G A).  G c x m, A m x n with
 * row stride lda, Y c x n. */
void cur_oracle_sketch(const double *G, int64_t c, const double *A, int64_t m,
                       int64_t n, int64_t lda, double *Y);

/* LU with partial pivoting used as an index selector (Sec. 3.2.1/3.2.2):
 * the candidates are the p rows of M (p x q, stride ldm).  For step
 * t = 0..steps-1 the pivot is the eligible row with the largest |W[i,t]| of the
 * current Schur complement W (ties: smallest index); every other eligible row
 * is then eliminated against it.  A zero pivot column selects the smallest
 * eligible index and eliminates nothing.  excluded[i] != 0 marks rows that may
 * not be chosen (already selected indices); chosen rows are marked in it.
 * min_gap (if not NULL) receives min over steps of |pivot| - |runner-up|.
 * Returns 0, or -1 if fewer than `steps` eligible rows exist. */
int cur_oracle_lupp(const double *M, int64_t p, int64_t q, int64_t ldm,
                    int64_t steps, uint8_t *excluded, int64_t *piv,
                    double *min_gap);

/* Generalised inverse M^+ of a p x q matrix through Householder QR with column
 * pivoting (Businger & Golub 1965), the core solve "U = A(I,J)^+, default QR"
 * of Algorithm 1.  With M P = Q R, the numerical rank k counts leading
 * |R_ii| > thr, and X = P [R_11^{-1} Q_1^T ; 0] (q x p, row-major, dense).
 * thr < 0 selects thr = max(p,q) * 2^-52 * |R_00|.
 * perm (q entries) and rdiag (min(p,q) entries) may be NULL.  Returns k. */
int64_t cur_oracle_qrcp_pinv(const double *M, int64_t p, int64_t q,
                             int64_t ldm, double thr, double *X, int64_t *perm,
                             double *rdiag);

/* Output record of cur_oracle_run.  Arrays are caller-owned with the stated
 * capacities (max_rank = R, max iterations = K). */
typedef struct cur_oracle_out {
  int64_t *I;         /* R entries: selected rows, selection order           */
  int64_t *J;         /* R entries: selected columns, selection order        */
  double *U;          /* R*R: U (|J| x |I|) written with row stride |I|      */
  double *rho_hist;   /* K: rho_k after each iteration                       */
  double *gap_col;    /* K: min LUPP gap of the column selection, iteration k */
  double *gap_row;    /* K: min LUPP gap of the row selection, iteration k   */
  double *scale_row;  /* K: max |S^row| of iteration k (gap_row normaliser)  */
  double *S_final;    /* c*n or NULL: final column residual S^col            */
  int64_t hist_cap;   /* K                                                    */
  int64_t rank;       /* |I| = |J| at exit                                    */
  int64_t iters;      /* iterations run                                       */
  double rho;         /* final rho                                            */
  double normY;       /* ||G A||_F                                            */
  double maxabsY;     /* max |G A| (gap_col normaliser)                       */
  int status;         /* 0 ok, 7 tolerance not reached at max_rank, <0 error  */
} cur_oracle_out;

/* The whole method (Algorithm 1).
 *   A m x n (stride lda); tol = epsilon; b = block size; c = sketch rows;
 *   G = explicit c x m sketch or NULL (then generated from seed as above);
 *   max_rank <= min(m, n) (0 selects min(m, n));
 *   mode 0: the row and column residuals as Algorithm 1 states them, with
 *           U = A(I,J)^+ recomputed by QRCP every iteration,
 *           S^row = A(:,J_k) - C U R(:,J_k), S^col = GA - (GC) U R;
 *   mode 1: the same residuals through Lemma 1, S_k = S_{k-1} - S(:,J_k)
 *           N_k^+ S(I_k,:) with N_k = S_{k-1}(I_k,J_k) (N_k^+ by QRCP with the
 *           absolute threshold |I| * 2^-52 * |R_00(N_1)|), and U = A(I,J)^+ by
 *           QRCP once at exit.  Identical in exact arithmetic (Lemma 1).
 * Stopping: the loop runs while rho > tol and |J| < max_rank. */
int cur_oracle_run(const double *A, int64_t m, int64_t n, int64_t lda,
                   double tol, int64_t b, int64_t c, uint64_t seed,
                   const double *G, int64_t max_rank, int mode,
                   cur_oracle_out *out);

/* cur_oracle_run with the initial sketch taken of Asketch (m x n, stride n)
 * instead of A: Y = G Asketch; every later step uses A.  Asketch = NULL is
 * cur_oracle_run.  Used for the precision form of the sketch. */
int cur_oracle_run_sketched(const double *A, const double *Asketch, int64_t m, int64_t n,
                            int64_t lda, double tol, int64_t b, int64_t c, uint64_t seed,
                            const double *G, int64_t max_rank, int mode,
                            cur_oracle_out *out);

/* The loop of cur_oracle_run (Algorithm 1 after its initial sketch) started
 * from a given initial sketch Y = S_0^col (c x n, stride n) of A. */
int cur_oracle_run_y(const double *A, int64_t m, int64_t n, int64_t lda, double tol,
                     int64_t b, int64_t c, const double *Y, int64_t max_rank, int mode,
                     cur_oracle_out *out);

/* 8-bit Gaussian sketch: clamp(rint(16 Z), -127, 127), Z as above. */
void cur_oracle_gaussian_sketch_q8(uint64_t seed, int64_t c, int64_t m, double *G);

/* The same rounding of a given sketch: out = clamp(rint(16 G), -127, 127),
 * ties to even (the precision forms' reading of an explicit sketch). */
void cur_oracle_quantize_q8(const double *G, int64_t len, double *out);

/* S-digit base-256 fixed point of A per column (see cur_oracle.c). */
void cur_oracle_fixed_point(const double *A, int64_t m, int64_t n, int64_t lda, int S,
                            double *Afix);

/* The S base-256 digits of fix_S(x) at column scale 2^E, d[S-1] the most
 * significant (see cur_oracle.c). */
void cur_oracle_fixed_point_digits(double x, int E, int S, double *d);

/* Exact fixed-point sketch of the FP64 tensor-core form: per column the scale
 * 2^E_j > max |A(:,j)|, X = trunc(A 2^(Q - E_j)) (integers), and
 * Y(i,j) = RN(sum_k Gq(i,k) X(k,j)) 2^(E_j - Q) with the integer sum exact
 * and rounded once.  Gq c x m integer-valued; A m x n (stride lda); Y c x n. */
void cur_oracle_sketch_fx(const double *Gq, int64_t c, const double *A, int64_t m,
                          int64_t n, int64_t lda, int Q, double *Y);

/* The naive loop of Sec. 3.1: identical selections, but the residual
 * S = A - C U R is formed in full every iteration and sketched afresh
 * (G S) instead of recycling G A.  For tiny inputs only. */
int cur_oracle_run_naive(const double *A, int64_t m, int64_t n, int64_t lda,
                         double tol, int64_t b, int64_t c, const double *G,
                         int64_t max_rank, cur_oracle_out *out);

/* True relative error ||A - C U R||_F / ||A||_F for given I, J, U (|J| x |I|,
 * row stride r).  O(m n r). */
double cur_oracle_true_error(const double *A, int64_t m, int64_t n, int64_t lda,
                             const int64_t *I, const int64_t *J, int64_t r,
                             const double *U);

/* Host threads of the OpenMP-parallel outer loops (1 without OpenMP); the
 * results are the same for every thread count (no reduction is split). */
void cur_oracle_set_threads(int nthreads);
int cur_oracle_threads(void);

/* Risk-aware threshold of Sec. 3.3: eps (1+delta) sqrt(1 - 2 sqrt(-ln(alpha)/c)),
 * or -1 when c <= -4 ln(alpha) (bound undefined). */
double cur_oracle_risk_threshold(double eps, double delta, double alpha, double c);

#ifdef __cplusplus
}
#endif
#endif
