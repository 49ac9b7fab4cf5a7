/*
 * cur_oracle.c -- plain, slow, obviously-correct FP64 CPU restatement of
 * IterativeCUR (arXiv 2509.21963, Algorithm 1, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py; never by the product path.  No blocking,
 * fusion or reordering beyond what the paper states: each step is the textbook
 * loop, in the paper's order and notation.  Compile with -ffp-contract=off so
 * that every product and sum is rounded as written.
 *
 * Parity status of each function (what pins it, see tests/test_oracle_*.py):
 *   philox4x64_10    - numpy.random.Philox raw stream (independent executable)
 *   gaussian_sketch  - moments / Kolmogorov-Smirnov against N(0,1)
 *   sketch           - numpy matmul on small shapes
 *   lupp             - scipy.linalg.lu pivot order; brute-force definitions
 *   qrcp_pinv        - numpy inverse / pinv; scipy QRCP pivots; M X M = M
 *   run (modes 0,1)  - exact-rank recovery (Sec. 5.1), Example 1 (Sec. 3.2.1),
 *                      dependent-selection example (Sec. 3.2), Lemma 1,
 *                      interpolation S(:,J)=0, S(I,:)=0 (Sec. 3.2.2),
 *                      Theorem 2 brute force on tiny matrices (Sec. 4.2),
 *                      estimator vs truth (Sec. 3.3), naive loop (Sec. 3.1)
 *   run_sketched     - bit-equal to run when the sketched matrix is A
 *   run_y            - bit-equal to run started from run's own sketch
 *   true_error       - numpy norm(A - C U R) / norm(A)
 *   gaussian_sketch_q8, quantize_q8
 *                    - integer, |q| <= 127, |q - 16 g| <= 1/2 inside the clamp,
 *                      the clamp and ties-to-even on crafted values, moments
 *   fixed_point, fixed_point_digits
 *                    - |fix_S(x) - x| <= 2^(E-8S-1); one rounding half-to-even
 *                      of x 2^(8S-E) in exact rational arithmetic; grid values
 *                      unchanged; E = frexp of the column max; digits integer,
 *                      |d| <= 256, reassembling fix_S
 *   sketch_fx        - exact rational evaluation with Python integers; the
 *                      truncation error bound; integer data equal to an int64
 *                      matmul; truncation toward zero on a crafted entry
 * (tests/test_oracle_pins.py, tests/test_oracle_precision_pins.py).
 */
#include "cur_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon et al., SC'11).                                    */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL
#define PHILOX_W1 0xBB67AE8584CAA73BULL

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void cur_oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                              uint64_t out[4]) {
  uint64_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { /* key schedule: Weyl increments between rounds */
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(PHILOX_M0, x[0], &hi0, &lo0);
    mulhilo64(PHILOX_M1, x[2], &hi1, &lo1);
    uint64_t y0 = hi1 ^ x[1] ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x[3] ^ k1;
    uint64_t y3 = lo0;
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
  }
  out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
}

/* ------------------------------------------------------------------------ */
/* Gaussian sketch G (c x m).                                               */
/* ------------------------------------------------------------------------ */
static double uniform_open01(uint64_t x) {
  /* 53 high bits, shifted by half a step: never 0, never 1 */
  return ((double)(x >> 11) + 0.5) * 0x1.0p-53;
}

void cur_oracle_gaussian_sketch(uint64_t seed, int64_t c, int64_t m,
                                double *G) {
  const double two_pi = 6.283185307179586476925286766559;
  const uint64_t key[2] = {seed, 0x43555200ULL};
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < c; ++i) {
    for (int64_t q = 0; 4 * q < m; ++q) {
      uint64_t ctr[4] = {(uint64_t)q, (uint64_t)i, 0, 0};
      uint64_t x[4];
      cur_oracle_philox4x64_10(ctr, key, x);
      double u0 = uniform_open01(x[0]), u1 = uniform_open01(x[1]);
      double u2 = uniform_open01(x[2]), u3 = uniform_open01(x[3]);
      double r01 = sqrt(-2.0 * log(u0));
      double r23 = sqrt(-2.0 * log(u2));
      double t1 = two_pi * u1;
      double t3 = two_pi * u3;
      double z[4] = {r01 * cos(t1), r01 * sin(t1), r23 * cos(t3),
                     r23 * sin(t3)};
      for (int t = 0; t < 4; ++t) {
        int64_t k = 4 * q + t;
        if (k < m) G[i * m + k] = z[t];
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Y = G A.                                                                 */
/* ------------------------------------------------------------------------ */
void cur_oracle_sketch(const double *G, int64_t c, const double *A, int64_t m,
                       int64_t n, int64_t lda, double *Y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < c; ++i) {
    double *y = Y + i * n;
    for (int64_t j = 0; j < n; ++j) y[j] = 0.0;
    for (int64_t k = 0; k < m; ++k) {
      double g = G[i * m + k];
      const double *a = A + k * lda;
      for (int64_t j = 0; j < n; ++j) y[j] = y[j] + g * a[j];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* LU with partial pivoting as a row selector.                              */
/* ------------------------------------------------------------------------ */
int cur_oracle_lupp(const double *M, int64_t p, int64_t q, int64_t ldm,
                    int64_t steps, uint8_t *excluded, int64_t *piv,
                    double *min_gap) {
  double *W = (double *)malloc(sizeof(double) * (size_t)(p * q > 0 ? p * q : 1));
  uint8_t *own = NULL;
  if (excluded == NULL) {
    own = (uint8_t *)calloc((size_t)(p > 0 ? p : 1), 1);
    excluded = own;
  }
  for (int64_t i = 0; i < p; ++i)
    for (int64_t j = 0; j < q; ++j) W[i * q + j] = M[i * ldm + j];
  double gap_min = INFINITY;
  int rc = 0;
  for (int64_t t = 0; t < steps; ++t) {
    int64_t best = -1;
    double best_abs = -1.0, second_abs = -1.0;
    for (int64_t i = 0; i < p; ++i) {
      if (excluded[i]) continue;
      double a = fabs(W[i * q + t]);
      if (a > best_abs) {
        second_abs = best_abs;
        best_abs = a;
        best = i;
      } else if (a > second_abs) {
        second_abs = a;
      }
    }
    if (best < 0) { rc = -1; break; }
    double gap = best_abs - (second_abs > 0.0 ? second_abs : 0.0);
    if (gap < gap_min) gap_min = gap;
    piv[t] = best;
    excluded[best] = 1;
    if (best_abs == 0.0) continue; /* zero pivot: nothing to eliminate */
    const double *prow = W + best * q;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < p; ++i) {
      if (excluded[i]) continue;
      double l = W[i * q + t] / prow[t];
      for (int64_t j = t + 1; j < q; ++j) W[i * q + j] = W[i * q + j] - l * prow[j];
    }
  }
  if (min_gap) *min_gap = gap_min;
  free(W);
  free(own);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Generalised inverse by Householder QR with column pivoting.              */
/* ------------------------------------------------------------------------ */
int64_t cur_oracle_qrcp_pinv(const double *M, int64_t p, int64_t q,
                             int64_t ldm, double thr, double *X, int64_t *perm,
                             double *rdiag) {
  int64_t kmax = p < q ? p : q;
  double *R = (double *)malloc(sizeof(double) * (size_t)(p * q > 0 ? p * q : 1));
  double *V = (double *)calloc((size_t)(p * (kmax > 0 ? kmax : 1)), sizeof(double));
  double *tau = (double *)calloc((size_t)(kmax > 0 ? kmax : 1), sizeof(double));
  int64_t *pm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(q > 0 ? q : 1));
  for (int64_t i = 0; i < p; ++i)
    for (int64_t j = 0; j < q; ++j) R[i * q + j] = M[i * ldm + j];
  for (int64_t j = 0; j < q; ++j) pm[j] = j;

  for (int64_t j = 0; j < kmax; ++j) {
    /* pivot: remaining column of largest 2-norm over rows j..p-1 */
    int64_t best = j;
    double best_n2 = -1.0;
    for (int64_t col = j; col < q; ++col) {
      double s = 0.0;
      for (int64_t i = j; i < p; ++i) s = s + R[i * q + col] * R[i * q + col];
      if (s > best_n2) { best_n2 = s; best = col; }
    }
    if (best != j) {
      for (int64_t i = 0; i < p; ++i) {
        double t = R[i * q + j];
        R[i * q + j] = R[i * q + best];
        R[i * q + best] = t;
      }
      int64_t t = pm[j]; pm[j] = pm[best]; pm[best] = t;
    }
    /* Householder reflector H = I - tau v v^T mapping R[j:p, j] to alpha e1 */
    double *v = V + j * p; /* v[i] for i = j..p-1 */
    double normx = 0.0;
    for (int64_t i = j; i < p; ++i) normx = normx + R[i * q + j] * R[i * q + j];
    normx = sqrt(normx);
    if (normx == 0.0) { tau[j] = 0.0; continue; }
    double x0 = R[j * q + j];
    double alpha = (x0 >= 0.0) ? -normx : normx;
    for (int64_t i = j; i < p; ++i) v[i] = R[i * q + j];
    v[j] = x0 - alpha;
    double vn2 = 0.0;
    for (int64_t i = j; i < p; ++i) vn2 = vn2 + v[i] * v[i];
    tau[j] = 2.0 / vn2;
    for (int64_t col = j; col < q; ++col) {
      double d = 0.0;
      for (int64_t i = j; i < p; ++i) d = d + v[i] * R[i * q + col];
      double f = tau[j] * d;
      for (int64_t i = j; i < p; ++i) R[i * q + col] = R[i * q + col] - f * v[i];
    }
    R[j * q + j] = alpha;
    for (int64_t i = j + 1; i < p; ++i) R[i * q + j] = 0.0;
  }

  if (thr < 0.0) {
    double big = (p > q ? p : q);
    thr = kmax > 0 ? big * DBL_EPSILON * fabs(R[0]) : 0.0;
  }
  int64_t k = 0;
  while (k < kmax && fabs(R[k * q + k]) > thr) ++k;
  if (rdiag)
    for (int64_t i = 0; i < kmax; ++i) rdiag[i] = R[i * q + i];
  if (perm)
    for (int64_t j = 0; j < q; ++j) perm[j] = pm[j];

  /* Q^T = H_{k-1} ... H_0 applied to the identity (only the first k
   * reflectors matter for the first k rows of Q^T). */
  double *QT = (double *)calloc((size_t)(p * p > 0 ? p * p : 1), sizeof(double));
  for (int64_t i = 0; i < p; ++i) QT[i * p + i] = 1.0;
  for (int64_t j = 0; j < k; ++j) {
    if (tau[j] == 0.0) continue;
    const double *v = V + j * p;
    for (int64_t col = 0; col < p; ++col) {
      double d = 0.0;
      for (int64_t i = j; i < p; ++i) d = d + v[i] * QT[i * p + col];
      double f = tau[j] * d;
      for (int64_t i = j; i < p; ++i) QT[i * p + col] = QT[i * p + col] - f * v[i];
    }
  }
  /* Z = R_11^{-1} Q_1^T by back substitution (k x p) */
  double *Z = (double *)calloc((size_t)(k * p > 0 ? k * p : 1), sizeof(double));
  for (int64_t col = 0; col < p; ++col) {
    for (int64_t i = k - 1; i >= 0; --i) {
      double s = QT[i * p + col];
      for (int64_t l = i + 1; l < k; ++l) s = s - R[i * q + l] * Z[l * p + col];
      Z[i * p + col] = s / R[i * q + i];
    }
  }
  /* X = P [Z; 0] : row pm[i] of X is row i of Z */
  for (int64_t i = 0; i < q * p; ++i) X[i] = 0.0;
  for (int64_t i = 0; i < k; ++i)
    for (int64_t col = 0; col < p; ++col) X[pm[i] * p + col] = Z[i * p + col];

  free(Z); free(QT); free(pm); free(tau); free(V); free(R);
  return k;
}

/* ------------------------------------------------------------------------ */
/* Helpers of the main loop (plain loops).                                  */
/* ------------------------------------------------------------------------ */
static double frob(const double *X, int64_t len) {
  double s = 0.0;
  for (int64_t i = 0; i < len; ++i) s = s + X[i] * X[i];
  return sqrt(s);
}

/* U = A(I,J)^+ (|J| x |I|) recomputed by QRCP (paper default). */
static void core_by_qrcp(const double *A, int64_t lda, const int64_t *I,
                         const int64_t *J, int64_t r, double *U) {
  double *Mc = (double *)malloc(sizeof(double) * (size_t)(r * r));
  for (int64_t a = 0; a < r; ++a)
    for (int64_t bb = 0; bb < r; ++bb) Mc[a * r + bb] = A[I[a] * lda + J[bb]];
  cur_oracle_qrcp_pinv(Mc, r, r, r, -1.0, U, NULL, NULL);
  free(Mc);
}

/* S^row = A(:,J_k) - C U R(:,J_k) (m x bk), with C = A(:,J), R = A(I,:). */
static void row_residual(const double *A, int64_t m, int64_t lda,
                         const int64_t *I, const int64_t *J, int64_t r,
                         const double *U, const int64_t *Jk, int64_t bk,
                         double *Srow) {
  double *X = (double *)calloc((size_t)(r * bk + 1), sizeof(double));
  for (int64_t a = 0; a < r; ++a) /* X = U R(:,J_k), r x bk */
    for (int64_t t = 0; t < bk; ++t) {
      double s = 0.0;
      for (int64_t l = 0; l < r; ++l) s = s + U[a * r + l] * A[I[l] * lda + Jk[t]];
      X[a * bk + t] = s;
    }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i)
    for (int64_t t = 0; t < bk; ++t) {
      double s = 0.0;
      for (int64_t l = 0; l < r; ++l) s = s + A[i * lda + J[l]] * X[l * bk + t];
      Srow[i * bk + t] = A[i * lda + Jk[t]] - s;
    }
  free(X);
}

/* S^col = Y - (Y(:,J) U) R, with R = A(I,:) (c x n). */
static void col_residual(const double *Y, int64_t c, int64_t n,
                         const double *A, int64_t lda, const int64_t *I,
                         const int64_t *J, int64_t r, const double *U,
                         double *S) {
  double *W = (double *)calloc((size_t)(c * r + 1), sizeof(double));
  for (int64_t i = 0; i < c; ++i) /* W = Y(:,J) U, c x r */
    for (int64_t a = 0; a < r; ++a) {
      double s = 0.0;
      for (int64_t l = 0; l < r; ++l) s = s + Y[i * n + J[l]] * U[l * r + a];
      W[i * r + a] = s;
    }
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t i = 0; i < c; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double s = 0.0;
      for (int64_t a = 0; a < r; ++a) s = s + W[i * r + a] * A[I[a] * lda + j];
      S[i * n + j] = Y[i * n + j] - s;
    }
  free(W);
}

static void record(cur_oracle_out *out, int64_t k, double rho, double gc,
                   double gr, double sr) {
  if (k < out->hist_cap) {
    if (out->rho_hist) out->rho_hist[k] = rho;
    if (out->gap_col) out->gap_col[k] = gc;
    if (out->gap_row) out->gap_row[k] = gr;
    if (out->scale_row) out->scale_row[k] = sr;
  }
}

static double maxabs(const double *X, int64_t len) {
  double s = 0.0;
  for (int64_t i = 0; i < len; ++i) s = fabs(X[i]) > s ? fabs(X[i]) : s;
  return s;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1.                                                             */
/* ------------------------------------------------------------------------ */
/* Residual at rows / columns of A in the Lemma 1 form: with the block factors
 * L_l = S_{l-1}(:,J_l) N_l^+ (stored as the columns of L, m x r) and
 * Rt_l = S_{l-1}(I_l,:) (the rows of Rt, r x n), Lemma 1 applied k times gives
 * S_k = A - sum_l L_l Rt_l. */
static double lemma_residual_entry(const double *A, int64_t lda, const double *L,
                                   int64_t ldl, const double *Rt, int64_t n,
                                   int64_t r, int64_t i, int64_t j) {
  double s = 0.0;
  for (int64_t l = 0; l < r; ++l) s = s + L[i * ldl + l] * Rt[l * n + j];
  return A[i * lda + j] - s;
}

int cur_oracle_run(const double *A, int64_t m, int64_t n, int64_t lda,
                   double tol, int64_t b, int64_t c, uint64_t seed,
                   const double *Gin, int64_t max_rank, int mode,
                   cur_oracle_out *out) {
  return cur_oracle_run_sketched(A, NULL, m, n, lda, tol, b, c, seed, Gin, max_rank, mode, out);
}

int cur_oracle_run_sketched(const double *A, const double *Asketch, int64_t m, int64_t n,
                            int64_t lda, double tol, int64_t b, int64_t c, uint64_t seed,
                            const double *Gin, int64_t max_rank, int mode,
                            cur_oracle_out *out) {
  out->rank = 0; out->iters = 0; out->rho = 1.0; out->status = 0;
  if (m <= 0 || n <= 0 || b <= 0 || c < b || !(tol > 0.0)) { out->status = -1; return -1; }

  /* sketch matrix G (c x m) */
  double *G = (double *)malloc(sizeof(double) * (size_t)(c * m));
  if (Gin) memcpy(G, Gin, sizeof(double) * (size_t)(c * m));
  else cur_oracle_gaussian_sketch(seed, c, m, G);

  /* initial sketch S_0 = G A */
  double *Y = (double *)malloc(sizeof(double) * (size_t)(c * n));
  if (Asketch) cur_oracle_sketch(G, c, Asketch, m, n, n, Y);
  else cur_oracle_sketch(G, c, A, m, n, lda, Y);
  free(G);
  int rc = cur_oracle_run_y(A, m, n, lda, tol, b, c, Y, max_rank, mode, out);
  free(Y);
  return rc;
}

int cur_oracle_run_y(const double *A, int64_t m, int64_t n, int64_t lda, double tol,
                     int64_t b, int64_t c, const double *Y, int64_t max_rank, int mode,
                     cur_oracle_out *out) {
  int64_t mn = m < n ? m : n;
  if (max_rank <= 0 || max_rank > mn) max_rank = mn;
  out->rank = 0; out->iters = 0; out->rho = 1.0; out->status = 0;
  if (m <= 0 || n <= 0 || b <= 0 || c < b || !(tol > 0.0)) { out->status = -1; return -1; }

  /* rho_0 = ||S_0|| / ||G A|| = 1 */
  double nY = frob(Y, c * n);
  out->normY = nY;
  out->maxabsY = maxabs(Y, c * n);
  double *S = (double *)malloc(sizeof(double) * (size_t)(c * n));
  memcpy(S, Y, sizeof(double) * (size_t)(c * n));
  if (nY == 0.0) { /* G A = 0: nothing to approximate (reading of 0/0) */
    out->rho = 0.0;
    if (out->S_final) memcpy(out->S_final, S, sizeof(double) * (size_t)(c * n));
    free(S);
    return 0;
  }
  double rho = 1.0;

  int64_t *I = out->I, *J = out->J;
  double *U = (double *)calloc((size_t)(max_rank * max_rank + 1), sizeof(double));
  uint8_t *excl_col = (uint8_t *)calloc((size_t)n, 1);
  uint8_t *excl_row = (uint8_t *)calloc((size_t)m, 1);
  double *ST = (double *)malloc(sizeof(double) * (size_t)(n * c));
  double *Srow = (double *)malloc(sizeof(double) * (size_t)(m * b));
  double *N = (double *)malloc(sizeof(double) * (size_t)(b * b));
  double *Np = (double *)malloc(sizeof(double) * (size_t)(b * b));
  double *T1 = (double *)malloc(sizeof(double) * (size_t)(c * b));
  /* Lemma 1 factors (mode 1 only) */
  double *L = NULL, *Rt = NULL;
  if (mode == 1) {
    L = (double *)calloc((size_t)(m * max_rank), sizeof(double));
    Rt = (double *)calloc((size_t)(max_rank * n), sizeof(double));
  }
  double thr_scale = -1.0;
  int64_t r = 0, k = 0;

  while (rho > tol && r < max_rank) { /* loop while rho exceeds tol */
    int64_t bk = b < max_rank - r ? b : max_rank - r;
    /* column selection: J_k = LUPP on the sketched residual (candidates = columns) */
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < c; ++i) ST[j * c + i] = S[i * n + j];
    double gap_c = INFINITY, gap_r = INFINITY;
    cur_oracle_lupp(ST, n, c, c, bk, excl_col, J + r, &gap_c);
    /* row residual: S^row_k = A(:,J_k) - C U R(:,J_k) with the previous C, U, R */
    if (mode == 0) {
      row_residual(A, m, lda, I, J, r, U, J + r, bk, Srow);
    } else {
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < m; ++i)
        for (int64_t t = 0; t < bk; ++t)
          Srow[i * bk + t] = lemma_residual_entry(A, lda, L, max_rank, Rt, n, r, i, J[r + t]);
    }
    double srow_scale = maxabs(Srow, m * bk);
    /* row selection: I_k = LUPP on the row residual (candidates = rows) */
    cur_oracle_lupp(Srow, m, bk, bk, bk, excl_row, I + r, &gap_r);
    /* index updates: J = [J, J_k], I = [I, I_k] */
    int64_t rn = r + bk;
    if (mode == 0) {
      /* core: U = A(I,J)^+ by pivoted QR, recomputed */
      core_by_qrcp(A, lda, I, J, rn, U);
      /* column residual: S^col = G A - (G C) U R, G C = (G A)(:,J) */
      col_residual(Y, c, n, A, lda, I, J, rn, U, S);
    } else {
      /* Lemma 1 with I+ = I_k, J+ = J_k: S_k = S_{k-1} - S(:,J_k) N^+ S(I_k,:),
       * N = S_{k-1}(I_k, J_k) = S^row(I_k, :); sketched: G S(:,J_k) is the
       * column J_k of S^col, so S^col_k = S^col - S^col(:,J_k) N^+ S(I_k,:). */
      for (int64_t a = 0; a < bk; ++a)
        for (int64_t t = 0; t < bk; ++t) N[a * bk + t] = Srow[I[r + a] * bk + t];
      if (thr_scale < 0.0) { /* rank threshold: |R_00| of the first core */
        double *rdiag = (double *)malloc(sizeof(double) * (size_t)bk);
        cur_oracle_qrcp_pinv(N, bk, bk, bk, -1.0, Np, NULL, rdiag);
        thr_scale = fabs(rdiag[0]) * DBL_EPSILON;
        free(rdiag);
      }
      cur_oracle_qrcp_pinv(N, bk, bk, bk, thr_scale * (double)rn, Np, NULL, NULL);
      /* Rt_k = S_{k-1}(I_k, :) */
#pragma omp parallel for collapse(2) schedule(static)
      for (int64_t a = 0; a < bk; ++a)
        for (int64_t j = 0; j < n; ++j)
          Rt[(r + a) * n + j] = lemma_residual_entry(A, lda, L, max_rank, Rt, n, r, I[r + a], j);
      /* L_k = S^row N^+  (m x bk) */
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < m; ++i)
        for (int64_t a = 0; a < bk; ++a) {
          double s = 0.0;
          for (int64_t t = 0; t < bk; ++t) s = s + Srow[i * bk + t] * Np[t * bk + a];
          L[i * max_rank + r + a] = s;
        }
      /* S^col = S^col - (S^col(:,J_k) N^+) Rt_k */
      for (int64_t i = 0; i < c; ++i)
        for (int64_t a = 0; a < bk; ++a) {
          double s = 0.0;
          for (int64_t t = 0; t < bk; ++t) s = s + S[i * n + J[r + t]] * Np[t * bk + a];
          T1[i * bk + a] = s;
        }
#pragma omp parallel for collapse(2) schedule(static)
      for (int64_t i = 0; i < c; ++i)
        for (int64_t j = 0; j < n; ++j) {
          double s = 0.0;
          for (int64_t a = 0; a < bk; ++a) s = s + T1[i * bk + a] * Rt[(r + a) * n + j];
          S[i * n + j] = S[i * n + j] - s;
        }
    }
    r = rn;
    /* rho_k = ||S^col|| / ||G A|| */
    rho = frob(S, c * n) / nY;
    record(out, k, rho, gap_c, gap_r, srow_scale);
    ++k;
  }
  /* core at exit (Lemma 1 mode): U of the returned CUR */
  if (mode == 1 && r > 0) core_by_qrcp(A, lda, I, J, r, U);
  out->rank = r;
  out->iters = k;
  out->rho = rho;
  out->status = (rho > tol) ? 7 : 0;
  if (out->U)
    for (int64_t a = 0; a < r * r; ++a) out->U[a] = U[a];
  if (out->S_final) memcpy(out->S_final, S, sizeof(double) * (size_t)(c * n));
  free(Rt); free(L); free(T1); free(Np); free(N); free(Srow); free(ST);
  free(excl_row); free(excl_col); free(U); free(S);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Naive loop (Sec. 3.1): full residual, re-sketched every iteration.       */
/* ------------------------------------------------------------------------ */
int cur_oracle_run_naive(const double *A, int64_t m, int64_t n, int64_t lda,
                         double tol, int64_t b, int64_t c, const double *G,
                         int64_t max_rank, cur_oracle_out *out) {
  int64_t mn = m < n ? m : n;
  if (max_rank <= 0 || max_rank > mn) max_rank = mn;
  out->rank = 0; out->iters = 0; out->rho = 1.0; out->status = 0;
  double *Y = (double *)malloc(sizeof(double) * (size_t)(c * n));
  cur_oracle_sketch(G, c, A, m, n, lda, Y);
  double nY = frob(Y, c * n);
  out->normY = nY;
  if (nY == 0.0) { out->rho = 0.0; free(Y); return 0; }
  double *Sfull = (double *)malloc(sizeof(double) * (size_t)(m * n));
  double *GS = (double *)malloc(sizeof(double) * (size_t)(c * n));
  double *ST = (double *)malloc(sizeof(double) * (size_t)(n * c));
  double *Srow = (double *)malloc(sizeof(double) * (size_t)(m * b));
  double *U = (double *)calloc((size_t)(max_rank * max_rank + 1), sizeof(double));
  uint8_t *excl_col = (uint8_t *)calloc((size_t)n, 1);
  uint8_t *excl_row = (uint8_t *)calloc((size_t)m, 1);
  int64_t *I = out->I, *J = out->J;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) Sfull[i * n + j] = A[i * lda + j];
  double rho = 1.0;
  int64_t r = 0, k = 0;
  while (rho > tol && r < max_rank) {
    int64_t bk = b < max_rank - r ? b : max_rank - r;
    cur_oracle_sketch(G, c, Sfull, m, n, n, GS); /* G S, fresh */
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < c; ++i) ST[j * c + i] = GS[i * n + j];
    cur_oracle_lupp(ST, n, c, c, bk, excl_col, J + r, NULL);
    for (int64_t i = 0; i < m; ++i) /* S(:, J_k) read off the full residual */
      for (int64_t t = 0; t < bk; ++t) Srow[i * bk + t] = Sfull[i * n + J[r + t]];
    cur_oracle_lupp(Srow, m, bk, bk, bk, excl_row, I + r, NULL);
    r += bk;
    core_by_qrcp(A, lda, I, J, r, U);
    /* S = A - C U R in full */
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t a = 0; a < r; ++a) {
          double cu = 0.0;
          for (int64_t l = 0; l < r; ++l) cu = cu + A[i * lda + J[l]] * U[l * r + a];
          s = s + cu * A[I[a] * lda + j];
        }
        Sfull[i * n + j] = A[i * lda + j] - s;
      }
    cur_oracle_sketch(G, c, Sfull, m, n, n, GS);
    rho = frob(GS, c * n) / nY;
    record(out, k, rho, NAN, NAN, NAN);
    ++k;
  }
  out->rank = r; out->iters = k; out->rho = rho;
  out->status = (rho > tol) ? 7 : 0;
  if (out->U)
    for (int64_t a = 0; a < r * r; ++a) out->U[a] = U[a];
  free(excl_row); free(excl_col); free(U); free(Srow); free(ST); free(GS);
  free(Sfull); free(Y);
  return 0;
}

double cur_oracle_true_error(const double *A, int64_t m, int64_t n, int64_t lda,
                             const int64_t *I, const int64_t *J, int64_t r,
                             const double *U) {
  double *CU = (double *)calloc((size_t)(m * (r > 0 ? r : 1)), sizeof(double));
  for (int64_t i = 0; i < m; ++i) /* C U, m x r */
    for (int64_t a = 0; a < r; ++a) {
      double s = 0.0;
      for (int64_t l = 0; l < r; ++l) s = s + A[i * lda + J[l]] * U[l * r + a];
      CU[i * r + a] = s;
    }
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double s = 0.0;
      for (int64_t a = 0; a < r; ++a) s = s + CU[i * r + a] * A[I[a] * lda + j];
      double e = A[i * lda + j] - s;
      num = num + e * e;
      den = den + A[i * lda + j] * A[i * lda + j];
    }
  free(CU);
  return den > 0.0 ? sqrt(num / den) : 0.0;
}

/* Risk-aware stopping threshold (Sec. 3.3, Corollary): stopping when
 * ||G S||_F / ||G A||_F < eps * xi with xi = (1 + delta) sqrt(1 - 2 sqrt(-ln(alpha)/c))
 * bounds the probability of a problematic stop by alpha.  Requires
 * c > -4 ln(alpha); returns -1 otherwise. */
double cur_oracle_risk_threshold(double eps, double delta, double alpha, double c) {
  if (!(alpha > 0.0 && alpha < 1.0) || !(c > -4.0 * log(alpha))) return -1.0;
  double xi = (1.0 + delta) * sqrt(1.0 - 2.0 * sqrt(-log(alpha) / c));
  return eps * xi;
}

/* ------------------------------------------------------------------------ */
/* Precision form of the sketch (8-bit Gaussian, S-digit fixed-point A).    */
/* ------------------------------------------------------------------------ */
/* G_q[i,k] = clamp(rint(16 Z[i,k]), -127, 127) with Z the Gaussian sketch of
 * cur_oracle_gaussian_sketch (same seed): an 8-bit rounding of the Gaussian
 * sketch (the scale 16 cancels in rho and in the LUPP choices). */
void cur_oracle_gaussian_sketch_q8(uint64_t seed, int64_t c, int64_t m, double *G) {
  cur_oracle_gaussian_sketch(seed, c, m, G);
  cur_oracle_quantize_q8(G, c * m, G);
}

/* out[t] = clamp(rint(16 G[t]), -127, 127) (ties to even); out may alias G. */
void cur_oracle_quantize_q8(const double *G, int64_t len, double *out) {
  for (int64_t t = 0; t < len; ++t) {
    double q = rint(16.0 * G[t]);
    if (q > 127.0) q = 127.0;
    if (q < -127.0) q = -127.0;
    out[t] = q;
  }
}

/* fix_S(A): every column j gets the scale 2^E_j with max_k |A[k,j]| < 2^E_j
 * (E_j = 0 for a zero column); each entry x is written with S signed base-256
 * digits, d_{S-1} = rint(x 2^(8-E_j)), then repeatedly d = rint(256 r) of the
 * remainder r, so fix_S(x) = 2^(E_j - 8S) sum_s d_s 256^s (|d_s| <= 256).
 * Rounding is to nearest, ties to even.  Afix is m x n (stride n). */
void cur_oracle_fixed_point(const double *A, int64_t m, int64_t n, int64_t lda, int S,
                            double *Afix) {
  for (int64_t j = 0; j < n; ++j) {
    double mx = 0.0;
    for (int64_t k = 0; k < m; ++k) mx = fabs(A[k * lda + j]) > mx ? fabs(A[k * lda + j]) : mx;
    int E = 0;
    if (mx > 0.0) frexp(mx, &E); /* mx = f 2^E, f in [0.5, 1): mx < 2^E */
    for (int64_t k = 0; k < m; ++k) {
      double y = ldexp(A[k * lda + j], 8 - E);
      double v = 0.0;
      for (int s = S - 1; s >= 0; --s) {
        double d = rint(y);
        v = v * 256.0 + d;
        y = (y - d) * 256.0;
      }
      Afix[k * n + j] = ldexp(v, E - 8 * S);
    }
  }
}

/* The S digits of fix_S(x) for a column scale 2^E (the recursion above):
 * d[S-1] = rint(x 2^(8-E)), then d = rint(256 r) of each remainder r, most
 * significant first in d[S-1] ... d[0]. */
void cur_oracle_fixed_point_digits(double x, int E, int S, double *d) {
  double y = ldexp(x, 8 - E);
  for (int s = S - 1; s >= 0; --s) {
    d[s] = rint(y);
    y = (y - d[s]) * 256.0;
  }
}

/* ------------------------------------------------------------------------ */
/* Exact fixed-point sketch of the FP64 tensor-core form.                   */
/* ------------------------------------------------------------------------ */
/* Column j gets E_j with max_k |A(k,j)| < 2^E_j (frexp of the column max; 0
 * for a zero column).  Every entry is truncated toward zero onto the grid
 * 2^(E_j - Q): X(k,j) = trunc(A(k,j) 2^(Q - E_j)), an integer with |X| < 2^Q.
 * With Gq integer-valued, the integer sum V(i,j) = sum_k Gq(i,k) X(k,j) is
 * formed exactly (128-bit) and rounded once to FP64 (to nearest, ties to
 * even), then scaled: Y(i,j) = RN(V) 2^(E_j - Q) (a power-of-two scaling,
 * itself rounded only if the result is subnormal).  A column holding Inf or
 * NaN gives NaN in every row of Y.  Requires Q <= 52 and |Gq| <= 1024 (every
 * product then fits an int64; the sum is taken in 128 bits). */
void cur_oracle_sketch_fx(const double *Gq, int64_t c, const double *A, int64_t m,
                          int64_t n, int64_t lda, int Q, double *Y) {
#pragma omp parallel
  {
  int64_t *X = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
#pragma omp for schedule(dynamic, 16)
  for (int64_t j = 0; j < n; ++j) {
    double mx = 0.0;
    int finite = 1;
    for (int64_t k = 0; k < m; ++k) {
      double a = A[k * lda + j];
      if (!isfinite(a)) finite = 0;
      else if (fabs(a) > mx) mx = fabs(a);
    }
    if (!finite) {
      for (int64_t i = 0; i < c; ++i) Y[i * n + j] = NAN;
      continue;
    }
    int E = 0;
    if (mx > 0.0) frexp(mx, &E); /* mx = f 2^E, f in [0.5, 1): mx < 2^E */
    for (int64_t k = 0; k < m; ++k) X[k] = (int64_t)trunc(ldexp(A[k * lda + j], Q - E));
    for (int64_t i = 0; i < c; ++i) {
      __int128 v = 0;
      for (int64_t k = 0; k < m; ++k) v += (__int128)((int64_t)Gq[i * m + k] * X[k]);
      Y[i * n + j] = ldexp((double)v, E - Q);
    }
  }
  free(X);
  }
}

/* Host threads used by the loops above (OpenMP builds; 1 otherwise).  Only
 * independent outer loops run in parallel, so results do not depend on it. */
void cur_oracle_set_threads(int nthreads) {
#ifdef _OPENMP
  omp_set_num_threads(nthreads > 0 ? nthreads : 1);
#else
  (void)nthreads;
#endif
}

int cur_oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
