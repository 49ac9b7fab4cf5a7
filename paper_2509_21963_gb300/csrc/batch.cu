// batch.cu -- many independent IterativeCUR decompositions (arXiv 2509.21963,
// Algorithm 1 with the Lemma 1 residual recurrence) in ONE persistent
// cooperative launch.
//
// The grid is cut into teams of T co-resident CTAs.  A team takes the next
// job from a device-side queue (jobs sorted by estimated FP64 work, largest
// first) and runs the whole method for it without returning to the host:
//
//   G (Philox, c x m)      team-partitioned over Philox blocks
//   S = Y = G A, ||Y||_F   team-partitioned over columns of A
//   per iteration k (two team barriers):
//     J_k = LUPP(S)                 every CTA redundantly, in private scratch
//     S^row = A(:,J_k) - L Rt(:,J_k) team-partitioned over rows      | barrier
//     I_k = LUPP(S^row)             every CTA redundantly
//     N^+ = pinv(S^row(I_k,:))      every CTA redundantly (pivoted QR)
//     L_k = S^row N^+               team-partitioned over rows
//     Rt_k = A(I_k,:) - L(I_k,:) Rt, S -= (S(:,J_k) N^+) Rt_k, ||S||_F
//                                   team-partitioned over columns   | barrier
//   U = A(I,J)^+                    team pivoted QR (one barrier per
//                                   reflector) + shared-memory panel solve
//                                   (8, 4 or 2 right-hand sides per panel)
//
// Redundant small steps replace barriers: every CTA of a team computes the
// same pivots from the same data with the same code and reduction order, so
// no broadcast is needed.  Team-shared data written by other CTAs is read
// with L2-only loads (__ldcg) after a team barrier (release/acquire fences).
// The arithmetic is FP64 throughout (FP32 A is widened exactly on load).
#include "batch.cuh"
#include "gridbar.cuh"
#include "rng.cuh"

#include <cooperative_groups.h>
#include <cfloat>

namespace cur {
namespace {

constexpr int kTB = 8;     // outputs per thread and pass in the residual products (the
                           // serving kernel's; the batch kernel takes 4 or 8, tuned per batch)
constexpr int kLch = 128;  // rows of L^T / Rt staged per shared-memory chunk
constexpr int kIch = 256;  // rows of A per sketch staging chunk
constexpr int kMaxWarps = 32;

// ---------------------------------------------------------------------------
// Teams and reductions
// ---------------------------------------------------------------------------
struct Team {
  GridBar* bar;     // this team's barrier (software teams)
  DevStatus* st;    // launch-wide status (timeouts)
  int T;            // CTAs in the team
  int rank;         // this CTA's rank in the team
  bool cluster;     // the team is a thread-block cluster (hardware barrier)
  __device__ int64_t gtid() const { return (int64_t)rank * blockDim.x + threadIdx.x; }
  __device__ int64_t gsize() const { return (int64_t)T * blockDim.x; }
  // All threads of all CTAs of the team; false on timeout, or when another CTA
  // recorded an error while this one waited.
  __device__ bool sync() const {
    if (T == 1) {
      __syncthreads();
      return true;
    }
    if (cluster) {  // barrier.cluster arrive.release / wait.acquire: the CTAs of a
                    // cluster are co-scheduled by the hardware, so this wait always ends
      cooperative_groups::this_cluster().sync();
      return true;
    }
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) s_ok = bar_arrive_wait(bar, (unsigned)T, st) ? 1 : 0;
    __syncthreads();
    return s_ok != 0;
  }
};

// The single-CTA "team" for private work (N^+): a plain block barrier.
__device__ __forceinline__ Team cta_team(const Team& t) {
  Team c = t;
  c.T = 1;
  c.rank = 0;
  c.cluster = false;
  return c;
}

// Sum over the CTA in a fixed order (warp tree, then warps in order); the
// result is returned to every thread.
__device__ double cta_sum(double v) {
  __shared__ double red[kMaxWarps];
  __shared__ double total;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    total = s;
  }
  __syncthreads();
  return total;
}

// Magnitude keys: the bit pattern of |x| orders like |x| for every non-NaN
// double, so pivot searches compare integers (an FP64 compare-and-select takes
// ~230 cycles on GB300, an integer one a few); NaN gets -2, below every number.
__device__ __forceinline__ long long mkey(double x) {
  const long long k = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL;
  return k > 0x7FF0000000000000LL ? -2 : k;
}

// (key, index) maximum: larger key wins, equal keys -> smaller index;
// index < 0 means "none".
__device__ __forceinline__ bool better(long long k1, int64_t i1, long long k2, int64_t i2) {
  if (i2 < 0) return i1 >= 0;
  if (i1 < 0) return false;
  return k1 > k2 || (k1 == k2 && i1 < i2);
}

__device__ void cta_argmax(long long& k, int64_t& idx) {
  __shared__ long long rk[kMaxWarps];
  __shared__ long long ri[kMaxWarps];
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_down_sync(0xffffffffu, k, o);
    const long long oi = __shfl_down_sync(0xffffffffu, (long long)idx, o);
    if (better(ok, oi, k, idx)) { k = ok; idx = oi; }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { rk[wid] = k; ri[wid] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long bk = rk[0];
    int64_t bi = ri[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (better(rk[w], ri[w], bk, bi)) { bk = rk[w]; bi = ri[w]; }
    rk[0] = bk;
    ri[0] = bi;
  }
  __syncthreads();
  k = rk[0];
  idx = ri[0];
  __syncthreads();
}

template <typename AT>
__device__ __forceinline__ double lda_(const AT* A, int64_t idx) { return (double)A[idx]; }

__device__ __forceinline__ double* dyn_smem() {
  extern __shared__ __align__(16) double batch_dyn_smem[];
  return batch_dyn_smem;
}

// Cycle accounting by the team leader (thread 0 of team rank 0).
struct PhaseClock {
  unsigned long long* prof;
  long long t;
  __device__ void lap(int ph) {
    if (!prof) return;
    const long long now = clock64();
    atomicAdd(prof + ph, (unsigned long long)(now - t));
    t = now;
  }
};

// ---------------------------------------------------------------------------
// LUPP (both selections of Algorithm 1) in one CTA, on a private copy.
// W holds nf feature rows of ncand candidates (W[t * ldw + i]); mask marks
// excluded candidates and receives the chosen ones.  Step t takes the
// eligible candidate of largest |W[t][i]| (ties: smallest index; all zero:
// smallest eligible, no elimination) and eliminates feature t from every
// other eligible candidate.  Returns false when no candidate is left.
// ---------------------------------------------------------------------------
__device__ bool cta_lupp(double* W, int64_t ldw, int nf, int64_t ncand, int steps, uint8_t* mask,
                         int64_t* piv, double* prow) {
  for (int t = 0; t < steps; ++t) {
    long long bk = -1;
    int64_t bi = -1;
    for (int64_t i = threadIdx.x; i < ncand; i += blockDim.x) {
      if (mask[i]) continue;
      const long long a = mkey(W[t * ldw + i]);
      if (a > bk) { bk = a; bi = i; }  // NaN (-2) never wins
    }
    cta_argmax(bk, bi);
    if (bi < 0) return false;
    if (threadIdx.x == 0) { piv[t] = bi; mask[bi] = 1; }
    if (bk > 0 && t + 1 < nf) {
      for (int u = t + 1 + threadIdx.x; u < nf; u += blockDim.x) prow[u] = W[u * ldw + bi];
      __syncthreads();
      const double pivv = W[t * ldw + bi];
      for (int64_t i = threadIdx.x; i < ncand; i += blockDim.x) {
        if (mask[i]) continue;
        const double l = W[t * ldw + i] / pivv;   // divided, as the oracle does
        for (int u = t + 1; u < nf; ++u) W[u * ldw + i] = W[u * ldw + i] - l * prow[u];
      }
    }
    __syncthreads();
  }
  return true;
}

// ---------------------------------------------------------------------------
// Generalised inverse by Householder QR with column pivoting (Businger-Golub,
// the "default QR" of Sec. 3.3), for a team of T CTAs.
// Mc: q columns of length p (Mc[col * p + i]); column col belongs to CTA
// col % T, which alone updates it.  Step j: the team picks the remaining
// column of largest norm over rows j..p-1 (exact norms, recomputed while the
// previous reflector is applied; ties -> smallest column), every CTA builds
// the reflector from it, and each owner applies it to its columns.  One team
// barrier per step.  After the loop, rank k = number of leading |R_jj| > thr,
// and X = P [R11^{-1} Q1^T; 0] (q x p, row stride ldx) column by column.
// ---------------------------------------------------------------------------

__device__ void qr_local_best(const Team& tm, const QrWs& w, int64_t q, double* slot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long bk = -1;
  int64_t bi = -1;
  for (int64_t col = tm.rank + (int64_t)tm.T * wid; col < q; col += (int64_t)tm.T * nw) {
    if (lane == 0 && !w.used[col]) {
      const long long k = mkey(w.norm2[col]);
      if (better(k, col, bk, bi)) { bk = k; bi = col; }
    }
  }
  cta_argmax(bk, bi);
  if (threadIdx.x == 0) { slot[0] = __longlong_as_double(bk); slot[1] = (double)bi; }
}

// Apply H_j = I - tau v v^T (v = vloc, rows j..p-1) to one column x of the
// trailing matrix with one warp, and return the column's squared norm over
// rows j+1..p-1 (the next pivot search needs it).  Columns of at most 32 R rows
// stay in registers between the dot product and the update (one pass over L2);
// longer ones take two passes with eight loads in flight per lane.
template <int R>
__device__ __forceinline__ double qr_col_apply_reg(double* x, const double* vloc, int64_t j,
                                                   int64_t p, double tau, int lane) {
  double y[R], v[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int64_t i = j + lane + 32 * t;
    y[t] = i < p ? __ldcg(x + i) : 0.0;
    v[t] = i < p ? vloc[i] : 0.0;
  }
  if (tau != 0.0) {
    double d = 0.0;
#pragma unroll
    for (int t = 0; t < R; ++t) d += v[t] * y[t];
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    const double f = tau * d;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int64_t i = j + lane + 32 * t;
      y[t] = y[t] - f * v[t];
      if (i < p) x[i] = y[t];
    }
  }
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int64_t i = j + lane + 32 * t;
    if (i > j && i < p) s += y[t] * y[t];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

__device__ __forceinline__ double qr_col_apply_l2(double* x, const double* vloc, int64_t j,
                                                  int64_t p, double tau, int lane) {
  double f = 0.0;
  if (tau != 0.0) {
    double d[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) d[u] = 0.0;
    int64_t i = j + lane;
    for (; i + 224 < p; i += 256) {
      double a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = __ldcg(x + i + 32 * u);
#pragma unroll
      for (int u = 0; u < 8; ++u) d[u] += vloc[i + 32 * u] * a[u];
    }
    for (; i < p; i += 32) d[0] += vloc[i] * __ldcg(x + i);
    double dd = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7]));
    for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
    f = tau * dd;
  }
  double sq[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) sq[u] = 0.0;
  int64_t i = j + lane;
  for (; i + 224 < p; i += 256) {
    double y[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) y[u] = __ldcg(x + i + 32 * u);
    if (tau != 0.0) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        y[u] = y[u] - f * vloc[i + 32 * u];
        x[i + 32 * u] = y[u];
      }
    }
    sq[0] += (i > j) ? y[0] * y[0] : 0.0;  // only the row i = j (lane 0, first block) is excluded
#pragma unroll
    for (int u = 1; u < 8; ++u) sq[u] += y[u] * y[u];
  }
  for (; i < p; i += 32) {
    double y = __ldcg(x + i);
    if (tau != 0.0) {
      y = y - f * vloc[i];
      x[i] = y;
    }
    if (i > j) sq[0] += y * y;
  }
  double s = ((sq[0] + sq[1]) + (sq[2] + sq[3])) + ((sq[4] + sq[5]) + (sq[6] + sq[7]));
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Factorisation; false on a team barrier failure.  Every read of Mc goes
// through L2 (__ldcg): the team's scratch is reused by jobs of other shapes,
// so a line cached in this SM's L1 may hold another CTA's older data.
__device__ bool team_qr_factor(const Team& tm, const QrWs& w, int64_t p, int64_t q, double* vloc) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t kmax = p < q ? p : q;
  __shared__ long long s_pc;
  // initial norms of the owned columns
  for (int64_t col = tm.rank + (int64_t)tm.T * wid; col < q; col += (int64_t)tm.T * nw) {
    const double* x = w.Mc + col * p;
    double s = 0.0;
    for (int64_t i = lane; i < p; i += 32) {
      const double xi = __ldcg(x + i);
      s += xi * xi;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) { w.norm2[col] = s; w.used[col] = 0; }
  }
  __syncthreads();
  qr_local_best(tm, w, q, w.slots + 2 * tm.rank);
  if (!tm.sync()) return false;

  for (int64_t j = 0; j < kmax; ++j) {
    const double* slot = w.slots + (j & 1) * 2 * tm.T;
    if (threadIdx.x < 32) {  // warp 0 reads the T candidates, all loads in flight together
      long long bk = -1;
      int64_t bi = -1;
      constexpr int kR = 8;
      long long cv[kR];
      double ci[kR];
#pragma unroll
      for (int u = 0; u < kR; ++u) {
        const int r = threadIdx.x + 32 * u;
        cv[u] = r < tm.T ? __double_as_longlong(__ldcg(slot + 2 * r)) : -1;
        ci[u] = r < tm.T ? __ldcg(slot + 2 * r + 1) : -1.0;
      }
#pragma unroll
      for (int u = 0; u < kR; ++u)
        if (better(cv[u], (int64_t)ci[u], bk, bi)) { bk = cv[u]; bi = (int64_t)ci[u]; }
      for (int r = threadIdx.x + 32 * kR; r < tm.T; r += 32) {  // teams above 256 CTAs
        const long long k = __double_as_longlong(__ldcg(slot + 2 * r));
        const int64_t i = (int64_t)__ldcg(slot + 2 * r + 1);
        if (better(k, i, bk, bi)) { bk = k; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {  // (key, index) max is order independent
        const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, (long long)bi, o);
        if (better(ok, oi, bk, bi)) { bk = ok; bi = oi; }
      }
      if (threadIdx.x == 0) s_pc = bi;
    }
    __syncthreads();
    const int64_t pc = s_pc;
    if (pc < 0) return false;  // no column left (uniform: every CTA read the same slots)
    // the pivot column, rows j..p-1, into this CTA's reflector buffer
    double tail = 0.0;
    const double* xc = w.Mc + pc * p;
    for (int64_t i = j + threadIdx.x; i < p; i += blockDim.x) {
      double x = __ldcg(xc + i);
      vloc[i] = x;
      if (i > j) tail += x * x;
    }
    tail = cta_sum(tail);
    __shared__ double s_tau, s_alpha;
    if (threadIdx.x == 0) {  // the reflector's scalars, once (sqrt and divide are costly in FP64)
      const double x0 = vloc[j];
      const double normx = sqrt(x0 * x0 + tail);
      double tau = 0.0, alpha = x0;
      if (normx != 0.0) {
        alpha = (x0 >= 0.0) ? -normx : normx;
        const double v0 = x0 - alpha;
        tau = 2.0 / (v0 * v0 + tail);
        vloc[j] = v0;
      }
      s_tau = tau;
      s_alpha = alpha;
    }
    __syncthreads();
    const double tau = s_tau, alpha = s_alpha;
    if (tm.rank == 0) {
      for (int64_t i = j + threadIdx.x; i < p; i += blockDim.x) w.V[j * p + i] = vloc[i];
      if (threadIdx.x == 0) { w.tau[j] = tau; w.rdiag[j] = alpha; w.perm[j] = pc; }
    }
    if (pc % tm.T == tm.rank && threadIdx.x == 0) w.used[pc] = 1;
    __syncthreads();
    // apply H_j to the owned remaining columns, recomputing their norms over j+1..p-1
    for (int64_t col = tm.rank + (int64_t)tm.T * wid; col < q; col += (int64_t)tm.T * nw) {
      if (w.used[col]) continue;
      double* x = w.Mc + col * p;
      const int64_t len = p - j;
      double s;
      if (len <= 4 * 32) s = qr_col_apply_reg<4>(x, vloc, j, p, tau, lane);
      else if (len <= 8 * 32) s = qr_col_apply_reg<8>(x, vloc, j, p, tau, lane);
      else if (len <= 24 * 32) s = qr_col_apply_reg<24>(x, vloc, j, p, tau, lane);
      else s = qr_col_apply_l2(x, vloc, j, p, tau, lane);
      if (lane == 0) w.norm2[col] = s;
    }
    __syncthreads();
    qr_local_best(tm, w, q, w.slots + ((j + 1) & 1) * 2 * tm.T + 2 * tm.rank);
    if (!tm.sync()) return false;
  }
  return true;
}

// Numerical rank after a factorisation: the number of leading |R_jj| > thr
// (thr < 0: max(p,q) 2^-52 |R_00|).  Same value in every thread.
// rinv (this CTA's buffer, >= kmax entries) receives 1 / R_jj for j < k.
__device__ int64_t qr_rank(const QrWs& w, int64_t p, int64_t q, double thr, double* rinv) {
  __shared__ long long s_k;
  const int64_t kmax = p < q ? p : q;
  if (threadIdx.x == 0) {
    const double r00 = kmax > 0 ? fabs(__ldcg(w.rdiag)) : 0.0;
    double t = thr;
    if (t < 0.0) t = kmax > 0 ? (double)(p > q ? p : q) * DBL_EPSILON * r00 : 0.0;
    int64_t k = 0;
    while (k < kmax && fabs(__ldcg(w.rdiag + k)) > t) ++k;
    s_k = k;
  }
  __syncthreads();
  const int64_t k = s_k;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) rinv[i] = 1.0 / __ldcg(w.rdiag + i);
  __syncthreads();
  return k;
}

// X = P [R11^{-1} Q1^T; 0] (q x p, row stride ldx): column `col` of Q^T is
// H_{k-1} ... H_0 e_col, then back substitution with R11, then the rows are
// scattered by the pivots.  One thread per column of X.
__device__ void team_qr_solve(const Team& tm, const QrWs& w, int64_t p, int64_t q, int64_t k,
                              double* X, int64_t ldx, const double* rinv) {
  for (int64_t col = tm.gtid(); col < p; col += tm.gsize()) {
    double* z = w.QT + col;  // z[i * p], this thread's alone
    for (int64_t i = 0; i < p; ++i) z[i * p] = (i == col) ? 1.0 : 0.0;
    for (int64_t jj = 0; jj < k; ++jj) {
      const double t = __ldcg(w.tau + jj);
      if (t == 0.0) continue;
      const double* v = w.V + jj * p;
      double d = 0.0;
      for (int64_t i = jj; i < p; ++i) d += __ldcg(v + i) * z[i * p];
      const double f = t * d;
      for (int64_t i = jj; i < p; ++i) z[i * p] = z[i * p] - f * __ldcg(v + i);
    }
    for (int64_t i = k - 1; i >= 0; --i) {
      double s = z[i * p];
      for (int64_t l = i + 1; l < k; ++l) {
        const int64_t pl = __ldcg(w.perm + l);
        s = s - __ldcg(w.Mc + pl * p + i) * z[l * p];
      }
      z[i * p] = s * rinv[i];
    }
    for (int64_t row = 0; row < q; ++row) X[row * ldx + col] = 0.0;
    for (int64_t i = 0; i < k; ++i) X[__ldcg(w.perm + i) * ldx + col] = z[i * p];
  }
}

// The same solve with PW right-hand sides of X resident in shared memory
// (Zs: PW columns of length p, column-major), panels spread over the team's
// CTAs.  Each reflector is read once per panel and applied with two block
// barriers; the back substitution runs column-oriented (R's column perm[i] is
// contiguous in Mc) with one block barrier per row.  Each of the block's
// threads owns at most PR rows (p <= PR * blockDim.x).
// Panel widths: the widest that fits the dynamic shared memory, with the rows
// per thread that 160 KB of panel gives 256 threads at that width.
__host__ __device__ inline int panel_rows(int pw) { return pw == 8 ? 10 : pw == 4 ? 20 : 40; }
__host__ __device__ inline int panel_width(int64_t p, size_t bytes, int threads) {
  for (int pw = 8; pw >= 2; pw >>= 1)
    if ((size_t)p * pw * sizeof(double) <= bytes && p <= (int64_t)panel_rows(pw) * threads)
      return pw;
  return 0;
}
static_assert((size_t)10 * 256 * 8 * sizeof(double) >= kBatchMaxPanelBytes &&
                  (size_t)20 * 256 * 4 * sizeof(double) >= kBatchMaxPanelBytes &&
                  (size_t)40 * 256 * 2 * sizeof(double) >= kBatchMaxPanelBytes,
              "at each width, every core that fits the panel has at most panel_rows rows per thread");

// Warp sums of PW values at once by a reduce-scatter butterfly: at each of the
// first log2(PW) levels a lane keeps half of its values and adds its partner's
// other half, then the single remaining value is summed over the lanes left;
// PW - 1 + log2(32 / PW) shuffle-adds instead of 5 PW (the FP64 adds share the
// narrow FP64 pipe with the solve's FMAs).  Every lane returns the warp total
// of component scatter_component<PW>(lane).
template <int PW>
__device__ __forceinline__ double warp_sum_scatter(double (&v)[PW], int lane) {
  int off = 16;
#pragma unroll
  for (int w = PW; w > 1; w >>= 1) {
    const int h = w >> 1;
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const double keep = hi ? v[h + k] : v[k];
      const double give = hi ? v[k] : v[h + k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, give, off);
    }
    off >>= 1;
  }
  double s = v[0];
  for (; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

template <int PW>
__device__ __forceinline__ int scatter_component(int lane) {
  int c = 0, off = 16;
#pragma unroll
  for (int w = PW; w > 1; w >>= 1) {
    if (lane & off) c += w >> 1;
    off >>= 1;
  }
  return c;
}

template <int PW, int PR>
__device__ void team_qr_solve_panel(const Team& tm, const QrWs& w, int64_t p, int64_t q, int64_t k,
                                    double* X, int64_t ldx, double* Zs, const double* rinv) {
  __shared__ double s_red[kMaxWarps][PW];
  __shared__ double s_d[PW];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int NT = blockDim.x;
  const int64_t npanel = (p + PW - 1) / PW;
  for (int64_t g = tm.rank; g < npanel; g += tm.T) {
    const int64_t c0 = g * PW;
    const int wc = (int)min((int64_t)PW, p - c0);
    for (int64_t e = tid; e < p * PW; e += NT) {
      const int64_t c = e / p, i = e - c * p;
      Zs[e] = (c < wc && i == c0 + c) ? 1.0 : 0.0;
    }
    for (int64_t e = tid; e < q * wc; e += NT) {
      const int64_t row = e / wc, c = e - row * wc;
      X[row * ldx + c0 + c] = 0.0;
    }
    __syncthreads();
    for (int64_t jj = 0; jj < k; ++jj) {
      const double t = __ldcg(w.tau + jj);
      if (t == 0.0) continue;
      const double* v = w.V + jj * p;
      double acc[PW];
#pragma unroll
      for (int c = 0; c < PW; ++c) acc[c] = 0.0;
      // rows stay with thread i % NT for every reflector, so each row of the
      // panel is only ever touched by one thread (no barrier between the
      // update of H_jj and the dot of H_jj+1); the reflector's entries of this
      // thread's rows are loaded once (all in flight together) and reused by
      // the update
      const int64_t i0 = (jj / NT) * NT + tid;
      double vr[PR];
#pragma unroll
      for (int q = 0; q < PR; ++q) {
        const int64_t i = i0 + (int64_t)q * NT;
        vr[q] = (i >= jj && i < p) ? __ldcg(v + i) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < PR; ++q) {
        const int64_t i = i0 + (int64_t)q * NT;
        if (i < jj || i >= p) continue;
#pragma unroll
        for (int c = 0; c < PW; ++c) acc[c] += vr[q] * Zs[c * p + i];
      }
      const double tot = warp_sum_scatter<PW>(acc, lane);
      if ((lane & (32 / PW - 1)) == 0) s_red[wid][scatter_component<PW>(lane)] = tot;
      __syncthreads();
      if (tid < PW) {
        double sum = 0.0;
        for (int w2 = 0; w2 < nw; ++w2) sum += s_red[w2][tid];
        s_d[tid] = t * sum;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < PR; ++q) {
        const int64_t i = i0 + (int64_t)q * NT;
        if (i < jj || i >= p) continue;
#pragma unroll
        for (int c = 0; c < PW; ++c) Zs[c * p + i] -= s_d[c] * vr[q];
      }
    }
    for (int64_t i = k - 1; i >= 0; --i) {
      __syncthreads();
      const double ri = rinv[i];
      const int64_t pi = __ldcg(w.perm + i);
      double zi[PW];
#pragma unroll
      for (int c = 0; c < PW; ++c) zi[c] = Zs[c * p + i] * ri;
      const double* Rcol = w.Mc + pi * p;  // R(l, i) for l < i
      for (int64_t l = tid; l < i; l += NT) {
        const double rl = __ldcg(Rcol + l);
#pragma unroll
        for (int c = 0; c < PW; ++c) Zs[c * p + l] -= rl * zi[c];
      }
      if (tid == 0)
        for (int c = 0; c < wc; ++c) X[pi * ldx + c0 + c] = zi[c];
    }
    __syncthreads();
  }
}

// Solve with the widest shared-memory panel that fits `panel_bytes`, else the
// unpanelled solve (which needs the p x p QT scratch).
__device__ void team_qr_solve_best(const Team& tm, const QrWs& w, int64_t p, int64_t q, int64_t k,
                                   double* X, int64_t ldx, size_t panel_bytes, const double* rinv) {
  switch (panel_width(p, panel_bytes, (int)blockDim.x)) {
    case 8: team_qr_solve_panel<8, 10>(tm, w, p, q, k, X, ldx, dyn_smem(), rinv); break;
    case 4: team_qr_solve_panel<4, 20>(tm, w, p, q, k, X, ldx, dyn_smem(), rinv); break;
    case 2: team_qr_solve_panel<2, 40>(tm, w, p, q, k, X, ldx, dyn_smem(), rinv); break;
    default: team_qr_solve(tm, w, p, q, k, X, ldx, rinv);
  }
}

// ---------------------------------------------------------------------------
// One job.
// ---------------------------------------------------------------------------
template <typename AT, int TB>
__device__ void run_job(const BatchParams& P, const Team& tm, const BatchJobDev& jb,
                        BatchOutDev* out, const TeamWs& tw, const CtaWs& cw) {
  __shared__ double s_stage[kLch * TB > 8 * kIch ? kLch * TB : 8 * kIch];
  __shared__ double s_prow[kBatchMaxB > kBatchMaxC ? kBatchMaxB : kBatchMaxC];
  __shared__ int64_t s_Jk[kBatchMaxB], s_Ik[kBatchMaxB];
  const int tid = threadIdx.x, NT = blockDim.x;
  const AT* A = static_cast<const AT*>(jb.A);
  const int64_t m = jb.m, n = jb.n, lda = jb.lda, c = jb.c, b = jb.b, rmax = jb.rmax;
  int64_t* Iout = P.Iout + jb.off_ij;
  int64_t* Jout = P.Jout + jb.off_j;
  double* Uout = P.Uout + jb.off_u;
  double* G = tw.G;      // c x m
  double* S = tw.S;      // c x n
  double* SrowT = tw.SrowT;  // b x m
  double* Lt = tw.Lt;    // rmax x m
  double* Rt = tw.Rt;    // rmax x n

  PhaseClock pc{(P.prof && tm.rank == 0 && tid == 0) ? P.prof : nullptr, clock64()};
  const long long t_job = clock64();
  // private state
  for (int64_t i = tid; i < n; i += NT) cw.maskc[i] = 0;
  for (int64_t i = tid; i < m; i += NT) cw.maskr[i] = 0;

  // ---- sketch matrix G (c x m), Philox blocks of four entries -------------
  const int64_t bpr = (m + 3) / 4;
  for (int64_t g = tm.gtid(); g < c * bpr; g += tm.gsize()) {
    const int64_t i = g / bpr, qb = g - i * bpr;
    double z[4];
    gaussian_block(jb.seed, i, qb, z);
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (4 * qb + t < m) G[i * m + 4 * qb + t] = z[t];
  }
  if (!tm.sync()) return;

  // ---- initial sketch S = Y = G A, ||Y||_F ---------------------------------
  double ss = 0.0;
  for (int64_t j0 = (int64_t)tm.rank * NT; j0 < n; j0 += tm.gsize()) {
    const int64_t j = j0 + tid;
    for (int64_t q0 = 0; q0 < c; q0 += 8) {
      const int nq = (int)min((int64_t)8, c - q0);
      double acc[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t] = 0.0;
      for (int64_t i0 = 0; i0 < m; i0 += kIch) {
        const int ni = (int)min((int64_t)kIch, m - i0);
        __syncthreads();
        for (int e = tid; e < 8 * kIch; e += NT) {
          const int t = e / kIch, ii = e - t * kIch;
          s_stage[e] = (t < nq && ii < ni) ? __ldcg(G + (q0 + t) * m + i0 + ii) : 0.0;
        }
        __syncthreads();
        if (j < n) {
          for (int ii = 0; ii < ni; ++ii) {
            const double a = lda_(A, (i0 + ii) * lda + j);
#pragma unroll
            for (int t = 0; t < 8; ++t) acc[t] += s_stage[t * kIch + ii] * a;
          }
        }
      }
      if (j < n)
        for (int t = 0; t < nq; ++t) {
          S[(q0 + t) * n + j] = acc[t];
          ss += acc[t] * acc[t];
        }
    }
  }
  ss = cta_sum(ss);
  if (tid == 0) tw.parts[tm.rank] = ss;
  if (!tm.sync()) return;
  double nY2 = 0.0;
  for (int r = 0; r < tm.T; ++r) nY2 += __ldcg(tw.parts + r);
  const double nY = sqrt(nY2);
  pc.lap(0);

  double rho = 1.0;
  int64_t r = 0, iters = 0;
  int status = 0;
  double thr_scale = -1.0;
  if (!isfinite(nY)) {
    status = 2;  // CUR_ENONFINITE
  } else if (nY == 0.0) {
    rho = 0.0;
  }

  // ---- the loop of Algorithm 1 --------------------------------------------------
  while (status == 0 && rho > jb.tol && r < rmax) {
    const int bk = (int)min(b, rmax - r);
    // column selection: J_k = LUPP(S), privately
    for (int64_t e = tid; e < c * n; e += NT) cw.W[e] = __ldcg(S + e);
    __syncthreads();
    if (!cta_lupp(cw.W, n, (int)c, n, bk, cw.maskc, s_Jk, s_prow)) { status = 5; break; }
    __syncthreads();
    // S(:, J_k) for the sketched update (read before anyone updates S)
    for (int e = tid; e < (int)c * bk; e += NT) {
      const int qq = e / bk, t = e - qq * bk;
      cw.SJ[e] = __ldcg(S + qq * n + s_Jk[t]);
    }
    pc.lap(1);
    // row residual: S^row = A(:,J_k) - L Rt(:,J_k), rows over the team
    for (int64_t i0 = (int64_t)tm.rank * NT; i0 < m; i0 += tm.gsize()) {
      const int64_t i = i0 + tid;
      for (int t0 = 0; t0 < bk; t0 += TB) {
        const int nt = min(TB, bk - t0);
        double acc[TB];
#pragma unroll
        for (int t = 0; t < TB; ++t) acc[t] = 0.0;
        for (int64_t l0 = 0; l0 < r; l0 += kLch) {
          const int nl = (int)min((int64_t)kLch, r - l0);
          __syncthreads();
          for (int e = tid; e < kLch * TB; e += NT) {
            const int ll = e / TB, t = e - ll * TB;
            s_stage[e] = (ll < nl && t < nt) ? __ldcg(Rt + (l0 + ll) * n + s_Jk[t0 + t]) : 0.0;
          }
          __syncthreads();
          if (i < m) {
            for (int ll = 0; ll < nl; ++ll) {
              const double a = __ldcg(Lt + (l0 + ll) * m + i);
#pragma unroll
              for (int t = 0; t < TB; ++t) acc[t] += a * s_stage[ll * TB + t];
            }
          }
        }
        if (i < m)
          for (int t = 0; t < nt; ++t)
            SrowT[(t0 + t) * m + i] = lda_(A, i * lda + s_Jk[t0 + t]) - acc[t];
      }
    }
    if (!tm.sync()) { status = 6; break; }
    pc.lap(2);

    // row selection: I_k = LUPP(S^row), privately
    for (int64_t e = tid; e < (int64_t)bk * m; e += NT) cw.W[e] = __ldcg(SrowT + e);
    __syncthreads();
    if (!cta_lupp(cw.W, m, bk, m, bk, cw.maskr, s_Ik, s_prow)) { status = 5; break; }
    __syncthreads();
    const int64_t rn = r + bk;
    // N = S^row(I_k, :) (bk x bk), columns t contiguous; N^+ privately
    for (int e = tid; e < bk * bk; e += NT) {
      const int t = e / bk, a = e - t * bk;
      cw.qr.Mc[e] = __ldcg(SrowT + t * m + s_Ik[a]);
    }
    __syncthreads();
    {
      // the rank threshold scales with |R_00| of the first block's core and
      // with the current rank (Sec. 3.3): thr = 2^-52 |R_00(N_1)| (r + b_k)
      const Team ct = cta_team(tm);
      team_qr_factor(ct, cw.qr, bk, bk, cw.vloc);
      if (thr_scale < 0.0) thr_scale = fabs(cw.qr.rdiag[0]) * DBL_EPSILON;
      const int64_t kN = qr_rank(cw.qr, bk, bk, thr_scale * (double)rn, cw.vloc);
      team_qr_solve(ct, cw.qr, bk, bk, kN, cw.Np, bk, cw.vloc);
      __syncthreads();
    }
    // T1 = S(:,J_k) N^+ (c x bk), privately
    for (int e = tid; e < (int)c * bk; e += NT) {
      const int qq = e / bk, a = e - qq * bk;
      double s = 0.0;
      for (int t = 0; t < bk; ++t) s = s + cw.SJ[qq * bk + t] * cw.Np[t * bk + a];
      cw.T1[e] = s;
    }
    pc.lap(3);
    // L_k = S^row N^+ into rows r..r+bk-1 of L^T, rows over the team
    for (int64_t i = tm.gtid(); i < m; i += tm.gsize()) {
      for (int a = 0; a < bk; ++a) {
        double s = 0.0;
        for (int t = 0; t < bk; ++t) s = s + __ldcg(SrowT + t * m + i) * cw.Np[t * bk + a];
        Lt[(r + a) * m + i] = s;
      }
    }
    __syncthreads();
    // Rt_k = A(I_k,:) - L(I_k,:) Rt and S -= T1 Rt_k, columns over the team
    double ssum = 0.0;
    for (int64_t j0 = (int64_t)tm.rank * NT; j0 < n; j0 += tm.gsize()) {
      const int64_t j = j0 + tid;
      for (int a0 = 0; a0 < bk; a0 += TB) {
        const int na = min(TB, bk - a0);
        double acc[TB];
#pragma unroll
        for (int a = 0; a < TB; ++a) acc[a] = 0.0;
        for (int64_t l0 = 0; l0 < r; l0 += kLch) {
          const int nl = (int)min((int64_t)kLch, r - l0);
          __syncthreads();
          for (int e = tid; e < kLch * TB; e += NT) {
            const int ll = e / TB, a = e - ll * TB;
            s_stage[e] = (ll < nl && a < na) ? __ldcg(Lt + (l0 + ll) * m + s_Ik[a0 + a]) : 0.0;
          }
          __syncthreads();
          if (j < n) {
            for (int ll = 0; ll < nl; ++ll) {
              const double rv = __ldcg(Rt + (l0 + ll) * n + j);
#pragma unroll
              for (int a = 0; a < TB; ++a) acc[a] += s_stage[ll * TB + a] * rv;
            }
          }
        }
        if (j < n)
          for (int a = 0; a < na; ++a)
            Rt[(r + a0 + a) * n + j] = lda_(A, s_Ik[a0 + a] * lda + j) - acc[a];
      }
      if (j < n) {
        for (int64_t qq = 0; qq < c; ++qq) {
          double s = 0.0;
          for (int a = 0; a < bk; ++a) s = s + cw.T1[qq * bk + a] * Rt[(r + a) * n + j];
          const double y = S[qq * n + j] - s;
          S[qq * n + j] = y;
          ssum += y * y;
        }
      }
    }
    ssum = cta_sum(ssum);
    if (tid == 0) tw.parts[tm.rank] = ssum;
    if (tm.rank == 0)
      for (int a = tid; a < bk; a += NT) { Iout[r + a] = s_Ik[a]; Jout[r + a] = s_Jk[a]; }
    if (!tm.sync()) { status = 6; break; }
    pc.lap(4);
    double s2 = 0.0;
    for (int q = 0; q < tm.T; ++q) s2 += __ldcg(tw.parts + q);
    r = rn;
    rho = sqrt(s2) / nY;
    ++iters;
    if (tm.rank == 0 && tid == 0 && P.rho_hist)
      P.rho_hist[jb.off_hist + iters - 1] = rho;
  }

  // ---- core at exit: U = A(I,J)^+ -------------------------------------------------
  if (status == 0 && r > 0) {
    for (int64_t e = tm.gtid(); e < r * r; e += tm.gsize()) {
      const int64_t col = e / r, i = e - col * r;
      tw.qr.Mc[e] = lda_(A, __ldcg(Iout + i) * lda + __ldcg(Jout + col));
    }
    if (!tm.sync()) status = 6;
    if (status == 0 && !team_qr_factor(tm, tw.qr, r, r, cw.vloc)) status = 6;
    pc.lap(5);
    if (status == 0) {
      const int64_t k = qr_rank(tw.qr, r, r, -1.0, cw.vloc);
      team_qr_solve_best(tm, tw.qr, r, r, k, Uout, r, P.panel_bytes, cw.vloc);
    }
  }
  if (status == 0 && rho > jb.tol) status = 7;  // CUR_TOL_UNREACHED
  if (tm.rank == 0 && tid == 0) {
    out->rank = r;
    out->iters = iters;
    out->rho = rho;
    out->normY = nY;
    out->status = status;
  }
  tm.sync();
  pc.lap(6);
  if (pc.prof) atomicAdd(pc.prof + 7, 1ULL);
  if (tm.rank == 0 && tid == 0) out->cycles = clock64() - t_job;
}

// Two team classes: the first nbig teams have team_big CTAs and take the
// queue positions [0, big_cut) (the largest jobs: the queue is ordered by
// estimated work), then help with the rest; the other teams have `team` CTAs
// and take positions [big_cut, njobs) only.  A job's team size is thus set by
// its class, and the largest jobs no longer hold a small team to the end.
template <typename AT, int TB>
__global__ void __launch_bounds__(256, 1) batch_kernel(BatchParams P) {
  const int bigctas = P.nbig * P.team_big;
  const bool big = (int)blockIdx.x < bigctas;
  const int T = big ? P.team_big : P.team;
  const int local = big ? (int)blockIdx.x : (int)blockIdx.x - bigctas;
  const int team = big ? local / T : P.nbig + local / T;
  Team tm;
  tm.T = T;
  tm.rank = local % T;
  tm.st = P.st;
  tm.cluster = false;
  char* tbase = P.team_scratch + (size_t)team * P.team_bytes;
  TeamWs tw = carve_team(tbase, P.dims, T);
  tm.bar = tw.bar;
  CtaWs cw = carve_cta(P.cta_scratch + (size_t)blockIdx.x * P.cta_bytes, P.dims);
  __shared__ long long s_job;
  for (;;) {
    if (tm.rank == 0 && threadIdx.x == 0) {
      long long pos = big ? (long long)atomicAdd(P.next, 1ULL) : P.big_cut;
      if (pos >= P.big_cut) pos = P.big_cut + (long long)atomicAdd(P.next_small, 1ULL);
      *tw.job_slot = pos;
    }
    if (!tm.sync()) return;
    if (threadIdx.x == 0) s_job = __ldcg(tw.job_slot);
    __syncthreads();
    const long long pos = s_job;
    if (pos >= P.njobs) return;
    const int jid = P.order[pos];
    BatchJobDev jb = P.jobs[jid];
    run_job<AT, TB>(P, tm, jb, P.out + jid, tw, cw);
    if (*((volatile int*)&P.st->err) != 0) return;
  }
}

// Whole-GPU core solve: U = A(I,J)^+ (or any p x q generalised inverse) by
// one team made of the whole grid, for the single-matrix path's large cores.
__global__ void __launch_bounds__(256, 1) core_qr_kernel(CoreQrParams P) {
  Team tm;
  tm.bar = P.bar;
  tm.st = P.st;
  tm.T = (int)gridDim.x;
  tm.rank = (int)blockIdx.x;
  tm.cluster = false;
  double* vloc = P.vloc + (size_t)blockIdx.x * P.vloc_stride;
  if (!team_qr_factor(tm, P.w, P.p, P.q, vloc)) return;
  const int64_t k = qr_rank(P.w, P.p, P.q, P.thr, vloc);
  team_qr_solve_best(tm, P.w, P.p, P.q, k, P.X, P.ldx, P.panel_bytes, vloc);
  if (blockIdx.x == 0 && threadIdx.x == 0 && P.rank_out) *P.rank_out = k;
}

// Serving form: one thread-block cluster of T CTAs per job (blocks
// [jid T, (jid + 1) T) along x), every job with its own workspace (team part,
// T CTA parts), so launches of different waves can run concurrently.
template <typename AT>
__global__ void __launch_bounds__(256, 1) serve_kernel(BatchParams P) {
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  Team tm;
  tm.T = (int)cl.num_blocks();
  tm.rank = (int)cl.block_rank();
  tm.st = P.st;
  tm.cluster = true;
  tm.bar = nullptr;
  const long long jid = blockIdx.x / tm.T;
  if (jid >= P.njobs) return;  // whole clusters only: uniform within the cluster
  const BatchJobDev jb = P.jobs[jid];
  const BatchDims d{jb.m, jb.n, jb.c, jb.b, jb.rmax};
  const BatchLayout L = batch_layout_dev(d, tm.T);
  const size_t tb = (L.team_bytes + 255) & ~(size_t)255, cb = (L.cta_bytes + 255) & ~(size_t)255;
  TeamWs tw = carve_team(jb.ws, d, tm.T);
  CtaWs cw = carve_cta(jb.ws + tb + (size_t)tm.rank * cb, d);
  run_job<AT, kTB>(P, tm, jb, P.out + jid, tw, cw);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <typename AT, int TB>
static int max_ctas_tb(const LaunchEnv& env, int threads, size_t dyn_smem) {
  if (cudaFuncSetAttribute(batch_kernel<AT, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kBatchMaxPanelBytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<AT, TB>, threads,
                                                    dyn_smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * env.num_sms;
}

// CTAs every tile variant of the batch kernel can keep co-resident.
template <typename AT>
static int max_ctas_t(const LaunchEnv& env, int threads, size_t dyn_smem) {
  const int a = max_ctas_tb<AT, 4>(env, threads, dyn_smem);
  const int b = max_ctas_tb<AT, 8>(env, threads, dyn_smem);
  return a < b ? a : b;
}

int batch_max_ctas(const LaunchEnv& env, int threads, bool a_f32, size_t dyn_smem) {
  return a_f32 ? max_ctas_t<float>(env, threads, dyn_smem)
               : max_ctas_t<double>(env, threads, dyn_smem);
}

size_t batch_panel_bytes(int64_t rmax) {
  const int pw = panel_width(rmax, kBatchMaxPanelBytes, 256);
  return (size_t)rmax * pw * sizeof(double);
}

cudaError_t launch_batch(const LaunchEnv& env, const BatchParams& P, int grid, int threads,
                         bool a_f32) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = P.panel_bytes;
  cfg.stream = env.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (P.tile_n == 4)
    return a_f32 ? cudaLaunchKernelEx(&cfg, batch_kernel<float, 4>, P)
                 : cudaLaunchKernelEx(&cfg, batch_kernel<double, 4>, P);
  return a_f32 ? cudaLaunchKernelEx(&cfg, batch_kernel<float, 8>, P)
               : cudaLaunchKernelEx(&cfg, batch_kernel<double, 8>, P);
}

}  // namespace cur

namespace cur {

size_t serve_job_scratch_bytes(const BatchDims& d, int team) {
  const BatchLayout L = batch_layout_dev(d, team);
  const size_t tb = (L.team_bytes + 255) & ~(size_t)255, cb = (L.cta_bytes + 255) & ~(size_t)255;
  return tb + (size_t)team * cb;
}

template <typename AT>
static cudaError_t serve_attr(size_t panel) {
  cudaError_t e = cudaFuncSetAttribute(serve_kernel<AT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBatchMaxPanelBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(serve_kernel<AT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  (void)panel;
  return e;
}

int serve_max_clusters(const LaunchEnv& env, int team, bool a_f32, size_t panel) {
  cudaError_t e = a_f32 ? serve_attr<float>(panel) : serve_attr<double>(panel);
  if (e != cudaSuccess) { cudaGetLastError(); return 0; }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)team);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = panel;
  cfg.stream = env.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)team;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  e = a_f32 ? cudaOccupancyMaxActiveClusters(&n, serve_kernel<float>, &cfg)
            : cudaOccupancyMaxActiveClusters(&n, serve_kernel<double>, &cfg);
  if (e != cudaSuccess) { cudaGetLastError(); return 0; }
  return n;
}

cudaError_t launch_serve(const LaunchEnv& env, const BatchParams& P, int team, bool a_f32) {
  if (P.njobs <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(P.njobs * team));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = P.panel_bytes;
  cfg.stream = env.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)team;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (a_f32) return cudaLaunchKernelEx(&cfg, serve_kernel<float>, P);
  return cudaLaunchKernelEx(&cfg, serve_kernel<double>, P);
}

}  // namespace cur

namespace cur {

size_t core_qr_work_bytes(int64_t p, int64_t q, int T) {
  const int64_t kmax = p < q ? p : q;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t b = al(sizeof(double) * (size_t)(q * p));                       // Mc
  b += al(sizeof(double) * (size_t)(kmax * p));                           // V
  if (batch_panel_bytes(p) == 0) b += al(sizeof(double) * (size_t)(p * p));  // QT
  b += 3 * al(sizeof(double) * (size_t)kmax) + al(8 * (size_t)kmax);      // tau, rdiag, perm
  b += al((size_t)q) + al(sizeof(double) * (size_t)q);                   // used, norm2
  b += al(sizeof(double) * 4 * (size_t)T);                                // slots
  b += al(sizeof(double) * (size_t)(p > q ? p : q)) * (size_t)T;          // vloc per CTA
  b += al(sizeof(GridBar)) + al(sizeof(long long));
  return b;
}

int core_qr_grid(const LaunchEnv& env, int64_t p) {
  const size_t panel = batch_panel_bytes(p);
  if (cudaFuncSetAttribute(core_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kBatchMaxPanelBytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, core_qr_kernel, 256, panel) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm >= 1 ? env.num_sms : 0;   // one CTA per SM
}

cudaError_t launch_core_qr(const LaunchEnv& env, double* Mc, int64_t p, int64_t q, double thr,
                           double* X, int64_t ldx, void* work, int T, DevStatus* st,
                           int64_t* rank_out) {
  const int64_t kmax = p < q ? p : q;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* b = static_cast<char*>(work);
  auto take = [&](size_t x) { char* r = b; b += al(x); return r; };
  CoreQrParams P;
  P.w.Mc = Mc;
  (void)take(sizeof(double) * (size_t)(q * p));   // Mc lives at the start of the work area
  P.w.V = reinterpret_cast<double*>(take(sizeof(double) * (size_t)(kmax * p)));
  const size_t panel = batch_panel_bytes(p);
  P.w.QT = panel ? nullptr : reinterpret_cast<double*>(take(sizeof(double) * (size_t)(p * p)));
  P.w.tau = reinterpret_cast<double*>(take(sizeof(double) * (size_t)kmax));
  P.w.rdiag = reinterpret_cast<double*>(take(sizeof(double) * (size_t)kmax));
  (void)take(sizeof(double) * (size_t)kmax);
  P.w.perm = reinterpret_cast<int64_t*>(take(8 * (size_t)kmax));
  P.w.used = reinterpret_cast<uint8_t*>(take((size_t)q));
  P.w.norm2 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)q));
  P.w.slots = reinterpret_cast<double*>(take(sizeof(double) * 4 * (size_t)T));
  P.vloc_stride = al(sizeof(double) * (size_t)(p > q ? p : q)) / sizeof(double);
  P.vloc = reinterpret_cast<double*>(take(sizeof(double) * P.vloc_stride * (size_t)T));
  P.bar = reinterpret_cast<GridBar*>(take(sizeof(GridBar)));
  P.p = p;
  P.q = q;
  P.thr = thr;
  P.X = X;
  P.ldx = ldx;
  P.st = st;
  P.panel_bytes = panel;
  P.rank_out = rank_out;
  cudaError_t e = cudaMemsetAsync(P.bar, 0, sizeof(GridBar), env.stream);
  if (e != cudaSuccess) return e;
  void* args[] = {&P};
  return cudaLaunchCooperativeKernel((const void*)core_qr_kernel, dim3(T), dim3(256), args, panel,
                                     env.stream);
}

}  // namespace cur
