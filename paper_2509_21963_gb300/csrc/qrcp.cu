// qrcp.cu -- core solve of IterativeCUR (arXiv 2509.21963, Algorithm 1: the
// core U = A(I,J)^+ by the paper's default QR): generalised inverse of a p x q matrix
// by Householder QR with column pivoting (Businger & Golub 1965),
//   M P = Q R,  k = #{|R_ii| > thr},  X = P [R_11^{-1} Q_1^T ; 0]   (q x p).
// Also used for N_k^+ of Lemma 1, N_k = S(I_k, J_k).
//
// Factorisation: one cooperative launch.  M is copied column-major (columns
// contiguous); CTA g owns the columns col = g (mod G) and a warp per column
// computes norms and applies reflectors.  Pivoting is virtual: a permutation
// array records which physical column is pivot j, so no column is ever moved.
// One bounded grid barrier per step publishes the per-CTA norm maxima; every
// CTA then rebuilds the reflector from the (untouched) pivot column in shared
// memory.  Solve: an independent launch, one warp per column of the identity:
// apply H_0..H_{k-1}, then column-oriented back substitution with R_11.
#include <climits>

#include <cooperative_groups.h>
#include <map>
#include <mutex>

#include "gridbar.cuh"

// Shared-memory bytes of the single-CTA variant (0 if it does not apply).
static size_t qrcp_small_smem(int64_t p, int64_t q) {
  int64_t kmax = p < q ? p : q;
  size_t b = sizeof(double) * (size_t)(q * p + p * p + q + 4 * kmax) + sizeof(int) * (size_t)(2 * q);
  return b <= 200 * 1024 ? b : 0;
}

namespace cur {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct QrcpParams {
  const double* M; int64_t p, q, ldm;
  int thr_mode; double thr; double* scale_dev;
  QrcpWork w; DevStatus* st;
};

// Squared norms compare as integers (the bit patterns of non-negative doubles
// order like their values; FP64 compares cost FP64 pipe slots on GB300).  A NaN
// gets -2, below every number; callers use -3 for "no column".
__device__ __forceinline__ long long norm_key(double x) {
  const long long k = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL;
  return k > 0x7FF0000000000000LL ? -2 : k;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kThreads) qrcp_factor_kernel(QrcpParams P) {
  extern __shared__ double v[];  // reflector, p entries (indices >= j used)
  __shared__ double s_red_a[kWarps];
  __shared__ long long s_red_i[kWarps];
  __shared__ double s_nrm2;
  __shared__ long long s_jp;
  __shared__ double s_tau, s_alpha;
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int64_t p = P.p, q = P.q, kmax = p < q ? p : q;
  double* Rc = P.w.Rc;

  // column-major working copy of the owned columns
  for (int64_t col = cta + (int64_t)G * wid; col < q; col += (int64_t)G * kWarps) {
    for (int64_t i = lane; i < p; i += 32) Rc[col * p + i] = P.M[i * P.ldm + col];
    if (lane == 0) P.w.used[col] = 0;
  }
  __syncthreads();

  for (int64_t j = 0; j < kmax; ++j) {
    double* slot = P.w.slots + (size_t)((j & 1) * G) * 2;
    // A. squared norms of the owned, unused columns over rows j..p-1
    double ba = -1.0;
    long long bi = LLONG_MAX;
    for (int64_t col = cta + (int64_t)G * wid; col < q; col += (int64_t)G * kWarps) {
      if (P.w.used[col]) continue;
      double s = 0.0;
      for (int64_t i = j + lane; i < p; i += 32) { double x = __ldcg(Rc + col * p + i); s = fma(x, x, s); }
      s = warp_sum(s);
      if (s > ba || (s == ba && col < bi)) { ba = s; bi = col; }
    }
    if (lane == 0) { s_red_a[wid] = ba; s_red_i[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      double a = -1.0; long long ii = LLONG_MAX;
      for (int w = 0; w < kWarps; ++w)
        if (s_red_a[w] > a || (s_red_a[w] == a && s_red_i[w] < ii)) { a = s_red_a[w]; ii = s_red_i[w]; }
      slot[2 * cta] = a;
      slot[2 * cta + 1] = __longlong_as_double(ii);
    }
    __threadfence();
    if (!grid_barrier(P.w.bar, P.st)) return;
    // B. global pivot (largest norm, smallest index) and its reflector
    if (wid == 0) {
      const SlotWin c = warp_slot_best(slot, 2, G, lane);
      if (lane == 0) { s_nrm2 = c.a; s_jp = c.i; }
    }
    __syncthreads();
    const long long jp = s_jp;
    if (jp == LLONG_MAX) { if (tid == 0) dev_set_err(P.st, kDevNoCandidate); return; }
    for (int64_t i = j + tid; i < p; i += kThreads) v[i] = __ldcg(Rc + jp * p + i);
    __syncthreads();
    if (tid == 0) {
      double normx = sqrt(s_nrm2);
      double x0 = v[j];
      if (normx == 0.0) {
        s_tau = 0.0; s_alpha = 0.0;
      } else {
        double alpha = x0 >= 0.0 ? -normx : normx;
        s_alpha = alpha;
        v[j] = x0 - alpha;
        s_tau = 0.0;  // set after the norm of v below
      }
    }
    __syncthreads();
    if (s_alpha != 0.0) {  // tau = 2 / ||v||^2
      double s = 0.0;
      for (int64_t i = j + tid; i < p; i += kThreads) s = fma(v[i], v[i], s);
      s = warp_sum(s);
      if (lane == 0) s_red_a[wid] = s;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += s_red_a[w];
        s_tau = 2.0 / t;
      }
      __syncthreads();
    }
    const double tau = s_tau;
    if (cta == 0) {
      if (tid == 0) { P.w.perm[j] = jp; P.w.rdiag[j] = s_alpha; P.w.tau[j] = tau; }
      for (int64_t i = j + tid; i < p; i += kThreads) P.w.V[j * p + i] = v[i];
    }
    if (tid == 0 && (jp % G) == cta) P.w.used[jp] = 1;
    __syncthreads();
    // C. apply H_j = I - tau v v^T to the owned unused columns
    if (tau != 0.0) {
      for (int64_t col = cta + (int64_t)G * wid; col < q; col += (int64_t)G * kWarps) {
        if (P.w.used[col]) continue;
        double d = 0.0;
        for (int64_t i = j + lane; i < p; i += 32) d = fma(v[i], __ldcg(Rc + col * p + i), d);
        d = warp_sum(d) * tau;
        for (int64_t i = j + lane; i < p; i += 32) {
          double* r = Rc + col * p + i;
          *r = fma(-d, v[i], __ldcg(r));
        }
      }
    }
    __syncthreads();
  }
  // numerical rank (CTA 0 wrote every rdiag itself)
  if (cta == 0 && tid == 0) {
    double thr;
    double r0 = kmax > 0 ? fabs(P.w.rdiag[0]) : 0.0;
    if (P.thr_mode == 0) {
      thr = (double)(p > q ? p : q) * 0x1.0p-52 * r0;
    } else if (P.thr_mode == 1) {
      thr = P.thr;
    } else {
      double sc = *P.scale_dev;
      if (sc < 0.0) { sc = 0x1.0p-52 * r0; *P.scale_dev = sc; }
      thr = P.thr * sc;
    }
    int64_t k = 0;
    while (k < kmax && fabs(P.w.rdiag[k]) > thr) ++k;
    *P.w.rank = k;
  }
  // columns never pivoted (q > p): append in increasing order after kmax
  if (cta == 0 && tid == 0 && q > kmax) {
    int64_t pos = kmax;
    for (int64_t col = 0; col < q; ++col) {
      bool used = false;
      for (int64_t jj = 0; jj < kmax; ++jj) used |= (P.w.perm[jj] == col);
      if (!used) P.w.perm[pos++] = col;
    }
  }
}

// Cooperative variant with each CTA's columns resident in shared memory
// (Rloc[li * p + i] for column col = cta + li * G).  Every CTA publishes its
// best candidate's norm, index and current column to a double-buffered slot,
// so one bounded grid barrier per step suffices; the reflector is rebuilt by
// every CTA from the winner's slot.  At exit the columns go back to Rc for the
// solve kernel.
__global__ void __launch_bounds__(kThreads) qrcp_factor_smem_kernel(QrcpParams P, int nloc) {
  extern __shared__ double shm[];
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int p = (int)P.p, q = (int)P.q, kmax = p < q ? p : q;
  double* Rloc = shm;                          // nloc * p
  double* v = Rloc + (size_t)nloc * p;         // p (reflector)
  int* usedl = reinterpret_cast<int*>(v + p);  // nloc
  __shared__ double s_red_a[kWarps];
  __shared__ long long s_red_i[kWarps];
  __shared__ long long s_jp;
  __shared__ int s_wcta;
  __shared__ double s_tau, s_alpha, s_nrm2;
  const int stride = p + 2;

  for (int li = wid; li < nloc; li += kWarps) {
    const int col = cta + li * G;
    for (int i = lane; i < p; i += 32) Rloc[li * p + i] = col < q ? P.M[(int64_t)i * P.ldm + col] : 0.0;
    if (lane == 0) usedl[li] = col < q ? 0 : 1;
  }
  __syncthreads();

  for (int j = 0; j < kmax; ++j) {
    double* slot = P.w.slots + (size_t)((j & 1) * G) * stride;
    double ba = -1.0;
    long long bi = LLONG_MAX;
    for (int li = wid; li < nloc; li += kWarps) {
      if (usedl[li]) continue;
      const double* r = Rloc + li * p;
      double s0 = 0.0, s1 = 0.0;
      int i = j + lane;
      for (; i + 32 < p; i += 64) { s0 = fma(r[i], r[i], s0); s1 = fma(r[i + 32], r[i + 32], s1); }
      if (i < p) s0 = fma(r[i], r[i], s0);
      double sn = warp_sum(s0 + s1);
      const long long col = cta + (long long)li * G;
      if (sn > ba || (sn == ba && col < bi)) { ba = sn; bi = col; }
    }
    if (lane == 0) { s_red_a[wid] = ba; s_red_i[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      double a = -1.0; long long ii = LLONG_MAX;
      for (int w = 0; w < kWarps; ++w)
        if (s_red_a[w] > a || (s_red_a[w] == a && s_red_i[w] < ii)) { a = s_red_a[w]; ii = s_red_i[w]; }
      s_red_a[0] = a; s_red_i[0] = ii;
    }
    __syncthreads();
    {
      double* my = slot + (size_t)cta * stride;
      const long long bii = s_red_i[0];
      if (tid == 0) { my[0] = s_red_a[0]; my[1] = __longlong_as_double(bii); }
      if (bii != LLONG_MAX) {
        const double* r = Rloc + (int)((bii - cta) / G) * p;
        for (int i = j + tid; i < p; i += kThreads) my[2 + i] = r[i];
      }
    }
    __threadfence();
    if (!grid_barrier(P.w.bar, P.st)) return;
    if (wid == 0) {
      const SlotWin c = warp_slot_best(slot, (size_t)stride, G, lane);
      if (lane == 0) { s_nrm2 = c.a; s_jp = c.i; s_wcta = c.g; }
    }
    __syncthreads();
    const long long jp = s_jp;
    if (jp == LLONG_MAX) { if (tid == 0) dev_set_err(P.st, kDevNoCandidate); return; }
    const double* wsrc = slot + (size_t)s_wcta * stride + 2;
    for (int i = j + tid; i < p; i += kThreads) v[i] = __ldcg(wsrc + i);
    __syncthreads();
    if (tid == 0) {
      double normx = sqrt(s_nrm2), x0 = v[j];
      if (normx == 0.0) {
        s_alpha = 0.0;
      } else {
        s_alpha = x0 >= 0.0 ? -normx : normx;
        v[j] = x0 - s_alpha;
      }
    }
    __syncthreads();
    if (s_alpha != 0.0) {
      double sacc = 0.0;
      for (int i = j + tid; i < p; i += kThreads) sacc = fma(v[i], v[i], sacc);
      sacc = warp_sum(sacc);
      if (lane == 0) s_red_a[wid] = sacc;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += s_red_a[w];
        s_tau = 2.0 / t;
      }
    } else if (tid == 0) {
      s_tau = 0.0;
    }
    __syncthreads();
    const double tau = s_tau;
    if (cta == 0) {
      if (tid == 0) { P.w.perm[j] = jp; P.w.rdiag[j] = s_alpha; P.w.tau[j] = tau; }
      for (int i = j + tid; i < p; i += kThreads) P.w.V[(int64_t)j * p + i] = v[i];
    }
    if (tid == 0 && (jp % G) == cta) usedl[(int)((jp - cta) / G)] = 1;
    __syncthreads();
    if (tau != 0.0) {
      for (int li = wid; li < nloc; li += kWarps) {
        if (usedl[li]) continue;
        double* r = Rloc + li * p;
        double d0 = 0.0, d1 = 0.0;
        int i = j + lane;
        for (; i + 32 < p; i += 64) { d0 = fma(v[i], r[i], d0); d1 = fma(v[i + 32], r[i + 32], d1); }
        if (i < p) d0 = fma(v[i], r[i], d0);
        const double d = warp_sum(d0 + d1) * tau;
        for (int i2 = j + lane; i2 < p; i2 += 32) r[i2] = fma(-d, v[i2], r[i2]);
      }
    }
    __syncthreads();
  }
  // write the columns back for the solve (frozen pivot columns hold R above the diagonal)
  for (int li = wid; li < nloc; li += kWarps) {
    const int col = cta + li * G;
    if (col >= q) continue;
    for (int i = lane; i < p; i += 32) P.w.Rc[(int64_t)col * p + i] = Rloc[li * p + i];
  }
  if (cta == 0 && tid == 0) {
    double thr;
    double r0 = kmax > 0 ? fabs(P.w.rdiag[0]) : 0.0;
    if (P.thr_mode == 0) {
      thr = (double)(p > q ? p : q) * 0x1.0p-52 * r0;
    } else if (P.thr_mode == 1) {
      thr = P.thr;
    } else {
      double sc = *P.scale_dev;
      if (sc < 0.0) { sc = 0x1.0p-52 * r0; *P.scale_dev = sc; }
      thr = P.thr * sc;
    }
    int64_t k = 0;
    while (k < kmax && fabs(P.w.rdiag[k]) > thr) ++k;
    *P.w.rank = k;
    if (q > kmax) {
      int64_t pos = kmax;
      for (int64_t col = 0; col < q; ++col) {
        bool u = false;
        for (int64_t jj = 0; jj < kmax; ++jj) u |= (P.w.perm[jj] == col);
        if (!u) P.w.perm[pos++] = col;
      }
    }
  }
}

struct SolveParams {
  int64_t p, q;
  const double* Rc; const double* V; const double* tau; const double* rdiag;
  const int64_t* perm; const int64_t* rank;
  double* Ywork;  // p * p: column l of Q^T then Z
  double* X; int64_t ldx;
  const DevStatus* st;   // a factorisation that recorded an error left no rank or permutation
};

// One warp per column l of the identity.
__global__ void __launch_bounds__(kThreads) qrcp_solve_kernel(SolveParams S) {
  const int lane = threadIdx.x & 31;
  const int64_t l = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (l >= S.p) return;
  if (S.st && *((const volatile int*)&S.st->err) != 0) return;
  const int64_t p = S.p, k = *S.rank;
  double* y = S.Ywork + l * p;
  for (int64_t i = lane; i < p; i += 32) y[i] = (i == l) ? 1.0 : 0.0;
  __syncwarp();
  for (int64_t j = 0; j < k; ++j) {  // y = H_{k-1} ... H_0 e_l
    double t = S.tau[j];
    if (t == 0.0) continue;
    const double* vj = S.V + j * p;
    double d = 0.0;
    for (int64_t i = j + lane; i < p; i += 32) d = fma(vj[i], y[i], d);
    d = warp_sum(d) * t;
    for (int64_t i = j + lane; i < p; i += 32) y[i] = fma(-d, vj[i], y[i]);
    __syncwarp();
  }
  // back substitution R_11 z = y(0:k), column oriented
  for (int64_t i = k - 1; i >= 0; --i) {
    double zi = y[i] / S.rdiag[i];
    __syncwarp();
    const double* rcol = S.Rc + S.perm[i] * p;  // R(0:i, i) lives in pivot column i
    for (int64_t a = lane; a < i; a += 32) y[a] = fma(-zi, rcol[a], y[a]);
    if (lane == 0) y[i] = zi;
    __syncwarp();
  }
  for (int64_t i = lane; i < S.q; i += 32) {
    double val = (i < k) ? y[i] : 0.0;
    S.X[S.perm[i] * S.ldx + l] = val;
  }
}

// Solve for p <= kSolveSmallP: the same arithmetic as qrcp_solve_kernel with
// the reflectors and R_11 staged in shared memory (shared by the CTA's
// warps, one warp per column l of the identity), the column y in registers
// (row i = lane + 32 s in y[s]) and R_11's diagonal applied as reciprocals,
// so a reflector costs one warp reduction and a back-substitution step a
// multiply and an FMA (GB300 runs a dependent FP64 operation in ~64 cycles, a
// divide in ~560).
constexpr int kSolveSmallP = 64;
// Four warps per CTA: one warp per SM sub-partition, so a CTA's FP64 work
// stays latency bound instead of queueing on the SM's FP64 pipe (eight warps
// per CTA kept that pipe ~70 % busy on the 7 SMs of a p = 50 solve).
constexpr int kSolveSmallThreads = 128;

__global__ void __launch_bounds__(kSolveSmallThreads) qrcp_solve_small_kernel(SolveParams S) {
  extern __shared__ double ssm[];
  if (S.st && *((const volatile int*)&S.st->err) != 0) return;
  const int p = (int)S.p, q = (int)S.q;
  const int k = (int)*S.rank;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double* Vs = ssm;                      // k * p: reflector j at Vs[j * p], zero above row j
  double* Rs = Vs + (size_t)k * p;       // k * k: R(a, i) at Rs[i * k + a], a < i
  double* tau = Rs + (size_t)k * k;      // k
  double* rinv = tau + k;                // k
  int* perm = reinterpret_cast<int*>(rinv + k);   // q
  for (int e = threadIdx.x; e < k * p; e += kSolveSmallThreads) {
    const int j = e / p, i = e - j * p;
    Vs[e] = i >= j ? S.V[(int64_t)j * p + i] : 0.0;
  }
  for (int e = threadIdx.x; e < k * k; e += kSolveSmallThreads) {
    const int i = e / k, a = e - i * k;
    Rs[e] = a < i ? S.Rc[S.perm[i] * p + a] : 0.0;
  }
  for (int j = threadIdx.x; j < k; j += kSolveSmallThreads) { tau[j] = S.tau[j]; rinv[j] = 1.0 / S.rdiag[j]; }
  for (int i = threadIdx.x; i < q; i += kSolveSmallThreads) perm[i] = (int)S.perm[i];
  __syncthreads();
  const int l = blockIdx.x * (kSolveSmallThreads / 32) + wid;
  if (l >= p) return;
  double y0 = lane == l ? 1.0 : 0.0, y1 = lane + 32 == l ? 1.0 : 0.0;   // rows lane, lane + 32
  const bool r1 = lane + 32 < p;
  for (int j = 0; j < k; ++j) {   // y = H_{k-1} ... H_0 e_l
    const double t = tau[j];
    if (t == 0.0) continue;
    const double v0 = lane < p ? Vs[j * p + lane] : 0.0;
    const double v1 = r1 ? Vs[j * p + lane + 32] : 0.0;
    double d = fma(v1, y1, v0 * y0);
    d = warp_sum(d) * t;
    y0 = fma(-d, v0, y0);
    y1 = fma(-d, v1, y1);
  }
  for (int i = k - 1; i >= 0; --i) {   // R_11 z = y(0:k), column oriented
    const double yi = __shfl_sync(0xffffffffu, i < 32 ? y0 : y1, i & 31);
    const double zi = yi * rinv[i];
    if (lane < i) y0 = fma(-zi, Rs[i * k + lane], y0);
    if (lane + 32 < i) y1 = fma(-zi, Rs[i * k + lane + 32], y1);
    if (lane == i) y0 = zi;
    if (lane + 32 == i) y1 = zi;
  }
  for (int i = lane; i < q; i += 32)   // row i of z sits in this lane (k <= p <= 64)
    S.X[(int64_t)perm[i] * S.ldx + l] = i < k ? (i < 32 ? y0 : y1) : 0.0;
}

// Single-CTA variant for small p, q (every N_k and small cores).  GB300 runs
// FP64 at ~2 DFMA/clk/SM, so a 50 x 50 problem has too little work for one
// thread per column to hide FP64 and shared-memory latency.  Here every column
// gets a group of 8 threads that split its rows (segments i = i0 + s, s + 8,
// ...) and combine with a 3-step shuffle; R is row-major in shared memory
// (R[i*q + col]) and the pivot column is read as a broadcast.  Pivot columns
// are frozen in place, so reflector j is (vhead[j], R[j+1.., perm[j]]) and
// R(i, i') = R[i, perm[i']] for i < i'.  The same launch forms
// X = P [R_11^{-1} Q_1^T; 0] with one thread group per column of the identity.
constexpr int kSmallThreads = 512;
constexpr int kSmallSplitP = 24;                   // from here on the solve runs on many SMs
constexpr int kSeg = 8;                            // threads per column
constexpr int kGroups = kSmallThreads / kSeg;      // columns in flight

__device__ __forceinline__ double seg_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// kSolveHere = false: the CTA only factors, and writes R (column-major, pivot
// columns frozen), the reflectors, tau, R's diagonal, the permutation and the
// rank in the layout of qrcp_factor_smem_kernel, for qrcp_solve_kernel to form
// X with one warp per right-hand side over many SMs (the solve is 3 p^3 of the
// 4/3 p^3 + 3 p^3 flops, and one SM's FP64 rate is a 64th of the GPU's).
template <bool kSolveHere>
__global__ void __launch_bounds__(kSmallThreads) qrcp_small_kernel(QrcpParams P, double* X,
                                                                   int64_t ldx) {
  extern __shared__ double sm[];
  const int p = (int)P.p, q = (int)P.q, kmax = p < q ? p : q;
  double* R = sm;                                   // p * q, row-major
  double* Y = R + (size_t)p * q;                    // p * p, row-major (column l of the identity)
  double* nrm = Y + (size_t)p * p;                  // q
  double* rdiag = nrm + q;                          // kmax
  double* rinv = rdiag + kmax;                      // kmax
  double* tau = rinv + kmax;                        // kmax
  double* vhead = tau + kmax;                       // kmax
  int* perm = reinterpret_cast<int*>(vhead + kmax); // q
  int* used = perm + q;                             // q
  __shared__ int s_jp, s_k;
  __shared__ double s_tau;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int grp = tid / kSeg, sg = tid % kSeg;

  for (int e = tid; e < p * q; e += kSmallThreads) {
    int i = e / q, col = e - i * q;
    R[e] = P.M[(int64_t)i * P.ldm + col];
  }
  for (int col = tid; col < q; col += kSmallThreads) used[col] = 0;
  __syncthreads();

  for (int j = 0; j < kmax; ++j) {
    // squared norms over rows j..p-1 of the unused columns
    for (int col0 = 0; col0 < q; col0 += kGroups) {   // uniform trip count for the shuffles
      const int col = col0 + grp;
      double sacc = 0.0;
      if (col < q && !used[col])
        for (int i = j + sg; i < p; i += kSeg) { double x = R[i * q + col]; sacc = fma(x, x, sacc); }
      sacc = seg_sum(sacc);
      if (col < q && sg == 0) nrm[col] = used[col] ? -1.0 : sacc;
    }
    __syncthreads();
    if (wid == 0) {   // argmax over columns: largest norm, smallest index
      long long ba = -3;
      int bi = INT_MAX;
      for (int col = lane; col < q; col += 32) {
        const long long kc = used[col] ? -3 : norm_key(nrm[col]);
        if (kc > ba) { ba = kc; bi = col; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const long long oa = __shfl_down_sync(0xffffffffu, ba, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (oa > ba || (oa == ba && oi < bi)) { ba = oa; bi = oi; }
      }
      ba = __shfl_sync(0xffffffffu, ba, 0);
      if (ba < 0) {   // every remaining norm is NaN: no pivot
        if (lane == 0) { s_jp = -1; dev_set_err(P.st, kDevNoCandidate); }
        goto pivot_done;
      }
      {
      const int ii = __shfl_sync(0xffffffffu, bi, 0);
      const double a = __longlong_as_double(ba);
      double vv = 0.0;          // ||x_{j+1..p-1}||^2 of the pivot column
      for (int i = j + 1 + lane; i < p; i += 32) { double x = R[i * q + ii]; vv = fma(x, x, vv); }
      vv = warp_sum(vv);
      if (lane == 0) {
        const double x0 = R[j * q + ii];
        const double normx = sqrt(a);
        const double alpha = normx == 0.0 ? 0.0 : (x0 >= 0.0 ? -normx : normx);
        const double vh = x0 - alpha;
        const double t = alpha != 0.0 ? 2.0 / fma(vh, vh, vv) : 0.0;
        s_jp = ii; s_tau = t;
        perm[j] = ii; used[ii] = 1; rdiag[j] = alpha; vhead[j] = vh; tau[j] = t;
      }
      }
    }
  pivot_done:
    __syncthreads();
    const int jp = s_jp;
    if (jp < 0) return;
    const double tj = s_tau;
    if (tj != 0.0) {
      const double vh = vhead[j];
      for (int col0 = 0; col0 < q; col0 += kGroups) {
        const int col = col0 + grp;
        const bool act = col < q && !used[col];
        double d = 0.0;
        if (act) {
          if (sg == 0) d = vh * R[j * q + col];
          for (int i = j + 1 + sg; i < p; i += kSeg) d = fma(R[i * q + jp], R[i * q + col], d);
        }
        d = seg_sum(d) * tj;
        if (act) {
          if (sg == 0) R[j * q + col] = fma(-d, vh, R[j * q + col]);
          for (int i = j + 1 + sg; i < p; i += kSeg) R[i * q + col] = fma(-d, R[i * q + jp], R[i * q + col]);
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    double thr;
    double r0 = kmax > 0 ? fabs(rdiag[0]) : 0.0;
    if (P.thr_mode == 0) {
      thr = (double)(p > q ? p : q) * 0x1.0p-52 * r0;
    } else if (P.thr_mode == 1) {
      thr = P.thr;
    } else {
      double sc = *P.scale_dev;
      if (sc < 0.0) { sc = 0x1.0p-52 * r0; *P.scale_dev = sc; }
      thr = P.thr * sc;
    }
    int k = 0;
    while (k < kmax && fabs(rdiag[k]) > thr) ++k;
    s_k = k;
    *P.w.rank = k;
    if (q > kmax) {  // columns never pivoted, in increasing order
      int pos = kmax;
      for (int col = 0; col < q; ++col)
        if (!used[col]) perm[pos++] = col;
    }
  }
  __syncthreads();
  const int k = s_k;
  if constexpr (!kSolveHere) {
    for (int e = tid; e < p * q; e += kSmallThreads) {
      const int i = e % p, col = e / p;
      P.w.Rc[(int64_t)col * p + i] = R[i * q + col];
    }
    for (int e = tid; e < kmax * p; e += kSmallThreads) {
      const int j = e / p, i = e - j * p;
      if (i >= j) P.w.V[(int64_t)j * p + i] = i == j ? vhead[j] : R[i * q + perm[j]];
    }
    for (int j = tid; j < kmax; j += kSmallThreads) {
      P.w.tau[j] = tau[j];
      P.w.rdiag[j] = rdiag[j];
    }
    for (int col = tid; col < q; col += kSmallThreads) P.w.perm[col] = perm[col];
  } else {
  for (int i = tid; i < k; i += kSmallThreads) rinv[i] = 1.0 / rdiag[i];
  for (int e = tid; e < p * p; e += kSmallThreads) Y[e] = (e / p == e % p) ? 1.0 : 0.0;
  __syncthreads();
  for (int l0 = 0; l0 < p; l0 += kGroups) {
    const int l = l0 + grp;
    const bool act = l < p;
    for (int jj = 0; jj < k; ++jj) {   // y = H_{k-1} ... H_0 e_l
      __syncwarp();                     // rows written by the neighbouring lanes last step
      const double tjj = tau[jj];
      if (tjj == 0.0) continue;
      const int pc = perm[jj];
      const double vh = vhead[jj];
      double d = 0.0;
      if (act) {
        if (sg == 0) d = vh * Y[jj * p + l];
        for (int i = jj + 1 + sg; i < p; i += kSeg) d = fma(R[i * q + pc], Y[i * p + l], d);
      }
      d = seg_sum(d) * tjj;
      if (act) {
        if (sg == 0) Y[jj * p + l] = fma(-d, vh, Y[jj * p + l]);
        for (int i = jj + 1 + sg; i < p; i += kSeg) Y[i * p + l] = fma(-d, R[i * q + pc], Y[i * p + l]);
      }
    }
    for (int i = k - 1; i >= 0; --i) {  // back substitution with R_11, column oriented
      __syncwarp();
      const double zi = act ? Y[i * p + l] * rinv[i] : 0.0;
      __syncwarp();
      if (act) {
        if (sg == 0) Y[i * p + l] = zi;
        const int pc = perm[i];
        for (int a2 = sg; a2 < i; a2 += kSeg) Y[a2 * p + l] = fma(-zi, R[a2 * q + pc], Y[a2 * p + l]);
      }
    }
    __syncwarp();
    if (act)
      for (int i = sg; i < q; i += kSeg) X[(int64_t)perm[i] * ldx + l] = (i < k) ? Y[i * p + l] : 0.0;
  }
  }
}

// Cluster variant for mid-size problems (kSmallSplitP <= p <= 512, q <= CL
// kClMaxLocal): one thread-block cluster of CL CTAs (16 where the GPU schedules
// it, else 8) factors M, CTA r owning the columns col = r (mod CL) column-major
// in its shared memory, one warp per column at a time.  A step's pivot search,
// exchange and reflector take no global-memory round trip: each CTA stores its
// best candidate {norm^2 as an integer key, column, R(j, col), ||R(j+1:, col)||^2}
// into every CTA's shared memory (distributed shared memory), one cluster
// barrier publishes them, every CTA picks the same winner, copies the pivot
// column from its owner's shared memory and forms the reflector itself.  The
// norms of the next step are formed in the pass that applies the reflector.
// Output is the layout of qrcp_small_kernel<false> for qrcp_solve_kernel.
constexpr int kClMaxLocal = 16;      // columns per CTA handled by the cluster variant
constexpr int kClRec = 4;            // doubles per candidate record

__global__ void __launch_bounds__(kClMaxLocal * 32) qrcp_cluster_kernel(QrcpParams P) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double sm[];
  const int CL = (int)cl.num_blocks(), r = (int)cl.block_rank();
  const int p = (int)P.p, q = (int)P.q, kmax = p < q ? p : q;
  const int nlm = (q + CL - 1) / CL;                 // local column slots (same in every CTA)
  const int nloc = (q - r + CL - 1) / CL;            // columns this CTA owns
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  double* Rl = sm;                                   // nlm * p: local column c at Rl[c * p]
  double* vcol = Rl + (size_t)nlm * p;               // p: pivot column of this step
  double* rec = vcol + p;                            // 2 * CL * kClRec: records by step parity
  double* rdiag = rec + 2 * CL * kClRec;             // kmax
  double* tau = rdiag + kmax;                        // kmax
  double* vhead = tau + kmax;                        // kmax
  double* na = vhead + kmax;                         // nlm: ||R(j:, c)||^2 of this step
  double* ns1 = na + nlm;                            // nlm: ||R(j+1:, c)||^2 of this step
  int* used = reinterpret_cast<int*>(ns1 + nlm);     // nlm
  int* perm = used + nlm;                            // q
  int* gused = perm + q;                             // q
  __shared__ long long s_wk[kClMaxLocal];
  __shared__ int s_wc[kClMaxLocal];
  __shared__ double s_wx[kClMaxLocal], s_ws[kClMaxLocal];

  for (int c = wid; c < nloc; c += nw) {
    const int col = r + CL * c;
    double t1 = 0.0;
    for (int i = lane; i < p; i += 32) {
      const double x = P.M[(int64_t)i * P.ldm + col];
      Rl[c * p + i] = x;
      if (i >= 1) t1 = fma(x, x, t1);
    }
    t1 = warp_sum(t1);
    __syncwarp();
    if (lane == 0) { const double x0 = Rl[c * p]; ns1[c] = t1; na[c] = fma(x0, x0, t1); used[c] = 0; }
  }
  for (int col = tid; col < q; col += blockDim.x) gused[col] = 0;
  __syncthreads();

  bool nopivot = false;
  for (int j = 0; j < kmax; ++j) {
    const int par = j & 1;
    __syncwarp();   // lane 0's norms of the last pass
    // this warp's best unused column: largest norm, then smallest index; NaN
    // norms (key -2) rank below numbers, "none" is -3
    long long bk = -3;
    int bc = INT_MAX;
    double bx = 0.0, bs = 0.0;
    for (int c = wid; c < nloc; c += nw) {
      if (used[c]) continue;
      const long long k = norm_key(na[c]);
      const int col = r + CL * c;
      if (k > bk || (k == bk && col < bc)) { bk = k; bc = col; bx = Rl[c * p + j]; bs = ns1[c]; }
    }
    if (lane == 0) { s_wk[wid] = bk; s_wc[wid] = bc; s_wx[wid] = bx; s_ws[wid] = bs; }
    __syncthreads();
    if (wid == 0) {   // the CTA's best, stored into every CTA's record slot r
      long long k = lane < nw ? s_wk[lane] : -3;
      int c = lane < nw ? s_wc[lane] : INT_MAX;
      int src = lane;
      for (int o = 16; o > 0; o >>= 1) {
        const long long ok = __shfl_xor_sync(0xffffffffu, k, o);
        const int oc = __shfl_xor_sync(0xffffffffu, c, o);
        const int os = __shfl_xor_sync(0xffffffffu, src, o);
        if (ok > k || (ok == k && oc < c)) { k = ok; c = oc; src = os; }
      }
      if (lane < CL) {
        double* dst = cl.map_shared_rank(rec + (par * CL + r) * kClRec, lane);
        dst[0] = __longlong_as_double(k);
        dst[1] = __longlong_as_double((long long)c);
        dst[2] = src < nw ? s_wx[src] : 0.0;
        dst[3] = src < nw ? s_ws[src] : 0.0;
      }
    }
    cl.sync();   // release of the records (and of last step's columns), acquire of the others'

    // every warp: the winner among the CL records (integer compares only)
    long long wk = -3;
    int wc = INT_MAX;
    if (lane < CL) {
      const double* rr = rec + (par * CL + lane) * kClRec;
      wk = __double_as_longlong(rr[0]);
      wc = (int)__double_as_longlong(rr[1]);
    }
    int wl = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const long long ok = __shfl_xor_sync(0xffffffffu, wk, o);
      const int oc = __shfl_xor_sync(0xffffffffu, wc, o);
      const int ol = __shfl_xor_sync(0xffffffffu, wl, o);
      if (ok > wk || (ok == wk && oc < wc)) { wk = ok; wc = oc; wl = ol; }
    }
    if (wk < 0) {   // every remaining norm is NaN: no pivot (the same in every CTA)
      if (r == 0 && tid == 0) dev_set_err(P.st, kDevNoCandidate);
      nopivot = true;
      break;
    }
    const int jp = wc;
    const int own = jp % CL, cjp = jp / CL;
    if (tid != 0) {   // the pivot column's rows j.. from its owner (frozen from now on),
                      // while thread 0 forms the reflector's scalars
      const double* srcc = cl.map_shared_rank(Rl + (size_t)cjp * p, own);
      for (int i = j + tid - 1; i < p; i += blockDim.x - 1) vcol[i] = srcc[i];
    } else {
      const double* rr = rec + (par * CL + wl) * kClRec;
      const double x0 = rr[2], s1 = rr[3];
      const double normx = sqrt(__longlong_as_double(wk));
      double alpha = x0, vh = 0.0, t = 0.0;
      if (normx != 0.0) {   // (a zero column keeps R(j, j) = x0 and no reflector)
        alpha = x0 >= 0.0 ? -normx : normx;
        vh = x0 - alpha;
        t = 2.0 / fma(vh, vh, s1);
      }
      rdiag[j] = alpha; tau[j] = t; vhead[j] = vh;
      perm[j] = jp; gused[jp] = 1;
      if (own == r) used[cjp] = 1;
    }
    __syncthreads();

    // apply H_j to this CTA's unused columns; form their norms for step j + 1
    const double tj = tau[j], vh = vhead[j];
    for (int c = wid; c < nloc; c += nw) {
      if (used[c]) continue;
      double* R = Rl + (size_t)c * p;
      if (tj != 0.0) {
        double d = lane == 0 ? vh * R[j] : 0.0;
        for (int i = j + 1 + lane; i < p; i += 32) d = fma(vcol[i], R[i], d);
        d = warp_sum(d) * tj;
        if (lane == 0) R[j] = fma(-d, vh, R[j]);
        for (int i = j + 1 + lane; i < p; i += 32) R[i] = fma(-d, vcol[i], R[i]);
        __syncwarp();   // rows written by the neighbouring lanes
      }
      double t1 = 0.0;
      for (int i = j + 2 + lane; i < p; i += 32) t1 = fma(R[i], R[i], t1);
      t1 = warp_sum(t1);
      __syncwarp();
      if (lane == 0 && j + 1 < p) { const double x0 = R[j + 1]; ns1[c] = t1; na[c] = fma(x0, x0, t1); }
    }
  }

  if (nopivot) {   // every thread of the cluster took the break at the same step
    cl.sync();
    return;
  }
  if (r == 0 && tid == 0) {
    double thr;
    const double r0 = kmax > 0 ? fabs(rdiag[0]) : 0.0;
    if (P.thr_mode == 0) {
      thr = (double)(p > q ? p : q) * 0x1.0p-52 * r0;
    } else if (P.thr_mode == 1) {
      thr = P.thr;
    } else {
      double sc = *P.scale_dev;
      if (sc < 0.0) { sc = 0x1.0p-52 * r0; *P.scale_dev = sc; }
      thr = P.thr * sc;
    }
    int k = 0;
    while (k < kmax && fabs(rdiag[k]) > thr) ++k;
    *P.w.rank = k;
    int pos = kmax;   // columns never pivoted, in increasing order
    for (int col = 0; col < q && pos < q; ++col)
      if (!gused[col]) perm[pos++] = col;
  }
  __syncthreads();
  for (int c = wid; c < nloc; c += nw) {   // R column-major by original column
    const int col = r + CL * c;
    for (int i = lane; i < p; i += 32) P.w.Rc[(int64_t)col * p + i] = Rl[c * p + i];
  }
  for (int j = wid; j < kmax; j += nw) {   // reflector tails from the pivot columns' owners
    const int pc = perm[j];
    if (pc % CL != r) continue;
    const double* R = Rl + (size_t)(pc / CL) * p;
    for (int i = j + lane; i < p; i += 32) P.w.V[(int64_t)j * p + i] = i == j ? vhead[j] : R[i];
  }
  if (r == 0) {
    for (int j = tid; j < kmax; j += blockDim.x) { P.w.tau[j] = tau[j]; P.w.rdiag[j] = rdiag[j]; }
    for (int col = tid; col < q; col += blockDim.x) P.w.perm[col] = perm[col];
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

}  // namespace

// Shared-memory bytes of the cluster variant for a cluster of CL CTAs.
static size_t qrcp_cluster_smem(int64_t p, int64_t q, int CL) {
  const int64_t kmax = p < q ? p : q, nlm = (q + CL - 1) / CL;
  return sizeof(double) * (size_t)(nlm * p + p + 2 * CL * kClRec + 3 * kmax + 2 * nlm) +
         sizeof(int) * (size_t)(nlm + 2 * q);
}

static cudaLaunchConfig_t cluster_config(int CL, int threads, size_t smem, cudaStream_t stream,
                                         cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Largest cluster (16, else 8) the device co-schedules with the variant's
// largest shared-memory request and block, 0 if neither; probed once per device.
static int qrcp_cluster_size(int device) {
  static std::mutex mu;
  static std::map<int, int> cache;
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find(device);
  if (it != cache.end()) return it->second;
  int best = 0;
  const size_t smem = 200 * 1024;
  if (smem_opt_in((const void*)qrcp_cluster_kernel, smem) == cudaSuccess) {
    for (int CL : {16, 8}) {
      if (CL > 8 && cudaFuncSetAttribute((const void*)qrcp_cluster_kernel,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed,
                                         1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      cudaLaunchAttribute attr[1];
      cudaLaunchConfig_t cfg = cluster_config(CL, kClMaxLocal * 32, smem, nullptr, attr);
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, (const void*)qrcp_cluster_kernel, &cfg) ==
              cudaSuccess &&
          n >= 1) {
        best = CL;
        break;
      }
      cudaGetLastError();
    }
  }
  cudaGetLastError();
  cache[device] = best;
  return best;
}

size_t qrcp_work_bytes(int64_t p, int64_t q, int max_grid) {
  int64_t kmax = p < q ? p : q;
  size_t b = 0;
  auto add = [&](size_t bytes) { b += (bytes + 255) / 256 * 256; };
  add(sizeof(double) * (size_t)(q * p));        // Rc
  add(sizeof(double) * (size_t)(kmax * p));     // V
  add(sizeof(double) * (size_t)kmax);           // tau
  add(sizeof(double) * (size_t)kmax);           // rdiag
  add(sizeof(int64_t) * (size_t)q);             // perm
  add((size_t)q);                               // used
  add(sizeof(double) * 2 * (size_t)max_grid * (size_t)(p + 2));   // slots
  add(sizeof(GridBar));
  add(sizeof(int64_t));                         // rank
  add(sizeof(double) * (size_t)(p * p));        // solve work
  return b;
}

void qrcp_carve(void* base, int64_t p, int64_t q, int max_grid, QrcpWork* w) {
  int64_t kmax = p < q ? p : q;
  char* c = static_cast<char*>(base);
  auto take = [&](size_t bytes) { void* r = c; c += (bytes + 255) / 256 * 256; return r; };
  w->Rc = (double*)take(sizeof(double) * (size_t)(q * p));
  w->V = (double*)take(sizeof(double) * (size_t)(kmax * p));
  w->tau = (double*)take(sizeof(double) * (size_t)kmax);
  w->rdiag = (double*)take(sizeof(double) * (size_t)kmax);
  w->perm = (int64_t*)take(sizeof(int64_t) * (size_t)q);
  w->used = (uint8_t*)take((size_t)q);
  w->slots = (double*)take(sizeof(double) * 2 * (size_t)max_grid * (size_t)(p + 2));
  w->bar = (GridBar*)take(sizeof(GridBar));
  w->rank = (int64_t*)take(sizeof(int64_t));
  w->Ysolve = (double*)take(sizeof(double) * (size_t)(p * p));
  w->max_grid = max_grid;
}

// Shared memory of the resident-column cooperative variant for a grid of g.
static size_t qrcp_coop_smem(int64_t p, int64_t q, int g) {
  int64_t nloc = (q + g - 1) / g;
  return sizeof(double) * (size_t)(nloc * p + p) + sizeof(int) * (size_t)nloc;
}

bool qrcp_resident(const LaunchEnv& env, int64_t p, int64_t q) {
  return qrcp_small_smem(p, q) > 0 || qrcp_coop_smem(p, q, qrcp_grid(env, p, q)) <= 200 * 1024;
}

int qrcp_grid(const LaunchEnv& env, int64_t p, int64_t q) {
  if (q <= 128) return 1;
  int64_t g = (q + 7) / 8;   // about 8 columns (one per warp) per CTA
  if (g > env.num_sms) g = env.num_sms;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_qrcp_pinv(const LaunchEnv& env, const double* M, int64_t p, int64_t q,
                             int64_t ldm, int thr_mode, double thr, double* scale_dev,
                             double* X, int64_t ldx, const QrcpWork& w, int grid,
                             DevStatus* st) {
  if (p <= 0 || q <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(w.bar, 0, sizeof(GridBar), env.stream);
  if (e != cudaSuccess) return e;
  QrcpParams P;
  P.M = M; P.p = p; P.q = q; P.ldm = ldm; P.thr_mode = thr_mode; P.thr = thr;
  P.scale_dev = scale_dev; P.w = w; P.st = st;
  const int CL = (p >= kSmallSplitP && p <= 512) ? qrcp_cluster_size(env.device) : 0;
  if (CL > 0 && q <= (int64_t)CL * kClMaxLocal && qrcp_cluster_smem(p, q, CL) <= 200 * 1024) {
    const size_t csm = qrcp_cluster_smem(p, q, CL);
    e = smem_opt_in((const void*)qrcp_cluster_kernel, csm);
    if (e != cudaSuccess) return e;
    int nw = (int)((q + CL - 1) / CL);
    nw = nw < 4 ? 4 : nw;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(CL, nw * 32, csm, env.stream, attr);
    e = cudaLaunchKernelEx(&cfg, qrcp_cluster_kernel, P);
  } else if (size_t ssm = qrcp_small_smem(p, q)) {
    if (p < kSmallSplitP) {  // tiny: factor and solve in one CTA
      e = smem_opt_in((const void*)qrcp_small_kernel<true>, ssm);
      if (e != cudaSuccess) return e;
      qrcp_small_kernel<true><<<1, kSmallThreads, ssm, env.stream>>>(P, X, ldx);
      return cudaGetLastError();
    }
    e = smem_opt_in((const void*)qrcp_small_kernel<false>, ssm);
    if (e != cudaSuccess) return e;
    qrcp_small_kernel<false><<<1, kSmallThreads, ssm, env.stream>>>(P, X, ldx);
    e = cudaGetLastError();
  } else if (const size_t csm = qrcp_coop_smem(p, q, grid); csm <= 200 * 1024) {
    if (csm > 0) {  // static shared memory adds to it: always opt in
      e = smem_opt_in((const void*)qrcp_factor_smem_kernel, csm);
      if (e != cudaSuccess) return e;
    }
    int nloc = (int)((q + grid - 1) / grid);
    void* args[] = {&P, &nloc};
    e = cudaLaunchCooperativeKernel((const void*)qrcp_factor_smem_kernel, dim3(grid),
                                    dim3(kThreads), args, csm, env.stream);
  } else {
    size_t smem = sizeof(double) * (size_t)p;
    if (smem > 0) {  // static shared memory adds to it: always opt in
      e = smem_opt_in((const void*)qrcp_factor_kernel, smem);
      if (e != cudaSuccess) return e;
    }
    void* args[] = {&P};
    e = cudaLaunchCooperativeKernel((const void*)qrcp_factor_kernel, dim3(grid), dim3(kThreads),
                                    args, smem, env.stream);
  }
  if (e != cudaSuccess) return e;
  SolveParams S;
  S.p = p; S.q = q; S.Rc = w.Rc; S.V = w.V; S.tau = w.tau; S.rdiag = w.rdiag; S.perm = w.perm;
  S.rank = w.rank; S.Ywork = w.Ysolve; S.X = X; S.ldx = ldx; S.st = st;
  unsigned blocks = (unsigned)((p + kWarps - 1) / kWarps);
  if (p <= kSolveSmallP) {
    const int64_t kmax = p < q ? p : q;
    const size_t ssm = sizeof(double) * (size_t)(kmax * p + kmax * kmax + 2 * kmax) +
                       sizeof(int) * (size_t)q;
    e = smem_opt_in((const void*)qrcp_solve_small_kernel, ssm);
    if (e != cudaSuccess) return e;
    const unsigned wpc = kSolveSmallThreads / 32;
    qrcp_solve_small_kernel<<<(unsigned)((p + wpc - 1) / wpc), kSolveSmallThreads, ssm, env.stream>>>(S);
    return cudaGetLastError();
  }
  qrcp_solve_kernel<<<blocks, kThreads, 0, env.stream>>>(S);
  return cudaGetLastError();
}

}  // namespace cur
