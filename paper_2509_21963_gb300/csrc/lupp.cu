// lupp.cu -- LU with partial pivoting as the index selector of IterativeCUR
// (arXiv 2509.21963, Sec. 3.2.1 column selection on the sketched residual
// S^col, Sec. 3.2.2 row selection on S^row; both selections of Algorithm 1).
//
// The candidates (columns of S^col, rows of A for S^row) are the ncand
// columns of an nr x ncand matrix X.  One cooperative launch performs all
// `steps` pivot steps: every CTA owns a contiguous slice of candidates in a
// working copy W (L2-resident: at most a few tens of MB), finds its local
// winner with warp-shuffle argmax on (|value| desc, index asc), publishes the
// winner's whole current column, and after ONE bounded grid barrier per step
// every CTA knows the global pivot and its column, and eliminates its own
// candidates with it (rank-1 Schur update, FP64).  Publication slots are
// double-buffered by step parity, which is what makes one barrier per step
// sufficient.
#include <climits>

#include "gridbar.cuh"

namespace cur {
namespace {

constexpr int kThreads = 256;

// Candidate magnitudes compare as integers: the bit pattern of |x| orders like
// |x| for every non-NaN double (GB300 runs FP64 instructions, compares
// included, at ~2 per clock per SM; integer compares run on the ALU).  A NaN
// gets -2, below "no candidate" (-1), so it never wins, as under FP64 compares.
__device__ __forceinline__ long long mag_key(double x) {
  const long long k = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL;
  return k > 0x7FF0000000000000LL ? -2 : k;
}

struct Best {
  long long a;  // mag_key of the value; -1 = none
  long long i;  // LLONG_MAX = none
};

__device__ __forceinline__ bool better(long long a, long long i, const Best& b) {
  return a > b.a || (a == b.a && i < b.i);
}

__device__ __forceinline__ Best warp_best(Best b) {
  for (int o = 16; o > 0; o >>= 1) {
    long long oa = __shfl_down_sync(0xffffffffu, b.a, o);
    long long oi = __shfl_down_sync(0xffffffffu, b.i, o);
    if (better(oa, oi, b)) { b.a = oa; b.i = oi; }
  }
  return b;
}

// warp_best with three 32-bit warp reductions (redux.sync) instead of five
// 64-bit shuffle rounds: the largest key's high word, then its low word among
// the lanes that hold that high word, then the smallest index among the lanes
// that hold the whole key.  Keys are >= -3 (shifted to >= 0 here); indices of
// candidates are below 2^31 (none: LLONG_MAX).  Every lane gets the result.
__device__ __forceinline__ Best warp_best_redux(const Best& b) {
  const unsigned long long u = (unsigned long long)(b.a + 3);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  const unsigned idx = (hi == mhi && lo == mlo && b.i != LLONG_MAX) ? (unsigned)b.i : 0xFFFFFFFFu;
  const unsigned mi = __reduce_min_sync(0xffffffffu, idx);
  Best r;
  r.a = (long long)(((unsigned long long)mhi << 32) | mlo) - 3;
  r.i = mi == 0xFFFFFFFFu ? LLONG_MAX : (long long)mi;
  return r;
}

// The winner among G per-CTA records {key, index, ...} (slot g at slot[g *
// stride]), read by one warp with every lane's loads in flight together; each
// lane returns the winner and its record number (-1 when no record has a
// candidate).
struct KeyWin {
  long long a, i;
  int g;
};
__device__ __forceinline__ KeyWin warp_slot_best_key(const double* slot, size_t stride, int G,
                                                     int lane) {
  constexpr int kR = 8;
  long long av[kR], iv[kR];
#pragma unroll
  for (int k = 0; k < kR; ++k) {
    const int g = lane + 32 * k;
    av[k] = -1;
    iv[k] = LLONG_MAX;
    if (g < G) {
      const double* s = slot + (size_t)g * stride;
      av[k] = __double_as_longlong(__ldcg(s));
      iv[k] = __double_as_longlong(__ldcg(s + 1));
    }
  }
  KeyWin c{-1, LLONG_MAX, -1};
#pragma unroll
  for (int k = 0; k < kR; ++k) {
    const int g = lane + 32 * k;
    if (g < G && (av[k] > c.a || (av[k] == c.a && iv[k] < c.i))) { c.a = av[k]; c.i = iv[k]; c.g = g; }
  }
  for (int g = lane + 32 * kR; g < G; g += 32) {  // grids above 256 CTAs
    const double* s = slot + (size_t)g * stride;
    const long long a = __double_as_longlong(__ldcg(s)), i = __double_as_longlong(__ldcg(s + 1));
    if (a > c.a || (a == c.a && i < c.i)) { c.a = a; c.i = i; c.g = g; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const long long oa = __shfl_xor_sync(0xffffffffu, c.a, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, c.i, o);
    const int og = __shfl_xor_sync(0xffffffffu, c.g, o);
    if (oa > c.a || (oa == c.a && oi < c.i)) { c.a = oa; c.i = oi; c.g = og; }
  }
  return c;
}

struct LuppParams {
  const double* X; int64_t ldx; int nr; int64_t ncand; int steps;
  uint8_t* mask; int64_t* piv;
  double* W;
  double* slots;  // [2][grid][stride]: abs, index bits, column values (stride: lupp_slot_stride)
  GridBar* bar; DevStatus* st;
};

__global__ void __launch_bounds__(kThreads) lupp_kernel(LuppParams p) {
  extern __shared__ double pv[];  // pivot column, nr entries
  __shared__ Best red[kThreads / 32];
  __shared__ Best s_win;
  __shared__ int s_wcta;
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int64_t per = (p.ncand + G - 1) / G;
  const int64_t lo = (int64_t)cta * per, hi = min(p.ncand, lo + per);
  const int64_t ldw = p.ncand;
  const int stride = (int)lupp_slot_stride(p.nr);

  for (int rr = 0; rr < p.nr; ++rr)
    for (int64_t i = lo + tid; i < hi; i += kThreads) p.W[rr * ldw + i] = p.X[rr * p.ldx + i];

  for (int t = 0; t < p.steps; ++t) {
    double* slot = p.slots + ((size_t)(t & 1) * G) * stride;
    // 1. local argmax over eligible owned candidates
    Best b{-1, LLONG_MAX};
    for (int64_t i = lo + tid; i < hi; i += kThreads) {
      if (p.mask[i]) continue;
      const long long a = mag_key(p.W[(int64_t)t * ldw + i]);
      if (better(a, i, b)) { b.a = a; b.i = i; }
    }
    b = warp_best(b);
    if (lane == 0) red[wid] = b;
    __syncthreads();
    if (wid == 0) {
      Best c = lane < kThreads / 32 ? red[lane] : Best{-1, LLONG_MAX};
      c = warp_best(c);
      if (lane == 0) s_win = c;
    }
    __syncthreads();
    Best mine = s_win;
    // 2. publish (|value|, index, current column) of the local winner
    double* my = slot + (size_t)cta * stride;
    if (tid == 0) { my[0] = __longlong_as_double(mine.a); my[1] = __longlong_as_double(mine.i); }
    if (mine.i != LLONG_MAX)
      for (int rr = t + tid; rr < p.nr; rr += kThreads) my[2 + rr] = p.W[rr * ldw + mine.i];
    __threadfence();
    if (!grid_barrier(p.bar, p.st)) return;
    // 3. global winner (every CTA computes the same answer)
    if (wid == 0) {
      const KeyWin c = warp_slot_best_key(slot, (size_t)stride, G, lane);
      if (lane == 0) { s_win = Best{c.a, c.i}; s_wcta = c.g; }
    }
    __syncthreads();
    Best w = s_win;
    if (w.i == LLONG_MAX) {  // no eligible candidate left anywhere
      if (tid == 0) dev_set_err(p.st, kDevNoCandidate);
      return;
    }
    const double* wcol = slot + (size_t)s_wcta * stride + 2;
    for (int rr = t + tid; rr < p.nr; rr += kThreads) pv[rr] = __ldcg(wcol + rr);
    if (cta == 0 && tid == 0) p.piv[t] = w.i;
    if (tid == 0 && w.i >= lo && w.i < hi) p.mask[w.i] = 1;
    __syncthreads();
    // 4. eliminate the owned eligible candidates against the pivot
    if (w.a > 0) {
      const double pt = pv[t];
      for (int64_t i = lo + tid; i < hi; i += kThreads) {
        if (p.mask[i]) continue;
        double l = p.W[(int64_t)t * ldw + i] / pt;
        for (int rr = t + 1; rr < p.nr; ++rr) {
          double* wp = p.W + rr * ldw + i;
          *wp = fma(-l, pv[rr], *wp);
        }
      }
    }
  }
}

// Blocked form of lupp_kernel for slices too large for shared memory: the
// features are taken in panels of KB rows.  Within a panel each CTA keeps its
// candidates' panel rows (Pn) and their multipliers (Lm) in shared memory and
// runs the steps there (one grid barrier per step, as above); the features
// below the panel are updated once per panel: the pivot candidates' trailing
// values follow by forward substitution, prow_s = W(:,p_s) - sum_{s'<s}
// l_{s',p_s} prow_{s'}, and every eligible candidate i then takes
// W(u,i) -= sum_s l_{s,i} prow_s(u).  Same pivots and arithmetic as the
// unblocked kernel up to the order of the trailing sums; W makes one L2 round
// trip per panel instead of one per step.
// Shared memory: Pn, Lm [KB][per]; prow [KB][nr]; pv [KB]; PL [KB][KB].
constexpr int kLuppKB = kLuppPanel;

__global__ void __launch_bounds__(kThreads) lupp_blocked_kernel(LuppParams p, int per, int KB) {
  extern __shared__ double sh[];
  double* Pn = sh;                                   // KB * per
  double* Lm = Pn + (size_t)KB * per;                // KB * per
  double* prow = Lm + (size_t)KB * per;              // KB * nr
  double* pv = prow + (size_t)KB * p.nr;             // KB
  double* PL = pv + KB;                              // KB * KB: PL[s * KB + s'] = l_{s', p_s}
  __shared__ Best red[kThreads / 32];
  __shared__ Best s_win;
  __shared__ int s_wcta;
  __shared__ long long s_piv[kLuppKB];
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int64_t lo = (int64_t)cta * per, hi = min(p.ncand, lo + per);
  const int own = (int)max((int64_t)0, hi - lo);
  const int64_t ldw = p.ncand;
  const int stride = (int)lupp_slot_stride(p.nr);  // >= 2 + 2 KB: abs, index, panel column, multipliers

  for (int rr = 0; rr < p.nr; ++rr)
    for (int64_t i = lo + tid; i < hi; i += kThreads) p.W[rr * ldw + i] = p.X[rr * p.ldx + i];
  __syncthreads();

  for (int t0 = 0; t0 < p.steps; t0 += KB) {
    const int nb = min(KB, p.nr - t0);          // rows of this panel
    const int ns = min(KB, p.steps - t0);       // steps of this panel
    for (int e = tid; e < nb * own; e += kThreads) {
      const int u = e / own, li = e - u * own;
      Pn[u * per + li] = p.W[(int64_t)(t0 + u) * ldw + lo + li];
      Lm[u * per + li] = 0.0;
    }
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
      const int t = t0 + s;
      double* slot = p.slots + ((size_t)(t & 1) * G) * stride;
      Best b{-1, LLONG_MAX};
      for (int li = tid; li < own; li += kThreads) {
        if (p.mask[lo + li]) continue;
        const long long a = mag_key(Pn[s * per + li]);
        if (better(a, lo + li, b)) { b.a = a; b.i = lo + li; }
      }
      b = warp_best(b);
      if (lane == 0) red[wid] = b;
      __syncthreads();
      if (wid == 0) {
        Best c = lane < kThreads / 32 ? red[lane] : Best{-1, LLONG_MAX};
        c = warp_best(c);
        if (lane == 0) s_win = c;
      }
      __syncthreads();
      const Best mine = s_win;
      double* my = slot + (size_t)cta * stride;
      if (tid == 0) { my[0] = __longlong_as_double(mine.a); my[1] = __longlong_as_double(mine.i); }
      if (mine.i != LLONG_MAX) {
        const int lw = (int)(mine.i - lo);
        for (int u = s + tid; u < nb; u += kThreads) my[2 + u] = Pn[u * per + lw];
        for (int q = tid; q < s; q += kThreads) my[2 + KB + q] = Lm[q * per + lw];
      }
      __threadfence();
      if (!grid_barrier(p.bar, p.st)) return;
      if (wid == 0) {
        const KeyWin c = warp_slot_best_key(slot, (size_t)stride, G, lane);
        if (lane == 0) { s_win = Best{c.a, c.i}; s_wcta = c.g; }
      }
      __syncthreads();
      const Best w = s_win;
      if (w.i == LLONG_MAX) {
        if (tid == 0) dev_set_err(p.st, kDevNoCandidate);
        return;
      }
      const double* wsl = slot + (size_t)s_wcta * stride;
      for (int u = s + tid; u < nb; u += kThreads) pv[u] = __ldcg(wsl + 2 + u);
      for (int q = tid; q < KB; q += kThreads) PL[s * KB + q] = q < s ? __ldcg(wsl + 2 + KB + q) : 0.0;
      if (tid == 0) {
        s_piv[s] = w.i;
        if (cta == 0) p.piv[t] = w.i;
        if (w.i >= lo && w.i < hi) p.mask[w.i] = 1;
      }
      __syncthreads();
      if (w.a > 0) {
        const double pivv = pv[s];
        for (int li = tid; li < own; li += kThreads) {
          if (p.mask[lo + li]) continue;
          const double l = Pn[s * per + li] / pivv;   // divided, as the oracle does
          Lm[s * per + li] = l;
          for (int u = s + 1; u < nb; ++u) Pn[u * per + li] = fma(-l, pv[u], Pn[u * per + li]);
        }
      }
      __syncthreads();
    }
    // write the panel rows back (later panels and the caller see W)
    for (int e = tid; e < nb * own; e += kThreads) {
      const int u = e / own, li = e - u * own;
      p.W[(int64_t)(t0 + u) * ldw + lo + li] = Pn[u * per + li];
    }
    const int r0 = t0 + nb;  // first trailing feature
    if (r0 < p.nr && t0 + ns < p.steps) {
      // pivot rows' trailing values: prow_s = W(:, p_s) - sum_{s' < s} l_{s', p_s} prow_{s'}
      for (int u = r0 + tid; u < p.nr; u += kThreads) {
        for (int s = 0; s < ns; ++s) {
          double v = __ldcg(p.W + (int64_t)u * ldw + s_piv[s]);
          for (int q = 0; q < s; ++q) v = fma(-PL[s * KB + q], prow[q * p.nr + u], v);
          prow[s * p.nr + u] = v;
        }
      }
      __syncthreads();
      // rank-ns update of the owned eligible candidates' trailing features
      for (int li = tid; li < own; li += kThreads) {
        if (p.mask[lo + li]) continue;
        double l[kLuppKB];
#pragma unroll
        for (int s = 0; s < kLuppKB; ++s) l[s] = s < ns ? Lm[s * per + li] : 0.0;
        for (int u = r0; u < p.nr; ++u) {
          double* wp = p.W + (int64_t)u * ldw + lo + li;
          double acc = *wp;
#pragma unroll
          for (int s = 0; s < kLuppKB; ++s)
            if (s < ns) acc = fma(-l[s], prow[s * p.nr + u], acc);
          *wp = acc;
        }
      }
    }
    __threadfence();
    __syncthreads();
  }
}

// Same selection with each CTA's candidate slice resident in shared memory:
// Wsh[rr * per + li] for candidate lo + li.  Used whenever the slice fits.
// The elimination of pivot t is split so that its FP64 work overlaps the
// exchange of step t+1: row t+1 (the next argmax) and the column of the CTA's
// next local best are updated at once and the record of step t+1 is
// published; then warp 0 waits for the grid barrier, reads every CTA's record
// and fetches the winner's column (into the second pivot buffer) while warps
// 1.. apply pivot t to the other rows.  At ~2 DFMA per clock per SM the FP64
// elimination takes as long as the exchange.  The multipliers divide,
// l_i = W(t, i) / pivot, as the oracle does.
__global__ void __launch_bounds__(kThreads) lupp_smem_kernel(LuppParams p, int per) {
  extern __shared__ double sh[];
  double* Wsh = sh;                                   // nr * per
  double* pvb = Wsh + (size_t)p.nr * per;             // 2 * nr: pivot columns, by step parity
  double* lm = pvb + 2 * p.nr;                        // per multipliers (0: skip)
  uint8_t* msk = reinterpret_cast<uint8_t*>(lm + per);   // per: not eligible
  __shared__ Best red[kThreads / 32];
  __shared__ Best s_win;
  __shared__ int s_ok;
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int64_t lo = (int64_t)cta * per;
  const int own = (int)max((int64_t)0, min((int64_t)per, p.ncand - lo));
  const int stride = (int)lupp_slot_stride(p.nr);
  unsigned long long* cnt = &p.bar->count;
  unsigned long long* xF = lupp_xchg(p.bar);          // [4] max key, by step mod 4
  unsigned long long* xM = xF + 4;                    // [4] max packed (key48, CTA)

  for (int e = tid; e < p.nr * own; e += kThreads) {
    int rr = e / own, li = e - rr * own;
    Wsh[rr * per + li] = p.X[rr * p.ldx + lo + li];
  }
  for (int li = tid; li < per; li += kThreads) {
    lm[li] = 0.0;
    msk[li] = li < own ? p.mask[lo + li] : 1;
  }
  __syncthreads();

  bool pending = false;   // pivot t-1 still to be applied to rows > t
  for (int t = 0; t < p.steps; ++t) {
    double* slot = p.slots + ((size_t)(t & 1) * G) * stride;
    const double* pv = pvb + (size_t)((t + 1) & 1) * p.nr;   // pivot t-1
    double* pvn = pvb + (size_t)(t & 1) * p.nr;              // pivot t (filled below)
    // row t with pivot t-1 (rows > t follow during the exchange), and the
    // local argmax over it; thread tid owns the slice entries li = tid (mod
    // kThreads) in every loop over li, so msk / lm / row t need no barrier
    const double pvt = pending ? pv[t] : 0.0;
    Best b{-1, LLONG_MAX};
    for (int li = tid; li < own; li += kThreads) {
      double v = Wsh[t * per + li];
      if (pending) { v = fma(-lm[li], pvt, v); Wsh[t * per + li] = v; }
      if (msk[li]) continue;
      const long long a = mag_key(v);
      if (better(a, lo + li, b)) { b.a = a; b.i = lo + li; }
    }
    b = warp_best_redux(b);
    if (lane == 0) red[wid] = b;
    __syncthreads();
    if (wid == 0) {
      Best c = lane < kThreads / 32 ? red[lane] : Best{-1, LLONG_MAX};
      c = warp_best_redux(c);
      if (lane == 0) s_win = c;
    }
    __syncthreads();
    const Best mine = s_win;
    double* my = slot + (size_t)cta * stride;
    if (tid == 0) { my[0] = __longlong_as_double(mine.a); my[1] = __longlong_as_double(mine.i); }
    if (mine.i != LLONG_MAX) {   // the candidate's column, rows > t with pivot t-1 applied
      const int lw = (int)(mine.i - lo);
      for (int rr = t + tid; rr < p.nr; rr += kThreads)
        my[2 + rr] = (rr == t || !pending) ? Wsh[rr * per + lw]
                                           : fma(-lm[lw], pv[rr], Wsh[rr * per + lw]);
    }
    __syncthreads();
    if (wid == 0) {
      // The exchange.  Every CTA folds its candidate into two maxima (the
      // exact 63-bit key; the key's top 48 bits with the CTA number, smaller
      // CTA winning ties) and then arrives with release semantics; after the
      // last arrival one CTA's record is read.  If that record's key is the
      // exact maximum it is the winner (every CTA with the same top 48 bits
      // and a smaller number would have won the packed maximum); otherwise
      // (a tie in the top 48 bits only) every record is read.
      const int x = t & 3;
      if (lane == 0) {
        if (mine.i != LLONG_MAX && mine.a >= -2) {
          const unsigned long long hi =
              mine.a >= 0 ? (unsigned long long)(mine.a >> 15) + 2ULL : 1ULL;   // NaN: 1
          if (mine.a >= 0) red_max_u64(xF + x, (unsigned long long)mine.a);
          red_max_u64(xM + x, (hi << 16) | (unsigned long long)(0xFFFF - cta));
        }
        red_release_add_u64(cnt, 1ULL);
      }
      __syncwarp();
      const bool ok = __all_sync(0xffffffffu, wait_count_acquire(cnt, (unsigned long long)(t + 1) * G, p.st));
      if (lane == 0) s_ok = ok ? 1 : 0;
      if (ok) {
        const unsigned long long F = __ldcg(xF + x), M = __ldcg(xM + x);
        const int gs = 0xFFFF - (int)(M & 0xFFFFu);
        bool hit = false;
        if (M != 0ULL && gs >= 0 && gs < G) {
          const double* rec = slot + (size_t)gs * stride;
          const long long ka = __double_as_longlong(__ldcg(rec));
          const long long ki = __double_as_longlong(__ldcg(rec + 1));
          if (ka >= 0 && (unsigned long long)ka == F) {
            hit = true;
            if (lane == 0) s_win = Best{ka, ki};
            for (int rr = t + lane; rr < p.nr; rr += 32) pvn[rr] = __ldcg(rec + 2 + rr);
          }
        }
        if (!hit) {   // the slow path: every record
          const KeyWin c = warp_slot_best_key(slot, (size_t)stride, G, lane);
          if (lane == 0) s_win = Best{c.a, c.i};
          if (c.i != LLONG_MAX) {
            const double* wcol = slot + (size_t)c.g * stride + 2;
            for (int rr = t + lane; rr < p.nr; rr += 32) pvn[rr] = __ldcg(wcol + rr);
          }
        }
        if (cta == 0 && lane == 0) {   // step t + 2's maxima (last read before step t's barrier)
          xF[(t + 2) & 3] = 0ULL;
          xM[(t + 2) & 3] = 0ULL;
        }
      }
    } else if (pending && t + 1 < p.nr) {   // rows > t with pivot t-1, meanwhile
      for (int rr = t + wid; rr < p.nr; rr += kThreads / 32 - 1) {   // warp per row
        if (rr == t) continue;
        const double pr = pv[rr];
        double* wr = Wsh + rr * per;
        for (int li = lane; li < own; li += 32) wr[li] = fma(-lm[li], pr, wr[li]);
      }
    }
    __syncthreads();
    if (!s_ok) return;
    const Best w = s_win;
    if (w.i == LLONG_MAX) {
      if (tid == 0) dev_set_err(p.st, kDevNoCandidate);
      return;
    }
    if (cta == 0 && tid == 0) p.piv[t] = w.i;
    pending = w.a > 0 && t + 1 < p.nr;   // a zero pivot eliminates nothing
    const double piv = pvn[t];
    for (int li = tid; li < own; li += kThreads) {
      if (lo + li == w.i) { msk[li] = 1; p.mask[w.i] = 1; }
      if (pending) lm[li] = msk[li] ? 0.0 : Wsh[t * per + li] / piv;
    }
  }
}

}  // namespace

size_t lupp_work_doubles(int64_t nr, int64_t ncand, int max_grid) {
  return (size_t)nr * ncand + 2 * (size_t)max_grid * (size_t)lupp_slot_stride(nr);
}

// Largest dynamic shared memory the resident-slice variant may use per CTA.
constexpr size_t kLuppSmemMax = 200 * 1024;

int lupp_grid(const LaunchEnv& env, int64_t nr, int64_t ncand) {
  int64_t g = (nr * ncand + 4095) / 4096;
  int64_t cap = env.num_sms;
  if (g > cap) g = cap;
  if (g > ncand) g = ncand;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_lupp(const LaunchEnv& env, const double* X, int64_t ldx, int64_t nr,
                        int64_t ncand, int64_t steps, uint8_t* mask, int64_t* piv,
                        const LuppWork& w, int grid, DevStatus* st) {
  if (steps <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(w.bar, 0, kLuppBarBytes, env.stream);
  if (e != cudaSuccess) return e;
  LuppParams p;
  p.X = X; p.ldx = ldx; p.nr = (int)nr; p.ncand = ncand; p.steps = (int)steps;
  p.mask = mask; p.piv = piv; p.W = w.W; p.slots = w.slot_val; p.bar = w.bar; p.st = st;
  const int64_t per = (ncand + grid - 1) / grid;
  const size_t smem_res = sizeof(double) * ((size_t)nr * per + 2 * nr + per) + (size_t)per;
  if (smem_res <= kLuppSmemMax) {
    if (smem_res > 0) {  // static shared memory adds to it: always opt in
      e = smem_opt_in((const void*)lupp_smem_kernel, smem_res);
      if (e != cudaSuccess) return e;
    }
    int per_i = (int)per;
    void* args[] = {&p, &per_i};
    return cudaLaunchCooperativeKernel((const void*)lupp_smem_kernel, dim3(grid), dim3(kThreads),
                                       args, smem_res, env.stream);
  }
  const int KB = kLuppKB;
  const size_t smem_blk =
      sizeof(double) * ((size_t)2 * KB * per + (size_t)KB * nr + KB + (size_t)KB * KB);
  if (smem_blk <= kLuppSmemMax) {
    e = smem_opt_in((const void*)lupp_blocked_kernel, smem_blk);
    if (e != cudaSuccess) return e;
    int per_i = (int)per, kb = KB;
    void* args[] = {&p, &per_i, &kb};
    return cudaLaunchCooperativeKernel((const void*)lupp_blocked_kernel, dim3(grid),
                                       dim3(kThreads), args, smem_blk, env.stream);
  }
  void* args[] = {&p};
  size_t smem = sizeof(double) * (size_t)(nr > 0 ? nr : 1);
  e = smem_opt_in((const void*)lupp_kernel, smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((const void*)lupp_kernel, dim3(grid), dim3(kThreads), args,
                                     smem, env.stream);
}

}  // namespace cur
