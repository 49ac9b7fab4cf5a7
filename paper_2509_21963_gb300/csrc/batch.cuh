// batch.cuh -- shared declarations of the batched IterativeCUR engine
// (batch.cu: the persistent kernel; cur_batch.cu: the C ABI and the tuner).
#pragma once

#include "cur_internal.cuh"

namespace cur {

constexpr int kBatchMaxB = 64;   // largest block size b of a batched job
constexpr int kBatchMaxC = 128;  // largest sketch size c of a batched job
// Phases timed by the team leaders: sketch, column LUPP, row residual, row
// LUPP + N^+, factor updates, core factorisation, core solve; the last slot
// counts jobs.
constexpr int kBatchPhases = 8;

// One job as the kernel sees it (validated and defaulted on the host).
struct BatchJobDev {
  const void* A;
  int64_t m, n, lda;
  double tol;
  int32_t b, c;
  uint64_t seed;
  int64_t rmax;      // min(m, n) or the caller's max_rank
  int64_t off_ij;    // offset of this job's I in Iout (rmax entries)
  int64_t off_j;     // offset of this job's J in Jout (rmax entries)
  int64_t off_u;     // offset of this job's U (rmax * rmax doubles; r x r used)
  int64_t off_hist;  // offset of this job's rho history (ceil(rmax / b) entries)
  char* ws;          // serving form: this job's own workspace (team part + CTA parts)
};

struct BatchOutDev {
  int64_t rank, iters;
  double rho, normY;
  int32_t status, pad;
  int64_t cycles;  // SM cycles of the team leader on this job
};

// Largest dimensions over the batch: they size the per-team and per-CTA
// scratch, which every job of the batch reuses.
struct BatchDims {
  int64_t M, N, C, B, R;
};

// Generalised-inverse workspace (team-shared for the core, CTA-private for N).
struct QrWs {
  double* Mc;     // q * p: column-major matrix, overwritten by R
  double* V;      // kmax * p reflectors
  double* tau;    // kmax
  double* rdiag;  // kmax
  int64_t* perm;  // kmax
  uint8_t* used;  // q
  double* norm2;  // q
  double* slots;  // 2 * T * 2 (pivot candidates per CTA, double-buffered)
  double* QT;     // p * p solve scratch
};

struct TeamWs {
  long long* job_slot;
  GridBar* bar;
  double* parts;  // T partial sums
  double *G, *S, *SrowT, *Lt, *Rt;
  QrWs qr;
};

struct CtaWs {
  double* W;                 // LUPP working copy
  uint8_t *maskc, *maskr;    // excluded columns / rows
  double *SJ, *T1, *Np;      // S(:,J_k), S(:,J_k) N^+, N^+
  double* vloc;              // this CTA's copy of the current reflector
  QrWs qr;                   // private QR of N
};

struct BatchLayout {
  size_t t_hdr, t_parts, t_G, t_S, t_SrowT, t_Lt, t_Rt, t_Mc, t_V, t_QT, t_tau, t_rdiag, t_perm,
      t_used, t_norm2, t_slots, team_bytes;
  size_t c_W, c_maskc, c_maskr, c_SJ, c_T1, c_Np, c_vloc, c_Mc, c_V, c_QT, c_tau, c_rdiag, c_perm,
      c_used, c_norm2, c_slots, cta_bytes;
};

__host__ __device__ inline BatchLayout batch_layout_dev(const BatchDims& d, int T) {
  BatchLayout L{};
  const size_t D = sizeof(double);
  size_t o = 0;
  auto put = [&](size_t bytes) {
    size_t at = o;
    o += (bytes + 255) & ~(size_t)255;
    return at;
  };
  L.t_hdr = put(256);
  L.t_parts = put(D * (size_t)T);
  L.t_G = put(D * (size_t)(d.C * d.M));
  L.t_S = put(D * (size_t)(d.C * d.N));
  L.t_SrowT = put(D * (size_t)(d.B * d.M));
  L.t_Lt = put(D * (size_t)(d.R * d.M));
  L.t_Rt = put(D * (size_t)(d.R * d.N));
  L.t_Mc = put(D * (size_t)(d.R * d.R));
  L.t_V = put(D * (size_t)(d.R * d.R));
  L.t_QT = put(D * (size_t)(d.R * d.R));
  L.t_tau = put(D * (size_t)d.R);
  L.t_rdiag = put(D * (size_t)d.R);
  L.t_perm = put(8 * (size_t)d.R);
  L.t_used = put((size_t)d.R);
  L.t_norm2 = put(D * (size_t)d.R);
  L.t_slots = put(D * 4 * (size_t)T);
  L.team_bytes = o;
  o = 0;
  const int64_t w = d.C * d.N > d.B * d.M ? d.C * d.N : d.B * d.M;
  L.c_W = put(D * (size_t)w);
  L.c_maskc = put((size_t)d.N);
  L.c_maskr = put((size_t)d.M);
  L.c_SJ = put(D * (size_t)(d.C * d.B));
  L.c_T1 = put(D * (size_t)(d.C * d.B));
  L.c_Np = put(D * (size_t)(d.B * d.B));
  L.c_vloc = put(D * (size_t)(d.R > d.B ? d.R : d.B));
  L.c_Mc = put(D * (size_t)(d.B * d.B));
  L.c_V = put(D * (size_t)(d.B * d.B));
  L.c_QT = put(D * (size_t)(d.B * d.B));
  L.c_tau = put(D * (size_t)d.B);
  L.c_rdiag = put(D * (size_t)d.B);
  L.c_perm = put(8 * (size_t)d.B);
  L.c_used = put((size_t)d.B);
  L.c_norm2 = put(D * (size_t)d.B);
  L.c_slots = put(D * 4);
  L.cta_bytes = o;
  return L;
}

__host__ __device__ inline TeamWs carve_team(char* base, const BatchDims& d, int T) {
  BatchLayout L = batch_layout_dev(d, T);
  TeamWs w;
  w.job_slot = reinterpret_cast<long long*>(base + L.t_hdr);
  w.bar = reinterpret_cast<GridBar*>(base + L.t_hdr + 64);
  w.parts = reinterpret_cast<double*>(base + L.t_parts);
  w.G = reinterpret_cast<double*>(base + L.t_G);
  w.S = reinterpret_cast<double*>(base + L.t_S);
  w.SrowT = reinterpret_cast<double*>(base + L.t_SrowT);
  w.Lt = reinterpret_cast<double*>(base + L.t_Lt);
  w.Rt = reinterpret_cast<double*>(base + L.t_Rt);
  w.qr.Mc = reinterpret_cast<double*>(base + L.t_Mc);
  w.qr.V = reinterpret_cast<double*>(base + L.t_V);
  w.qr.QT = reinterpret_cast<double*>(base + L.t_QT);
  w.qr.tau = reinterpret_cast<double*>(base + L.t_tau);
  w.qr.rdiag = reinterpret_cast<double*>(base + L.t_rdiag);
  w.qr.perm = reinterpret_cast<int64_t*>(base + L.t_perm);
  w.qr.used = reinterpret_cast<uint8_t*>(base + L.t_used);
  w.qr.norm2 = reinterpret_cast<double*>(base + L.t_norm2);
  w.qr.slots = reinterpret_cast<double*>(base + L.t_slots);
  return w;
}

__host__ __device__ inline CtaWs carve_cta(char* base, const BatchDims& d) {
  BatchLayout L = batch_layout_dev(d, 1);
  CtaWs w;
  w.W = reinterpret_cast<double*>(base + L.c_W);
  w.maskc = reinterpret_cast<uint8_t*>(base + L.c_maskc);
  w.maskr = reinterpret_cast<uint8_t*>(base + L.c_maskr);
  w.SJ = reinterpret_cast<double*>(base + L.c_SJ);
  w.T1 = reinterpret_cast<double*>(base + L.c_T1);
  w.Np = reinterpret_cast<double*>(base + L.c_Np);
  w.vloc = reinterpret_cast<double*>(base + L.c_vloc);
  w.qr.Mc = reinterpret_cast<double*>(base + L.c_Mc);
  w.qr.V = reinterpret_cast<double*>(base + L.c_V);
  w.qr.QT = reinterpret_cast<double*>(base + L.c_QT);
  w.qr.tau = reinterpret_cast<double*>(base + L.c_tau);
  w.qr.rdiag = reinterpret_cast<double*>(base + L.c_rdiag);
  w.qr.perm = reinterpret_cast<int64_t*>(base + L.c_perm);
  w.qr.used = reinterpret_cast<uint8_t*>(base + L.c_used);
  w.qr.norm2 = reinterpret_cast<double*>(base + L.c_norm2);
  w.qr.slots = reinterpret_cast<double*>(base + L.c_slots);
  return w;
}

struct BatchParams {
  const BatchJobDev* jobs;
  const int* order;            // queue position -> job (largest estimated work first)
  long long njobs;
  BatchOutDev* out;
  int64_t* Iout;
  int64_t* Jout;
  double* Uout;
  double* rho_hist;
  int64_t hist_len;            // unused bound marker (per-job lengths are in the jobs)
  unsigned long long* next;    // queue head (zeroed before each launch)
  DevStatus* st;
  char* team_scratch;
  size_t team_bytes;
  char* cta_scratch;
  size_t cta_bytes;
  BatchDims dims;
  int team;                    // CTAs per team (the small teams)
  int team_big;                // CTAs per big team (used when nbig > 0)
  int nbig;                    // big teams: CTAs [0, nbig * team_big)
  long long big_cut;           // queue positions [0, big_cut): the big jobs, served by big teams
  unsigned long long* next_small;   // head of the queue positions [big_cut, njobs)
  int tile_n;                  // outputs per thread and pass of the residual products (4 or 8)
  unsigned long long* prof;    // kBatchPhases cycle sums of the team leaders (zeroed per launch)
  size_t panel_bytes;          // dynamic shared memory for the core solve panel (0: none)
};

// Largest dynamic shared memory of the batch kernel (the core solve panel).
constexpr size_t kBatchMaxPanelBytes = 160 * 1024;
// Co-resident CTAs of the batch kernel (256 threads) with `dyn_smem` bytes.
int batch_max_ctas(const LaunchEnv& env, int threads, bool a_f32, size_t dyn_smem);
// Dynamic shared memory of the core solve for cores up to rmax: the widest
// panel (8, 4 or 2 columns of rmax doubles) that fits kBatchMaxPanelBytes with
// 256 threads; 0 when none fits (the per-column solve then runs).
size_t batch_panel_bytes(int64_t rmax);

// Whole-GPU pivoted-QR generalised inverse (the team QR of the batch kernel
// with one team made of every SM), X = P [R11^{-1} Q1^T; 0] (q x p, row stride
// ldx) of the p x q matrix Mc (column-major, overwritten; Mc must be the start
// of `work`, which holds core_qr_work_bytes(p, q, T) bytes).  thr < 0: rank
// threshold max(p,q) 2^-52 |R_00|.  core_qr_grid returns T (0: not runnable).
struct CoreQrParams {
  QrWs w;
  double* vloc;
  size_t vloc_stride;
  GridBar* bar;
  DevStatus* st;
  int64_t p, q;
  double thr;
  double* X;
  int64_t ldx;
  size_t panel_bytes;
  int64_t* rank_out;
};
size_t core_qr_work_bytes(int64_t p, int64_t q, int T);
int core_qr_grid(const LaunchEnv& env, int64_t p);
cudaError_t launch_core_qr(const LaunchEnv& env, double* Mc, int64_t p, int64_t q, double thr,
                           double* X, int64_t ldx, void* work, int T, DevStatus* st,
                           int64_t* rank_out);

// Serving form (one cluster of `team` CTAs per job, per-job workspaces).
size_t serve_job_scratch_bytes(const BatchDims& d, int team);
int serve_max_clusters(const LaunchEnv& env, int team, bool a_f32, size_t panel);
cudaError_t launch_serve(const LaunchEnv& env, const BatchParams& P, int team, bool a_f32);
// Cooperative launch of `grid` CTAs (a multiple of P.team, <= batch_max_ctas).
cudaError_t launch_batch(const LaunchEnv& env, const BatchParams& P, int grid, int threads,
                         bool a_f32);

}  // namespace cur
