// cur_api.cu -- C ABI and host orchestration of IterativeCUR (arXiv
// 2509.21963, Algorithm 1) on one GPU.
//
// Per run:  G (seeded Gaussian, c x m)  ->  S = Y = G A, ||Y||_F   (one pass of A)
// Per iteration k (the loop of Algorithm 1, residuals through Lemma 1):
//   J_k  = LUPP(S^col)                       cooperative selection kernel
//   S^row = A(:,J_k) - L Rt(:,J_k)           gather + FP64 GEMM   (m x b)
//   I_k  = LUPP(S^row)
//   Rt_k = A(I_k,:) - L(I_k,:) Rt            gather + FP64 GEMM   (b x n)
//   N^+  = pinv(S^row(I_k,:))                pivoted QR, one CTA
//   L_k  = S^row N^+                         FP64 GEMM            (m x b)
//   S^col -= (S^col(:,J_k) N^+) Rt_k, ||S^col||_F   fused GEMM + sum of squares
//   rho = ||S^col||_F / ||Y||_F              8-byte read-back, host decides
// At exit U = A(I,J)^+ by pivoted QR (the paper's default QR).
// Lemma 1 gives S_k = A - sum_l L_l Rt_l with L_l = S_{l-1}(:,J_l) N_l^+ and
// Rt_l = S_{l-1}(I_l,:): the same row and column residuals, without an
// explicit U inside the loop.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cur.h"
#include "../../include/cur_steps.h"
#include "cur_internal.cuh"
#include "ctx.cuh"
#include "batch.cuh"

using namespace cur;

struct cur_result {
  cur_ctx* ctx = nullptr;
  int64_t rank = 0, iters = 0;
  int status = CUR_OK;
  double rho = 1.0, normY = 0.0;
  int64_t* I = nullptr;
  int64_t* J = nullptr;
  double* U = nullptr;
  void* block = nullptr;      // one device allocation holding U, I and J
  size_t block_bytes = 0;
  std::vector<double> rho_hist;
  double phase_ms[CUR_PHASE_COUNT] = {0};
  int64_t launches = 0;
  bool host_valid = false;
  std::vector<int64_t> I_host, J_host;
  std::vector<double> U_host;
};

namespace {

// Largest r for which the core solve U = A(I,J)^+ runs (its reflector lives
// in shared memory); runs of larger matrices stop there (CUR_TOL_UNREACHED).
constexpr int64_t kMaxCoreRank = 16384;

int fail(cur_ctx* ctx, int code, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = msg;
  return code;
}

}  // namespace

int cur::ctx_fail_v(cur_ctx* ctx, int code, const char* msg) {
  if (ctx) ctx->err = msg;
  return code;
}

namespace {

// A failed call's error is also the runtime's pending error: clear it, so that
// the next call on this context does not report it again.
#define CK(expr)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      cudaGetLastError();                                                                 \
      return fail(ctx, CUR_ECUDA, "%s failed: %s (%d)", #expr, cudaGetErrorString(e_),    \
                  (int)e_);                                                               \
    }                                                                                     \
  } while (0)

#define TRY(expr)                   \
  do {                              \
    int s_ = (expr);                \
    if (s_ != CUR_OK) return s_;    \
  } while (0)

// Grow-only named workspace; contents are not preserved unless keep > 0.
int ensure(cur_ctx* ctx, BufId id, size_t bytes, size_t keep = 0) {
  DevBuf& b = ctx->buf[id];
  if (bytes == 0) bytes = 1;
  bytes = (bytes + 255) / 256 * 256;
  if (b.bytes >= bytes) return CUR_OK;
  size_t grow = b.bytes + b.bytes / 2;
  if (keep == 0 && grow > bytes) bytes = (grow + 255) / 256 * 256;
  if (ctx->budget && ctx->held - b.bytes + bytes > ctx->budget)
    return fail(ctx, CUR_EBUDGET, "workspace of %zu bytes exceeds the HBM budget of %zu bytes",
                ctx->held - b.bytes + bytes, ctx->budget);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, CUR_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  if (keep && b.p) {
    e = cudaMemcpyAsync(p, b.p, keep < b.bytes ? keep : b.bytes, cudaMemcpyDeviceToDevice,
                        ctx->stream);
    if (e != cudaSuccess) { cudaFree(p); return fail(ctx, CUR_ECUDA, "workspace copy failed"); }
  }
  if (b.p) {   // nothing on the context's streams may still use the old buffer
    cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
    if (ctx->side_stream) cudaStreamSynchronize(ctx->side_stream);
    cudaFree(b.p);
  }
  ctx->held = ctx->held - b.bytes + bytes;
  b.p = p;
  b.bytes = bytes;
  return CUR_OK;
}

template <typename T>
T* bp(cur_ctx* ctx, BufId id) { return static_cast<T*>(ctx->buf[id].p); }

LaunchEnv env_of(cur_ctx* ctx) { return LaunchEnv{ctx->stream, ctx->num_sms, ctx->device}; }

// Record a phase boundary: the interval from this event to the next one is
// charged to `phase` (-1 closes the previous interval).
void tick(cur_ctx* ctx, int phase) {
  if (!ctx->timing) return;
  size_t i = ctx->ev_phase.size();
  if (i >= ctx->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); ctx->timing = false; return; }
    ctx->ev_pool.push_back(e);
  }
  cudaEventRecord(ctx->ev_pool[i], ctx->stream);
  ctx->ev_phase.push_back(phase);
}

void collect_phases(cur_ctx* ctx, cur_result* res) {
  if (!ctx->timing) return;
  cudaStreamSynchronize(ctx->stream);
  for (size_t i = 0; i + 1 < ctx->ev_phase.size(); ++i) {
    int ph = ctx->ev_phase[i];
    if (ph < 0 || ph >= CUR_PHASE_COUNT) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev_pool[i], ctx->ev_pool[i + 1]) == cudaSuccess)
      res->phase_ms[ph] += ms;
    else
      cudaGetLastError();
  }
  ctx->ev_phase.clear();
}

// Read the device status block; translate a device error.
int read_status(cur_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->st_host, ctx->buf[B_STATUS].p, sizeof(DevStatus),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->st_host->err == kDevTimeout)
    return fail(ctx, CUR_ETIMEOUT, "a device-side grid barrier exceeded its cycle budget");
  if (ctx->st_host->err == kDevNoCandidate)
    return fail(ctx, CUR_EINVAL, "no eligible pivot: LUPP ran out of candidates, or every remaining QR column norm is NaN");
  if (ctx->st_host->err != 0) return fail(ctx, CUR_ECUDA, "device status %d", ctx->st_host->err);
  return CUR_OK;
}

DevStatus* dstat(cur_ctx* ctx) { return bp<DevStatus>(ctx, B_STATUS); }

int lupp_call(cur_ctx* ctx, BufId wid, const double* X, int64_t ldx, int64_t nr, int64_t ncand,
              int64_t steps, uint8_t* mask, int64_t* piv) {
  LaunchEnv env = env_of(ctx);
  int grid = lupp_grid(env, nr, ncand);
  TRY(ensure(ctx, wid, sizeof(double) * lupp_work_doubles(nr, ncand, grid) + 256));
  LuppWork w;
  w.W = bp<double>(ctx, wid);
  w.slot_val = w.W + (size_t)nr * ncand;
  w.bar = reinterpret_cast<GridBar*>(w.slot_val + 2 * (size_t)grid * (size_t)lupp_slot_stride(nr));
  w.max_grid = grid;
  CK(launch_lupp(env, X, ldx, nr, ncand, steps, mask, piv, w, grid, dstat(ctx)));
  ctx->launches += 1;
  return CUR_OK;
}

int pinv_call(cur_ctx* ctx, BufId wid, const double* M, int64_t p, int64_t q, int64_t ldm,
              int thr_mode, double thr, double* scale_dev, double* X, int64_t ldx) {
  LaunchEnv env = env_of(ctx);
  int grid = qrcp_grid(env, p, q);
  TRY(ensure(ctx, wid, qrcp_work_bytes(p, q, grid)));
  QrcpWork w;
  qrcp_carve(ctx->buf[wid].p, p, q, grid, &w);
  CK(launch_qrcp_pinv(env, M, p, q, ldm, thr_mode, thr, scale_dev, X, ldx, w, grid, dstat(ctx)));
  ctx->launches += 2;
  return CUR_OK;
}

int gemm(cur_ctx* ctx, GemmArgs g) {
  if (g.M <= 0 || g.N <= 0) return CUR_OK;
  CK(launch_gemm(env_of(ctx), g));
  ctx->launches += g.ksplit > 1 ? 2 : 1;
  return CUR_OK;
}

// (rlim, clim): extent of the source in its (r, c) index space.
int gather(cur_ctx* ctx, const void* X, bool f32, int64_t ldx, bool trans, const int64_t* ridx,
           const int64_t* cidx, int64_t rows, int64_t cols, int64_t rlim, int64_t clim,
           double* out, int64_t ldo) {
  if (rows <= 0 || cols <= 0) return CUR_OK;
  CK(launch_gather2d(env_of(ctx), X, f32, ldx, trans, ridx, cidx, rows, cols, rlim, clim, out, ldo));
  ctx->launches += 1;
  return CUR_OK;
}

// Square cores whose pivoted QR no longer fits the shared-memory kernels of
// qrcp.cu (rank above ~1800 on 152 SMs) are factored by the whole-GPU team QR
// of batch.cu when its solve panel fits (rank up to 10240); the rest by qrcp.cu.
bool team_core(const LaunchEnv& env, int64_t p, int64_t q) {
  return p == q && !qrcp_resident(env, p, q) && batch_panel_bytes(p) > 0;
}

// Core: U = A(I,J)^+ (r x r), relative rank threshold max(p,q) 2^-52 |R_00|.
// Mc: an r x r scratch for the small-core path.
int core_solve(cur_ctx* ctx, const void* A, bool f32, int64_t lda, int64_t m, int64_t n,
               const int64_t* I, const int64_t* J, int64_t r, double* Mc, double* U) {
  LaunchEnv env = env_of(ctx);
  const int T = team_core(env, r, r) ? core_qr_grid(env, r) : 0;
  if (T > 0) {
    TRY(ensure(ctx, B_TEAMCORE, core_qr_work_bytes(r, r, T)));
    double* W = bp<double>(ctx, B_TEAMCORE);
    // column-major A(I,J): W[col * r + i] = A(I[i], J[col])
    TRY(gather(ctx, A, f32, lda, true, J, I, r, r, n, m, W, r));
    CK(launch_core_qr(env, W, r, r, -1.0, U, r, W, T, dstat(ctx), nullptr));
    ctx->launches += 1;
    return CUR_OK;
  }
  TRY(gather(ctx, A, f32, lda, false, I, J, r, r, m, n, Mc, r));
  return pinv_call(ctx, B_QRBIG, Mc, r, r, r, 0, 0.0, nullptr, U, r);
}

int sum_parts(cur_ctx* ctx, const double* parts, int64_t n, double* out) {
  CK(launch_sum_parts(env_of(ctx), parts, n, out));
  ctx->launches += 1;
  return CUR_OK;
}

GemmArgs gargs(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
               bool tA, const void* B, int64_t ldb, bool tB, bool bf32, double beta,
               const double* Cin, int64_t ldcin, double* D, int64_t ldd) {
  GemmArgs g{};
  g.M = M; g.N = N; g.K = K; g.alpha = alpha; g.A = A; g.lda = lda; g.transA = tA;
  g.B = B; g.ldb = ldb; g.transB = tB; g.b_is_f32 = bf32; g.beta = beta; g.Cin = Cin;
  g.ldcin = ldcin; g.D = D; g.ldd = ldd; g.sumsq_part = nullptr; g.partial = nullptr;
  g.ksplit = 1;
  return g;
}

// Y = G A with FP64 arithmetic into Y, ||Y||^2 into status scalar[slot].
int sketch_f64(cur_ctx* ctx, const double* G, int64_t c, const void* A, bool a_f32, int64_t m,
               int64_t n, int64_t lda, double* Y, int slot, BufId parts_id) {
  LaunchEnv env = env_of(ctx);
  SketchPlan plan = plan_sketch_simt(env, c, m, n);
  double* partial = nullptr;
  if (plan.partial_doubles) {
    TRY(ensure(ctx, B_SPLITK, sizeof(double) * plan.partial_doubles));
    partial = bp<double>(ctx, B_SPLITK);
  }
  TRY(ensure(ctx, parts_id, sizeof(double) * (size_t)plan.sumsq_parts));
  double* parts = bp<double>(ctx, parts_id);
  CK(launch_sketch_simt(env, plan, G, m, c, A, a_f32, lda, m, n, Y, partial, parts));
  ctx->launches += plan.ks > 1 ? 2 : 1;
  TRY(sum_parts(ctx, parts, plan.sumsq_parts, &dstat(ctx)->scalar[slot]));
  return CUR_OK;
}

// Y = G A with A arriving from host memory: A is copied to A_dev in row blocks
// on the context's copy stream, and the sketch of each block starts as soon
// as its copy lands, so the copy of block k+1 overlaps the sketch of block k;
// the blocks' split-K slices are summed in one fixed-order reduction.
int sketch_f64_from_host(cur_ctx* ctx, const double* G, int64_t c, const void* A_host,
                         int64_t lda_host, void* A_dev, bool a_f32, int64_t m, int64_t n,
                         double* Y, int slot, BufId parts_id) {
  LaunchEnv env = env_of(ctx);
  const int nb = m >= 8192 ? 8 : (m >= 2048 ? 4 : 1);
  const int64_t rows = (m + nb - 1) / nb;
  const size_t es = a_f32 ? 4 : 8;
  if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  while ((int)ctx->copy_ev.size() < nb + 1) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->copy_ev.push_back(e);
  }
  std::vector<SketchPlan> plans;
  int64_t nslices = 0;
  for (int k = 0; k < nb; ++k) {
    const int64_t r0 = k * rows, rk = std::min(rows, m - r0);
    if (rk <= 0) break;
    plans.push_back(plan_sketch_simt(env, c, rk, n));
    nslices += plans.back().ks;
  }
  TRY(ensure(ctx, B_SPLITK, sizeof(double) * (size_t)nslices * (size_t)(c * n)));
  const int64_t nparts = sketch_reduce_parts(c, n);
  TRY(ensure(ctx, parts_id, sizeof(double) * (size_t)nparts));
  double* slices = bp<double>(ctx, B_SPLITK);
  // the copies may only overwrite A_dev once earlier work on the stream is done
  CK(cudaEventRecord(ctx->copy_ev[nb], ctx->stream));
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_ev[nb], 0));
  const char* src = static_cast<const char*>(A_host);
  char* dst = static_cast<char*>(A_dev);
  for (size_t k = 0; k < plans.size(); ++k) {
    const int64_t r0 = (int64_t)k * rows, rk = std::min(rows, m - r0);
    CK(cudaMemcpy2DAsync(dst + (size_t)r0 * n * es, (size_t)n * es, src + (size_t)r0 * lda_host * es,
                         (size_t)lda_host * es, (size_t)n * es, (size_t)rk, cudaMemcpyHostToDevice,
                         ctx->copy_stream));
    CK(cudaEventRecord(ctx->copy_ev[k], ctx->copy_stream));
  }
  int64_t z = 0;
  for (size_t k = 0; k < plans.size(); ++k) {
    const int64_t r0 = (int64_t)k * rows, rk = std::min(rows, m - r0);
    CK(cudaStreamWaitEvent(ctx->stream, ctx->copy_ev[k], 0));
    CK(launch_sketch_simt_slices(env, plans[k], G + r0, m, c, dst + (size_t)r0 * n * es, a_f32, n,
                                 rk, n, slices + (size_t)z * (size_t)(c * n)));
    z += plans[k].ks;
    ctx->launches += 1;
  }
  double* parts = bp<double>(ctx, parts_id);
  CK(launch_sketch_reduce(env, slices, (int)nslices, c, n, Y, parts));
  ctx->launches += 1;
  TRY(sum_parts(ctx, parts, nparts, &dstat(ctx)->scalar[slot]));
  return CUR_OK;
}

// Precision form: Y = G_q fix_S(A) on the tensor cores, ||Y||^2 into scalar[slot].
int sketch_q(cur_ctx* ctx, int S, const double* G, int64_t c, const float* A, int64_t m,
             int64_t n, int64_t lda, double* Y, int slot, BufId parts_id, BufId scratch_id) {
  LaunchEnv env = env_of(ctx);
  int ks = sketch_tc_plan_ks(env, m, n);
  TRY(ensure(ctx, scratch_id, sketch_tc_scratch_bytes(c, m, n, ks)));
  // one partial per 256 columns and 16 rows of the reduction
  const int64_t nparts_max = ((n + 255) / 256) * ((c + 15) / 16);
  TRY(ensure(ctx, parts_id, sizeof(double) * (size_t)nparts_max));
  int64_t nparts = 0;
  CK(launch_sketch_tc(env, S, G, c, A, lda, m, n, ctx->buf[scratch_id].p, ks, Y,
                      bp<double>(ctx, parts_id), &nparts, &dstat(ctx)->err));
  ctx->launches += 5;
  TRY(sum_parts(ctx, bp<double>(ctx, parts_id), nparts, &dstat(ctx)->scalar[slot]));
  return CUR_OK;
}

// FP64 form on the tensor cores: Y = RN(G_q trunc(A 2^(52-E_j))) 2^(E_j-52),
// ||Y||^2 into scalar[slot].
int sketch_fx(cur_ctx* ctx, const double* G, int64_t c, const double* A, int64_t m, int64_t n,
              int64_t lda, double* Y, int slot, BufId parts_id, BufId scratch_id) {
  LaunchEnv env = env_of(ctx);
  TRY(ensure(ctx, scratch_id, sketch_fx_scratch_bytes(c, m, n)));
  TRY(ensure(ctx, parts_id, sizeof(double) * (size_t)sketch_fx_max_parts(c, n)));
  int64_t nparts = 0;
  tick(ctx, CUR_PHASE_SCALES);
  CK(launch_sketch_fx_scales(env, G, c, A, lda, m, n, ctx->buf[scratch_id].p));
  tick(ctx, CUR_PHASE_SKETCH);
  CK(launch_sketch_fx_main(env, c, A, lda, m, n, ctx->buf[scratch_id].p, Y,
                           bp<double>(ctx, parts_id), &nparts, &dstat(ctx)->err));
  ctx->launches += 4 + (c + 63) / 64;
  TRY(sum_parts(ctx, bp<double>(ctx, parts_id), nparts, &dstat(ctx)->scalar[slot]));
  return CUR_OK;
}

// The FP64 tensor-core sketch with G generated from the seed: G and G_q on
// the side stream while the column-scale pass reads A on the context's stream
// (independent work: the FP64 Philox / Box-Muller kernel and an HBM-bound read),
// joined before the tensor-core pass.
int sketch_fx_seeded(cur_ctx* ctx, uint64_t seed, int64_t c, const double* A, int64_t m,
                     int64_t n, int64_t lda, double* Y, int slot, BufId parts_id, BufId scratch_id) {
  LaunchEnv env = env_of(ctx);
  TRY(ensure(ctx, B_OMEGA, sizeof(double) * (size_t)(c * m)));
  TRY(ensure(ctx, scratch_id, sketch_fx_scratch_bytes(c, m, n)));
  TRY(ensure(ctx, parts_id, sizeof(double) * (size_t)sketch_fx_max_parts(c, n)));
  if (!ctx->side_stream) CK(cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking));
  for (auto& ev : ctx->side_ev)
    if (!ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  LaunchEnv side = env;
  side.stream = ctx->side_stream;
  double* G = bp<double>(ctx, B_OMEGA);
  void* scratch = ctx->buf[scratch_id].p;
  tick(ctx, CUR_PHASE_SCALES);
  CK(cudaEventRecord(ctx->side_ev[0], env.stream));
  CK(cudaStreamWaitEvent(side.stream, ctx->side_ev[0], 0));
  CK(launch_gaussian(side, seed, c, m, G, m));
  CK(launch_sketch_fx_q8(side, G, c, m, n, scratch));
  CK(cudaEventRecord(ctx->side_ev[1], side.stream));
  CK(launch_sketch_fx_colscales(env, c, A, lda, m, n, scratch));
  CK(cudaStreamWaitEvent(env.stream, ctx->side_ev[1], 0));
  tick(ctx, CUR_PHASE_SKETCH);
  // (a column-blocked form that read the scales of block k + 1 on the side
  // stream during the tensor-core pass over block k was slower: 1.78 against
  // 1.63 ms at 20000^2, the pass slowing down next to the concurrent read)
  int64_t nparts = 0;
  CK(launch_sketch_fx_main(env, c, A, lda, m, n, scratch, Y, bp<double>(ctx, parts_id), &nparts,
                           &dstat(ctx)->err));
  ctx->launches += 5 + (c + 63) / 64;
  TRY(sum_parts(ctx, bp<double>(ctx, parts_id), nparts, &dstat(ctx)->scalar[slot]));
  return CUR_OK;
}

// The FP64 tensor-core sketch with A arriving from host memory.  A is copied
// into A_dev on the context's copy stream in column groups at least 8192
// columns wide (pitched copies with shorter rows run well below the host
// link's rate), each group in row blocks.  The column maxima of a row block
// are taken as soon as it lands; once a group is complete its exponents and
// its tensor-core pass follow, under the copy of the next group, so only the
// last group's pass is left when the copy ends.  G (given, or drawn from the
// seed) and G_q are formed on the side stream meanwhile.  Every group adds
// exact integer sums into its own columns, so Y equals the device-resident
// form's bit for bit.
int sketch_fx_from_host(cur_ctx* ctx, const double* G, uint64_t seed, int64_t c,
                        const void* A_host, int64_t lda_host, double* A_dev, int64_t m, int64_t n,
                        double* Y, int slot, BufId parts_id, BufId scratch_id) {
  LaunchEnv env = env_of(ctx);
  const int64_t ng = std::max<int64_t>(1, n / 8192);
  const int64_t w = ((n + ng - 1) / ng + 127) / 128 * 128;
  const int64_t nr = m >= 1024 ? std::min<int64_t>(8, m / 512) : 1;
  const int64_t rows = (m + nr - 1) / nr;
  const int nev = (int)(ng * nr);
  if (!G) TRY(ensure(ctx, B_OMEGA, sizeof(double) * (size_t)(c * m)));
  TRY(ensure(ctx, scratch_id, sketch_fx_scratch_bytes(c, m, n)));
  TRY(ensure(ctx, parts_id, sizeof(double) * (size_t)sketch_fx_max_parts(c, n)));
  if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  if (!ctx->side_stream) CK(cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking));
  for (auto& ev : ctx->side_ev)
    if (!ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  while ((int)ctx->copy_ev.size() < nev + 1) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->copy_ev.push_back(e);
  }
  LaunchEnv side = env;
  side.stream = ctx->side_stream;
  void* scratch = ctx->buf[scratch_id].p;
  const size_t es = sizeof(double);
  const char* src = static_cast<const char*>(A_host);
  tick(ctx, CUR_PHASE_SCALES);
  // the copies and the side stream may only start once earlier work on the
  // context's stream (a previous run reading A_dev, G or the scratch) is done
  CK(cudaEventRecord(ctx->copy_ev[nev], env.stream));
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_ev[nev], 0));
  CK(cudaStreamWaitEvent(side.stream, ctx->copy_ev[nev], 0));
  for (int64_t g = 0; g < ng; ++g) {
    const int64_t c0 = g * w, wg = std::min(w, n - c0);
    for (int64_t k = 0; k < nr; ++k) {
      const int64_t r0 = k * rows, rk = std::min(rows, m - r0);
      if (wg > 0 && rk > 0)
        CK(cudaMemcpy2DAsync(A_dev + r0 * n + c0, (size_t)n * es,
                             src + ((size_t)r0 * (size_t)lda_host + (size_t)c0) * es,
                             (size_t)lda_host * es, (size_t)wg * es, (size_t)rk,
                             cudaMemcpyHostToDevice, ctx->copy_stream));
      CK(cudaEventRecord(ctx->copy_ev[g * nr + k], ctx->copy_stream));
    }
  }
  if (!G) {
    G = bp<double>(ctx, B_OMEGA);
    CK(launch_gaussian(side, seed, c, m, const_cast<double*>(G), m));
    ctx->launches += 1;
  }
  CK(launch_sketch_fx_q8(side, G, c, m, n, scratch));
  CK(cudaEventRecord(ctx->side_ev[1], side.stream));
  CK(launch_sketch_fx_zero(env, c, A_dev, n, m, n, scratch));
  bool joined = false;
  for (int64_t g = 0; g < ng; ++g) {
    const int64_t c0 = g * w, c1 = std::min(n, c0 + w);
    if (c0 >= c1) break;
    for (int64_t k = 0; k < nr; ++k) {
      const int64_t r0 = k * rows, r1 = std::min(m, r0 + rows);
      CK(cudaStreamWaitEvent(env.stream, ctx->copy_ev[g * nr + k], 0));
      if (r0 < r1) {
        CK(launch_sketch_fx_colmax_block(env, c, A_dev, n, m, n, scratch, r0, r1, c0, c1));
        ctx->launches += 1;
      }
    }
    CK(launch_sketch_fx_colexp_range(env, c, A_dev, n, m, n, scratch, c0, c1));
    if (!joined) {
      CK(cudaStreamWaitEvent(env.stream, ctx->side_ev[1], 0));
      tick(ctx, CUR_PHASE_SKETCH);
      joined = true;
    }
    CK(launch_sketch_fx_main_range(env, c, A_dev, n, m, n, scratch, c0, c1, &dstat(ctx)->err));
    ctx->launches += 1 + (c + 63) / 64;
  }
  int64_t nparts = 0;
  CK(launch_sketch_fx_reduce(env, c, A_dev, n, m, n, scratch, Y, bp<double>(ctx, parts_id),
                             &nparts));
  ctx->launches += 2;
  TRY(sum_parts(ctx, bp<double>(ctx, parts_id), nparts, &dstat(ctx)->scalar[slot]));
  return CUR_OK;
}

int check_fx_form(cur_ctx* ctx, const void* A, int64_t lda, int dtype) {
  if (dtype != CUR_F64) return fail(ctx, CUR_EINVAL, "the FP64 tensor-core sketch needs FP64 A");
  if (lda % 2 != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0)
    return fail(ctx, CUR_EINVAL, "the FP64 tensor-core sketch needs lda %% 2 == 0 and a 16-byte aligned A");
  return CUR_OK;
}

int check_precision_form(cur_ctx* ctx, int S, const void* A, int64_t lda, int dtype, int64_t c) {
  if (S < 1 || S > 4) return fail(ctx, CUR_EINVAL, "unknown sketch_mode %d", S);
  if (dtype != CUR_F32) return fail(ctx, CUR_EINVAL, "the precision forms of the sketch need FP32 A");
  if (lda % 4 != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0)
    return fail(ctx, CUR_EINVAL, "the precision forms need lda %% 4 == 0 and a 16-byte aligned A");
  if (sketch_tc_cpad((int)c, S) < 0)
    return fail(ctx, CUR_EINVAL, "sketch_size %lld too large for sketch_mode %d (c <= 128, <= 80 for S = 3, <= 64 for S = 4)",
                (long long)c, S);
  return CUR_OK;
}

int validate(cur_ctx* ctx, const void* A, int64_t m, int64_t n, int64_t lda, int dtype,
             double tol, int b, int* c, const cur_opts* o, int64_t* max_rank, double* tol_eff) {
  if (!ctx) return CUR_EINVAL;
  if (!A) return fail(ctx, CUR_EINVAL, "A is NULL");
  if (m < 1 || n < 1) return fail(ctx, CUR_EINVAL, "m and n must be >= 1");
  if (lda < n) return fail(ctx, CUR_EINVAL, "lda (%lld) < n (%lld)", (long long)lda, (long long)n);
  if (dtype != CUR_F64 && dtype != CUR_F32) return fail(ctx, CUR_EINVAL, "unknown dtype %d", dtype);
  if (!(tol > 0.0)) return fail(ctx, CUR_EINVAL, "tol must be > 0 (got %g)", tol);
  if (b < 1) return fail(ctx, CUR_EINVAL, "block_size must be >= 1");
  if (*c == 0) *c = (11 * b) / 10;
  if (*c < b) return fail(ctx, CUR_EINVAL, "sketch_size (%d) < block_size (%d)", *c, b);
  int64_t mn = m < n ? m : n;
  if (mn > kMaxCoreRank) mn = kMaxCoreRank;
  *max_rank = mn;
  *tol_eff = tol;
  if (o) {
    if (o->max_rank < 0) return fail(ctx, CUR_EINVAL, "max_rank < 0");
    if (o->max_rank > 0 && o->max_rank < mn) *max_rank = o->max_rank;
    if (o->sketch_mode == CUR_SKETCH_F64_TC)
      TRY(check_fx_form(ctx, A, lda, dtype));
    else if (o->sketch_mode != CUR_SKETCH_F64)
      TRY(check_precision_form(ctx, o->sketch_mode, A, lda, dtype, *c));
    if (o->residual_planes != 0 && o->residual_planes != 2 && o->residual_planes != 3)
      return fail(ctx, CUR_EINVAL, "residual_planes must be 0, 2 or 3");
    if (o->residual_planes != 0 && b > 128)
      return fail(ctx, CUR_EINVAL, "residual_planes needs block_size <= 128");
    if (o->alpha != 0.0) {
      if (!(o->alpha > 0.0 && o->alpha < 1.0) || !(o->delta >= 0.0))
        return fail(ctx, CUR_EINVAL, "alpha must be in (0,1) and delta >= 0");
      double la = -std::log(o->alpha);
      if (!((double)*c > 4.0 * la))
        return fail(ctx, CUR_EINVAL, "risk-aware stop needs c > -4 ln(alpha) = %g", 4.0 * la);
      *tol_eff = tol * (1.0 + o->delta) * std::sqrt(1.0 - 2.0 * std::sqrt(la / (double)*c));
    }
  }
  return CUR_OK;
}

// A_host (optional): A arrives from host memory (row stride lda_host) and A is
// the device buffer it is copied into; the FP64 sketch then overlaps the copy.
int run_device(cur_ctx* ctx, const void* A, int64_t m, int64_t n, int64_t lda, int dtype,
               double tol, int b, int c, uint64_t seed, const cur_opts* o, cur_result** out,
               const void* A_host = nullptr, int64_t lda_host = 0) {
  int64_t max_rank;
  double tol_eff;
  TRY(validate(ctx, A, m, n, lda, dtype, tol, b, &c, o, &max_rank, &tol_eff));
  CK(cudaSetDevice(ctx->device));
  const bool f32 = dtype == CUR_F32;
  cudaStream_t s = ctx->stream;
  LaunchEnv env = env_of(ctx);
  ctx->timing = o && o->timing;
  ctx->ev_phase.clear();
  ctx->launches = 0;

  TRY(ensure(ctx, B_STATUS, sizeof(DevStatus)));
  CK(cudaMemsetAsync(ctx->buf[B_STATUS].p, 0, sizeof(DevStatus), s));
  double minus1 = -1.0;
  CK(cudaMemcpyAsync(&dstat(ctx)->scalar[2], &minus1, sizeof(double), cudaMemcpyHostToDevice, s));

  // sketch matrix G; initial sketch S_0 = Y = G A and ||Y||_F (the one full pass over A)
  const double* G = o ? o->omega : nullptr;
  const int smode0 = o ? o->sketch_mode : CUR_SKETCH_F64;
  const bool fx_seeded = smode0 == CUR_SKETCH_F64_TC && !G;
  if (!G && !fx_seeded) {
    TRY(ensure(ctx, B_OMEGA, sizeof(double) * (size_t)(c * m)));
    tick(ctx, CUR_PHASE_GAUSSIAN);
    CK(launch_gaussian(env, seed, c, m, bp<double>(ctx, B_OMEGA), m));
    ctx->launches += 1;
    G = bp<double>(ctx, B_OMEGA);
  }
  TRY(ensure(ctx, B_S, sizeof(double) * (size_t)(c * n)));
  double* S = bp<double>(ctx, B_S);
  TRY(ensure(ctx, B_PARTS, sizeof(double) * 4096));
  tick(ctx, CUR_PHASE_SKETCH);
  const int smode = o ? o->sketch_mode : CUR_SKETCH_F64;
  if (smode == CUR_SKETCH_F64 && A_host) {
    TRY(sketch_f64_from_host(ctx, G, c, A_host, lda_host, const_cast<void*>(A), f32, m, n, S, 0,
                             B_PARTS));
  } else if (smode == CUR_SKETCH_F64) {
    TRY(sketch_f64(ctx, G, c, A, f32, m, n, lda, S, 0, B_PARTS));
  } else if (smode == CUR_SKETCH_F64_TC && A_host) {
    TRY(sketch_fx_from_host(ctx, fx_seeded ? nullptr : G, seed, c, A_host, lda_host,
                            static_cast<double*>(const_cast<void*>(A)), m, n, S, 0, B_PARTS, B_FX));
  } else if (smode == CUR_SKETCH_F64_TC && fx_seeded) {
    TRY(sketch_fx_seeded(ctx, seed, c, static_cast<const double*>(A), m, n, lda, S, 0, B_PARTS,
                         B_FX));
  } else if (smode == CUR_SKETCH_F64_TC) {
    TRY(sketch_fx(ctx, G, c, static_cast<const double*>(A), m, n, lda, S, 0, B_PARTS, B_FX));
  } else {
    TRY(sketch_q(ctx, smode, G, c, static_cast<const float*>(A), m, n, lda, S, 0, B_PARTS, B_TC));
  }
  tick(ctx, -1);
  // ||G A||_F^2 comes back with the first iteration's rho (one host round trip
  // less per run); a non-finite or zero sketch is handled there, before that
  // iteration's results are used.
  double nY = -1.0;
  cur_result* res = new cur_result();
  res->ctx = ctx;
  auto take_norm = [&]() -> int {   // after a read_status: ||G A||_F from the status block
    const double nY2 = ctx->st_host->scalar[0];
    if (!std::isfinite(nY2)) return fail(ctx, CUR_ENONFINITE, "A contains Inf or NaN");
    nY = std::sqrt(nY2);
    res->normY = nY;
    return CUR_OK;
  };

  // index arrays and masks
  int64_t rcap = max_rank < 256 ? max_rank : 256;
  if (rcap < b) rcap = b < max_rank ? b : max_rank;
  auto fail_res = [&](int code) { delete res; return code; };
  int st;
  if ((st = ensure(ctx, B_I, sizeof(int64_t) * (size_t)max_rank)) != CUR_OK) return fail_res(st);
  if ((st = ensure(ctx, B_J, sizeof(int64_t) * (size_t)max_rank)) != CUR_OK) return fail_res(st);
  if ((st = ensure(ctx, B_MASKC, (size_t)n)) != CUR_OK) return fail_res(st);
  if ((st = ensure(ctx, B_MASKR, (size_t)m)) != CUR_OK) return fail_res(st);
  if ((st = ensure(ctx, B_LT, sizeof(double) * (size_t)(rcap * m))) != CUR_OK) return fail_res(st);
  if ((st = ensure(ctx, B_RT, sizeof(double) * (size_t)(rcap * n))) != CUR_OK) return fail_res(st);
  const size_t bsz = (size_t)b;
  if ((st = ensure(ctx, B_SROWT, sizeof(double) * bsz * m)) != CUR_OK) return fail_res(st);
  if ((st = ensure(ctx, B_N, sizeof(double) * bsz * bsz)) != CUR_OK) return fail_res(st);
  if ((st = ensure(ctx, B_NP, sizeof(double) * bsz * bsz)) != CUR_OK) return fail_res(st);
  if ((st = ensure(ctx, B_SJK, sizeof(double) * (size_t)c * bsz)) != CUR_OK) return fail_res(st);
  if ((st = ensure(ctx, B_T1, sizeof(double) * (size_t)c * bsz)) != CUR_OK) return fail_res(st);
  {
    cudaError_t e1 = cudaMemsetAsync(ctx->buf[B_MASKC].p, 0, (size_t)n, s);
    cudaError_t e2 = cudaMemsetAsync(ctx->buf[B_MASKR].p, 0, (size_t)m, s);
    cudaError_t e3 = cudaMemsetAsync(ctx->buf[B_I].p, 0, sizeof(int64_t) * (size_t)max_rank, s);
    cudaError_t e4 = cudaMemsetAsync(ctx->buf[B_J].p, 0, sizeof(int64_t) * (size_t)max_rank, s);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess)
      return fail_res(fail(ctx, CUR_ECUDA, "memset failed"));
  }
  int64_t* Id = bp<int64_t>(ctx, B_I);
  int64_t* Jd = bp<int64_t>(ctx, B_J);
  uint8_t* maskc = bp<uint8_t>(ctx, B_MASKC);
  uint8_t* maskr = bp<uint8_t>(ctx, B_MASKR);
  // residual products on the tensor cores: L and Rt as BF16 planes, K-major
  // (PLT: m rows, PRT: n rows, pitch kcap), and the gathered rows of the other
  // factor (QP: b rows)
  const int np = o ? o->residual_planes : 0;
  const int64_t kcap = np ? resid_plane_pitch(max_rank) : 0;
  __nv_bfloat16 *plt[3] = {nullptr, nullptr, nullptr}, *prt[3] = {nullptr, nullptr, nullptr},
                *pq[3] = {nullptr, nullptr, nullptr};
  if (np) {
    if ((st = ensure(ctx, B_PLT, 2 * (size_t)np * (size_t)(m * kcap))) != CUR_OK) return fail_res(st);
    if ((st = ensure(ctx, B_PRT, 2 * (size_t)np * (size_t)(n * kcap))) != CUR_OK) return fail_res(st);
    if ((st = ensure(ctx, B_QP, 2 * (size_t)np * (size_t)(b * kcap))) != CUR_OK) return fail_res(st);
    const int64_t kb = resid_plane_pitch(b);   // the planes of S^row and -N^+ for L_k
    if ((st = ensure(ctx, B_PS, 2 * (size_t)np * (size_t)(m * kb))) != CUR_OK) return fail_res(st);
    if ((st = ensure(ctx, B_PNP, 2 * (size_t)np * (size_t)(b * kb))) != CUR_OK) return fail_res(st);
    if ((st = ensure(ctx, B_PRK, 2 * (size_t)np * (size_t)(n * kb))) != CUR_OK) return fail_res(st);
    if ((st = ensure(ctx, B_PT1, 2 * (size_t)np * (size_t)(c * kb))) != CUR_OK) return fail_res(st);
    for (int q = 0; q < 3; ++q) {
      const size_t qq = (size_t)(q < np ? q : 0);
      plt[q] = bp<__nv_bfloat16>(ctx, B_PLT) + qq * (size_t)(m * kcap);
      prt[q] = bp<__nv_bfloat16>(ctx, B_PRT) + qq * (size_t)(n * kcap);
      pq[q] = bp<__nv_bfloat16>(ctx, B_QP) + qq * (size_t)(b * kcap);
    }
  }

  double rho = 1.0;
  int64_t r = 0;
  int64_t lt_bk = 0;   // rows of L^T still to form from the last iteration's S^row and N^+
  while (rho > tol_eff && r < max_rank) {  // Algorithm 1's loop test
    const int64_t bk = (int64_t)b < max_rank - r ? (int64_t)b : max_rank - r;
    if (r + bk > rcap) {  // grow the Lemma 1 factors, keeping their content
      int64_t nc = rcap * 2 > r + bk ? rcap * 2 : r + bk;
      if (nc > max_rank) nc = max_rank;
      if ((st = ensure(ctx, B_LT, sizeof(double) * (size_t)(nc * m), sizeof(double) * (size_t)(r * m))) != CUR_OK) return fail_res(st);
      if ((st = ensure(ctx, B_RT, sizeof(double) * (size_t)(nc * n), sizeof(double) * (size_t)(r * n))) != CUR_OK) return fail_res(st);
      rcap = nc;
    }
    double* LT = bp<double>(ctx, B_LT);   // rows: L_l^T (L is m x r)
    double* Rt = bp<double>(ctx, B_RT);   // rows: Rt_l  (r x n)
    double* SrowT = bp<double>(ctx, B_SROWT);
    int64_t* Jk = Jd + r;
    int64_t* Ik = Id + r;
    if (lt_bk > 0) {   // L_{k-1}^T = N^+^T S^row^T of the last iteration: needed only now that
                       // the loop goes on (its S^row and N^+ are still in place)
      tick(ctx, CUR_PHASE_FACTORS);
      double* LTk = LT + (size_t)(r - lt_bk) * m;
      if (np) {   // on the tensor cores: L^T_k(t, i) = 0 - sum_k' S^row(i, k') (-N^+(k', t))
        const int64_t kb = resid_plane_pitch(lt_bk);
        __nv_bfloat16 *ps[3], *pn[3];
        for (int q = 0; q < 3; ++q) {
          const size_t qq = (size_t)(q < np ? q : 0);
          ps[q] = bp<__nv_bfloat16>(ctx, B_PS) + qq * (size_t)(m * kb);
          pn[q] = bp<__nv_bfloat16>(ctx, B_PNP) + qq * (size_t)(lt_bk * kb);
        }
        cudaError_t e = launch_split_planes(env, SrowT, m, 1, lt_bk, m, ps, np, kb, 0);
        if (e == cudaSuccess)
          e = launch_split_planes(env, bp<double>(ctx, B_NP), lt_bk, 1, lt_bk, lt_bk, pn, np, kb, 0,
                                  true);
        if (e == cudaSuccess)
          e = cudaMemsetAsync(LTk, 0, sizeof(double) * (size_t)(lt_bk * m), s);
        if (e == cudaSuccess)
          e = launch_resid_tc(env, np, ps, kb, m, pn, kb, (int)lt_bk, lt_bk, LTk, m, &dstat(ctx)->err);
        if (e != cudaSuccess) return fail_res(fail(ctx, CUR_ECUDA, "L_k: %s", cudaGetErrorString(e)));
        ctx->launches += 3;
      } else if ((st = gemm(ctx, gargs(lt_bk, m, lt_bk, 1.0, bp<double>(ctx, B_NP), lt_bk, true, SrowT,
                                       m, false, false, 0.0, nullptr, 0, LTk, m))) != CUR_OK) {
        return fail_res(st);
      }
      if (np) {   // its planes: PLT(i, r - lt_bk + t) from L^T(r - lt_bk + t, i)
        if (cudaError_t e = launch_split_planes(env, LT + (size_t)(r - lt_bk) * m, m, 1, lt_bk, m,
                                                plt, np, kcap, r - lt_bk); e != cudaSuccess)
          return fail_res(fail(ctx, CUR_ECUDA, "split_planes: %s", cudaGetErrorString(e)));
        ctx->launches += 1;
      }
      lt_bk = 0;
    }

    // column selection: J_k = LUPP on S^col (candidates: the n columns)
    tick(ctx, CUR_PHASE_LUPP_COL);
    if ((st = lupp_call(ctx, B_LUPPW, S, n, c, n, bk, maskc, Jk)) != CUR_OK) return fail_res(st);
    // row residual: S^row^T = A(:,J_k)^T - Rt(:,J_k)^T L^T   (bk x m)
    tick(ctx, CUR_PHASE_ROW_RES);
    if ((st = gather(ctx, A, f32, lda, true, Jk, nullptr, bk, m, n, m, SrowT, m)) != CUR_OK)
      return fail_res(st);
    if (r > 0 && np) {   // S^row^T(t, i) -= sum_k L(i, k) Rt(k, J_k[t]) on the tensor cores
      cudaError_t e = launch_gather_plane_rows(env, prt, np, kcap, n, Jk, (int)bk,
                                               resid_plane_pitch(r), pq, kcap);
      if (e == cudaSuccess)
        e = launch_resid_tc(env, np, plt, kcap, m, pq, kcap, (int)bk, r, SrowT, m, &dstat(ctx)->err);
      if (e != cudaSuccess) return fail_res(fail(ctx, CUR_ECUDA, "resid_tc: %s", cudaGetErrorString(e)));
      ctx->launches += 2;
    } else if (r > 0) {
      if ((st = ensure(ctx, B_G1, sizeof(double) * (size_t)(rcap * bk))) != CUR_OK) return fail_res(st);
      double* G1 = bp<double>(ctx, B_G1);
      if ((st = gather(ctx, Rt, false, n, false, nullptr, Jk, r, bk, r, n, G1, bk)) != CUR_OK)
        return fail_res(st);
      if ((st = gemm(ctx, gargs(bk, m, r, -1.0, G1, bk, true, LT, m, false, false, 1.0, SrowT, m,
                                SrowT, m))) != CUR_OK) return fail_res(st);
    }
    // row selection: I_k = LUPP on S^row (candidates: the m rows)
    tick(ctx, CUR_PHASE_LUPP_ROW);
    if ((st = lupp_call(ctx, B_LUPPW, SrowT, m, bk, m, bk, maskr, Ik)) != CUR_OK) return fail_res(st);
    // N = S^row(I_k, :) = S_{k-1}(I_k, J_k)
    tick(ctx, CUR_PHASE_FACTORS);
    double* Nd = bp<double>(ctx, B_N);
    double* Np = bp<double>(ctx, B_NP);
    if ((st = gather(ctx, SrowT, false, m, true, Ik, nullptr, bk, bk, m, bk, Nd, bk)) != CUR_OK)
      return fail_res(st);
    // Rt_k = A(I_k,:) - L(I_k,:) Rt
    double* Rk = Rt + (size_t)r * n;
    if ((st = gather(ctx, A, f32, lda, false, Ik, nullptr, bk, n, m, n, Rk, n)) != CUR_OK)
      return fail_res(st);
    if (r > 0 && np) {   // R_k(t, j) -= sum_k Rt(k, j) L(I_k[t], k) on the tensor cores
      cudaError_t e = launch_gather_plane_rows(env, plt, np, kcap, m, Ik, (int)bk,
                                               resid_plane_pitch(r), pq, kcap);
      if (e == cudaSuccess)
        e = launch_resid_tc(env, np, prt, kcap, n, pq, kcap, (int)bk, r, Rk, n, &dstat(ctx)->err);
      if (e != cudaSuccess) return fail_res(fail(ctx, CUR_ECUDA, "resid_tc: %s", cudaGetErrorString(e)));
      ctx->launches += 2;
    } else if (r > 0) {
      if ((st = ensure(ctx, B_G2, sizeof(double) * (size_t)(rcap * bk))) != CUR_OK) return fail_res(st);
      double* G2 = bp<double>(ctx, B_G2);
      if ((st = gather(ctx, LT, false, m, false, nullptr, Ik, r, bk, r, m, G2, bk)) != CUR_OK)
        return fail_res(st);
      if ((st = gemm(ctx, gargs(bk, n, r, -1.0, G2, bk, true, Rt, n, false, false, 1.0, Rk, n,
                                Rk, n))) != CUR_OK) return fail_res(st);
    }
    if (np) {   // R_k's planes: PRT(j, r + t) from R_k(t, j)
      if (cudaError_t e = launch_split_planes(env, Rk, n, 1, bk, n, prt, np, kcap, r); e != cudaSuccess)
        return fail_res(fail(ctx, CUR_ECUDA, "split_planes: %s", cudaGetErrorString(e)));
      ctx->launches += 1;
    }
    // N^+ by pivoted QR; rank threshold |I| 2^-52 |R_00(N_1)|
    if ((st = pinv_call(ctx, B_QRSMALL, Nd, bk, bk, bk, 2, (double)(r + bk),
                        &dstat(ctx)->scalar[2], Np, bk)) != CUR_OK) return fail_res(st);
    // L_k^T = (S^row N^+)^T = N^+^T S^row^T (bk x m) is formed at the top of
    // the next iteration, if there is one
    lt_bk = bk;
    // column residual (Lemma 1): S^col -= (S^col(:,J_k) N^+) Rt_k, fused ||S^col||^2
    tick(ctx, CUR_PHASE_COL_RES);
    double* SJk = bp<double>(ctx, B_SJK);
    double* T1 = bp<double>(ctx, B_T1);
    if ((st = gather(ctx, S, false, n, false, nullptr, Jk, c, bk, c, n, SJk, bk)) != CUR_OK)
      return fail_res(st);
    if ((st = gemm(ctx, gargs(c, bk, bk, 1.0, SJk, bk, false, Np, bk, false, false, 0.0, nullptr, 0,
                              T1, bk))) != CUR_OK) return fail_res(st);
    if (np && c <= 128) {   // S^col(i, j) -= sum_t T1(i, t) R_k(t, j) on the tensor cores,
                            // then ||S^col||_F^2 in FP64
      const int64_t kb = resid_plane_pitch(bk);
      __nv_bfloat16 *pr[3], *pt[3];
      for (int q = 0; q < 3; ++q) {
        const size_t qq = (size_t)(q < np ? q : 0);
        pr[q] = bp<__nv_bfloat16>(ctx, B_PRK) + qq * (size_t)(n * kb);
        pt[q] = bp<__nv_bfloat16>(ctx, B_PT1) + qq * (size_t)(c * kb);
      }
      const int64_t nparts = resid_sumsq_parts();
      if ((st = ensure(ctx, B_PARTS, sizeof(double) * (size_t)nparts)) != CUR_OK) return fail_res(st);
      cudaError_t e = launch_split_planes(env, Rk, n, 1, bk, n, pr, np, kb, 0);
      if (e == cudaSuccess) e = launch_split_planes(env, T1, 1, bk, bk, c, pt, np, kb, 0);
      if (e == cudaSuccess)
        e = launch_resid_tc(env, np, pr, kb, n, pt, kb, (int)c, bk, S, n, &dstat(ctx)->err);
      if (e == cudaSuccess) e = launch_sumsq_parts(env, S, c, n, n, bp<double>(ctx, B_PARTS));
      if (e != cudaSuccess) return fail_res(fail(ctx, CUR_ECUDA, "S^col: %s", cudaGetErrorString(e)));
      ctx->launches += 4;
      if ((st = sum_parts(ctx, bp<double>(ctx, B_PARTS), nparts, &dstat(ctx)->scalar[1])) != CUR_OK)
        return fail_res(st);
    } else {
      GemmArgs g = gargs(c, n, bk, -1.0, T1, bk, false, Rk, n, false, false, 1.0, S, n, S, n);
      int64_t np = gemm_num_sumsq_parts(g);
      if ((st = ensure(ctx, B_PARTS, sizeof(double) * (size_t)np)) != CUR_OK) return fail_res(st);
      g.sumsq_part = bp<double>(ctx, B_PARTS);
      if ((st = gemm(ctx, g)) != CUR_OK) return fail_res(st);
      if ((st = sum_parts(ctx, g.sumsq_part, np, &dstat(ctx)->scalar[1])) != CUR_OK)
        return fail_res(st);
    }
    // rho_k (the host needs it for the loop test)
    tick(ctx, -1);
    const int st_iter = read_status(ctx);
    if (nY < 0.0) {
      if ((st = take_norm()) != CUR_OK) return fail_res(st);
      if (nY == 0.0) {  // G A = 0: nothing to approximate (this iteration is discarded)
        rho = 0.0;
        break;
      }
    }
    if (st_iter != CUR_OK) return fail_res(st_iter);
    r += bk;
    rho = std::sqrt(ctx->st_host->scalar[1]) / nY;
    res->rho_hist.push_back(rho);
  }
  if (nY < 0.0) {   // the loop did not run (tol >= 1): read the norm now
    if ((st = read_status(ctx)) != CUR_OK) return fail_res(st);
    if ((st = take_norm()) != CUR_OK) return fail_res(st);
    if (nY == 0.0) rho = 0.0;
  }

  // core of the returned CUR: U = A(I,J)^+ by pivoted QR
  res->rank = r;
  res->iters = (int64_t)res->rho_hist.size();
  res->rho = rho;
  res->status = rho > tol_eff ? CUR_TOL_UNREACHED : CUR_OK;
  if (r > 0) {
    // U, I and J in one block, reused from the context's pool of freed result
    // blocks when one is large enough (no allocation on the repeated-run path)
    const size_t ub = (sizeof(double) * (size_t)(r * r) + 255) / 256 * 256;
    const size_t need = ub + 2 * ((sizeof(int64_t) * (size_t)r + 255) / 256 * 256);
    void* blk = nullptr;
    size_t blk_bytes = 0;
    for (size_t k = 0; k < ctx->result_pool.size(); ++k)
      if (ctx->result_pool[k].second >= need) {
        blk = ctx->result_pool[k].first;
        blk_bytes = ctx->result_pool[k].second;
        ctx->result_pool.erase(ctx->result_pool.begin() + (std::ptrdiff_t)k);
        break;
      }
    if (!blk) {
      if (cudaMalloc(&blk, need) != cudaSuccess) {
        cudaGetLastError();
        return fail_res(fail(ctx, CUR_ENOMEM, "result allocation failed"));
      }
      blk_bytes = need;
    }
    res->block = blk;
    res->block_bytes = blk_bytes;
    res->U = static_cast<double*>(blk);
    res->I = reinterpret_cast<int64_t*>(static_cast<char*>(blk) + ub);
    res->J = reinterpret_cast<int64_t*>(static_cast<char*>(blk) + ub +
                                        (sizeof(int64_t) * (size_t)r + 255) / 256 * 256);
    CK(cudaMemcpyAsync(res->I, Id, sizeof(int64_t) * (size_t)r, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(res->J, Jd, sizeof(int64_t) * (size_t)r, cudaMemcpyDeviceToDevice, s));
    if ((st = ensure(ctx, B_CORE, sizeof(double) * (size_t)(r * r))) != CUR_OK) { cur_result_free(res); return st; }
    double* Mc = bp<double>(ctx, B_CORE);
    tick(ctx, CUR_PHASE_CORE);
    if (res->iters == 1 && !team_core(env, r, r)) {
      // One iteration: A(I,J) = A(I_1,J_1) = N_1 entry for entry (S_0 = A), the
      // core solve would run the same pivoted-QR kernels on it, and its rank
      // threshold max(p,q) 2^-52 |R_00| equals N_1^+'s (r 2^-52 |R_00(N_1)|), so
      // U = N_1^+ bit for bit: reuse it.
      CK(cudaMemcpyAsync(res->U, bp<double>(ctx, B_NP), sizeof(double) * (size_t)(r * r),
                         cudaMemcpyDeviceToDevice, s));
    } else if ((st = core_solve(ctx, A, f32, lda, m, n, res->I, res->J, r, Mc, res->U)) != CUR_OK) {
      cur_result_free(res);
      return st;
    }
    tick(ctx, -1);
    if ((st = read_status(ctx)) != CUR_OK) { cur_result_free(res); return st; }
  }
  collect_phases(ctx, res);
  res->launches = ctx->launches;
  *out = res;
  return res->status;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int cur_create(cur_ctx** out, int device, void* cuda_stream, size_t hbm_budget_bytes) {
  if (!out) return CUR_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return CUR_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) return CUR_ECUDA;
  cur_ctx* ctx = new cur_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->budget = hbm_budget_bytes;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMallocHost((void**)&ctx->st_host, sizeof(DevStatus)) != cudaSuccess) {
    delete ctx;
    return CUR_ENOMEM;
  }
  *out = ctx;
  return CUR_OK;
}

void cur_free(cur_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  // every stream that may still write a context buffer (a run that failed
  // after enqueueing its copies or side work) finishes before the frees
  cudaStreamSynchronize(ctx->stream);
  if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
  if (ctx->side_stream) cudaStreamSynchronize(ctx->side_stream);
  for (auto& b : ctx->buf)
    if (b.p) cudaFree(b.p);
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  for (auto e : ctx->copy_ev) cudaEventDestroy(e);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
  for (auto& pb : ctx->result_pool) cudaFree(pb.first);
  for (auto e : ctx->side_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->st_host) cudaFreeHost(ctx->st_host);
  delete ctx;
}

const char* cur_last_error(const cur_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int cur_run(cur_ctx* ctx, const void* A, int64_t m, int64_t n, int64_t lda, int dtype, double tol,
            int block_size, int sketch_size, uint64_t seed, cur_result** out) {
  return cur_run_opts(ctx, A, m, n, lda, dtype, tol, block_size, sketch_size, seed, nullptr, out);
}

int cur_run_opts(cur_ctx* ctx, const void* A, int64_t m, int64_t n, int64_t lda, int dtype,
                 double tol, int block_size, int sketch_size, uint64_t seed, const cur_opts* opts,
                 cur_result** out) {
  if (!out) return fail(ctx, CUR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctx) return CUR_EINVAL;
  if (sketch_size < 0) return fail(ctx, CUR_EINVAL, "sketch_size < 0");
  return run_device(ctx, A, m, n, lda, dtype, tol, block_size, sketch_size, seed, opts, out);
}

int cur_run_host(cur_ctx* ctx, const void* A_host, int64_t m, int64_t n, int64_t lda, int dtype,
                 double tol, int block_size, int sketch_size, uint64_t seed, const cur_opts* opts,
                 cur_result** out) {
  if (!out) return fail(ctx, CUR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctx) return CUR_EINVAL;
  if (!A_host) return fail(ctx, CUR_EINVAL, "A is NULL");
  if (m < 1 || n < 1 || lda < n) return fail(ctx, CUR_EINVAL, "bad shape");
  if (dtype != CUR_F64 && dtype != CUR_F32) return fail(ctx, CUR_EINVAL, "unknown dtype");
  size_t es = dtype == CUR_F64 ? 8 : 4;
  size_t bytes = es * (size_t)(m * n);
  CK(cudaSetDevice(ctx->device));
  TRY(ensure(ctx, B_AHOST, bytes));
  // the FP64 forms overlap the copy of A with the sketch; the precision forms
  // read A twice (column scales first): copy it whole
  const bool overlap = !opts || opts->sketch_mode == CUR_SKETCH_F64 ||
                       (opts->sketch_mode == CUR_SKETCH_F64_TC && dtype == CUR_F64);
  if (!overlap)
    CK(cudaMemcpy2DAsync(ctx->buf[B_AHOST].p, es * (size_t)n, A_host, es * (size_t)lda,
                         es * (size_t)n, (size_t)m, cudaMemcpyHostToDevice, ctx->stream));
  int st = run_device(ctx, ctx->buf[B_AHOST].p, m, n, n, dtype, tol, block_size, sketch_size, seed,
                      opts, out, overlap ? A_host : nullptr, lda);
  if (*out) {
    cur_result* r = *out;
    r->I_host.resize((size_t)r->rank);
    r->J_host.resize((size_t)r->rank);
    r->U_host.resize((size_t)(r->rank * r->rank));
    if (r->rank > 0) {
      CK(cudaMemcpyAsync(r->I_host.data(), r->I, sizeof(int64_t) * (size_t)r->rank,
                         cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaMemcpyAsync(r->J_host.data(), r->J, sizeof(int64_t) * (size_t)r->rank,
                         cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaMemcpyAsync(r->U_host.data(), r->U, sizeof(double) * (size_t)(r->rank * r->rank),
                         cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    r->host_valid = true;
  }
  return st;
}

int64_t cur_result_rank(const cur_result* r) { return r ? r->rank : 0; }
int64_t cur_result_iterations(const cur_result* r) { return r ? r->iters : 0; }
int cur_result_status(const cur_result* r) { return r ? r->status : CUR_EINVAL; }
double cur_result_err(const cur_result* r) { return r ? r->rho : NAN; }
double cur_result_sketch_norm(const cur_result* r) { return r ? r->normY : NAN; }
const int64_t* cur_result_I(const cur_result* r) { return r ? r->I : nullptr; }
const int64_t* cur_result_J(const cur_result* r) { return r ? r->J : nullptr; }
const double* cur_result_U(const cur_result* r) { return r ? r->U : nullptr; }
double cur_result_phase_ms(const cur_result* r, int phase) {
  return (r && phase >= 0 && phase < CUR_PHASE_COUNT) ? r->phase_ms[phase] : 0.0;
}
int64_t cur_result_kernel_launches(const cur_result* r) { return r ? r->launches : 0; }
const double* cur_result_rho_history(const cur_result* r) {
  return r && !r->rho_hist.empty() ? r->rho_hist.data() : nullptr;
}

int cur_result_copy_to_host(const cur_result* r, int64_t* I, int64_t* J, double* U) {
  if (!r) return CUR_EINVAL;
  size_t k = (size_t)r->rank;
  if (k == 0) return CUR_OK;
  if (r->host_valid) {
    if (I) memcpy(I, r->I_host.data(), sizeof(int64_t) * k);
    if (J) memcpy(J, r->J_host.data(), sizeof(int64_t) * k);
    if (U) memcpy(U, r->U_host.data(), sizeof(double) * k * k);
    return CUR_OK;
  }
  cur_ctx* ctx = r->ctx;
  if (I) CK(cudaMemcpyAsync(I, r->I, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, ctx->stream));
  if (J) CK(cudaMemcpyAsync(J, r->J, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, ctx->stream));
  if (U) CK(cudaMemcpyAsync(U, r->U, sizeof(double) * k * k, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CUR_OK;
}

void cur_result_free(cur_result* r) {
  if (!r) return;
  if (r->ctx) cudaStreamSynchronize(r->ctx->stream);
  if (r->block) {   // back to the context's pool (a few blocks), else freed
    if (r->ctx && r->ctx->result_pool.size() < 4)
      r->ctx->result_pool.emplace_back(r->block, r->block_bytes);
    else
      cudaFree(r->block);
  }
  delete r;
}

// ---- step entry points (cur_steps.h) ---------------------------------------

int cur_step_gaussian(cur_ctx* ctx, uint64_t seed, int64_t c, int64_t m, double* G) {
  if (!ctx) return CUR_EINVAL;
  if (c < 1 || m < 1 || !G) return fail(ctx, CUR_EINVAL, "bad arguments");
  CK(cudaSetDevice(ctx->device));
  CK(launch_gaussian(env_of(ctx), seed, c, m, G, m));
  return CUR_OK;
}

int cur_step_sketch(cur_ctx* ctx, const double* G, int64_t c, const void* A, int64_t m, int64_t n,
                    int64_t lda, int dtype, double* Y, double* sumsq_host) {
  if (!ctx) return CUR_EINVAL;
  if (!G || !A || !Y || c < 1 || m < 1 || n < 1 || lda < n || (dtype != CUR_F64 && dtype != CUR_F32))
    return fail(ctx, CUR_EINVAL, "bad arguments");
  CK(cudaSetDevice(ctx->device));
  TRY(ensure(ctx, B_STATUS, sizeof(DevStatus)));
  CK(cudaMemsetAsync(ctx->buf[B_STATUS].p, 0, sizeof(DevStatus), ctx->stream));
  TRY(sketch_f64(ctx, G, c, A, dtype == CUR_F32, m, n, lda, Y, 0, B_STEP_PARTS));
  if (sumsq_host) {
    TRY(read_status(ctx));
    *sumsq_host = ctx->st_host->scalar[0];
  }
  return CUR_OK;
}

int cur_step_gemm(cur_ctx* ctx, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                  int64_t lda, int transA, const double* B, int64_t ldb, int transB, double beta,
                  const double* C, int64_t ldc, double* D, int64_t ldd, double* sumsq_host) {
  if (!ctx) return CUR_EINVAL;
  if (M < 0 || N < 0 || K < 0 || !D || ldd < N || (beta != 0.0 && (!C || ldc < N)) ||
      (K > 0 && (!A || !B || lda < (transA ? M : K) || ldb < (transB ? K : N))))
    return fail(ctx, CUR_EINVAL, "bad arguments");
  CK(cudaSetDevice(ctx->device));
  TRY(ensure(ctx, B_STATUS, sizeof(DevStatus)));
  CK(cudaMemsetAsync(ctx->buf[B_STATUS].p, 0, sizeof(DevStatus), ctx->stream));
  if (M == 0 || N == 0) {
    if (sumsq_host) *sumsq_host = 0.0;
    return CUR_OK;
  }
  GemmArgs g = gargs(M, N, K, alpha, A, lda, transA != 0, B, ldb, transB != 0, false, beta,
                     beta != 0.0 ? C : nullptr, beta != 0.0 ? ldc : 0, D, ldd);
  int64_t np = 0;
  if (sumsq_host) {
    np = gemm_num_sumsq_parts(g);
    TRY(ensure(ctx, B_STEP_PARTS, sizeof(double) * (size_t)(np > 0 ? np : 1)));
    g.sumsq_part = bp<double>(ctx, B_STEP_PARTS);
  }
  TRY(gemm(ctx, g));
  if (sumsq_host) {
    TRY(sum_parts(ctx, g.sumsq_part, np, &dstat(ctx)->scalar[0]));
    TRY(read_status(ctx));
    *sumsq_host = ctx->st_host->scalar[0];
  }
  return CUR_OK;
}

int cur_step_resid_tc(cur_ctx* ctx, const double* P, int64_t ldp, const double* Q, int64_t ldq,
                      int64_t M, int64_t N, int64_t K, int planes, double* D, int64_t ldd) {
  if (!ctx) return CUR_EINVAL;
  if ((planes != 2 && planes != 3) || M < 0 || N < 1 || N > 128 || K < 0 || ldp < K || ldq < K ||
      ldd < M || !D || (K > 0 && (!P || !Q)))
    return fail(ctx, CUR_EINVAL, "bad arguments");
  CK(cudaSetDevice(ctx->device));
  TRY(ensure(ctx, B_STATUS, sizeof(DevStatus)));
  CK(cudaMemsetAsync(ctx->buf[B_STATUS].p, 0, sizeof(DevStatus), ctx->stream));
  if (M == 0 || K == 0) return CUR_OK;
  LaunchEnv env = env_of(ctx);
  const int64_t kp = resid_plane_pitch(K);
  TRY(ensure(ctx, B_STEP_RP, 2 * (size_t)planes * (size_t)(M * kp)));
  TRY(ensure(ctx, B_STEP_RQ, 2 * (size_t)planes * (size_t)(N * kp)));
  __nv_bfloat16* pp[3];
  __nv_bfloat16* qp[3];
  for (int p = 0; p < 3; ++p) {
    pp[p] = bp<__nv_bfloat16>(ctx, B_STEP_RP) + (size_t)(p < planes ? p : 0) * (size_t)(M * kp);
    qp[p] = bp<__nv_bfloat16>(ctx, B_STEP_RQ) + (size_t)(p < planes ? p : 0) * (size_t)(N * kp);
  }
  CK(launch_split_planes(env, P, 1, ldp, K, M, pp, planes, kp, 0));
  CK(launch_split_planes(env, Q, 1, ldq, K, N, qp, planes, kp, 0));
  CK(launch_resid_tc(env, planes, pp, kp, M, qp, kp, (int)N, K, D, ldd, &dstat(ctx)->err));
  ctx->launches += 3;
  return read_status(ctx);
}

int cur_step_gather(cur_ctx* ctx, const double* X, int64_t ldx, int trans, const int64_t* ridx,
                    const int64_t* cidx, int64_t rows, int64_t cols, int64_t rlim, int64_t clim,
                    double* out, int64_t ldo) {
  if (!ctx) return CUR_EINVAL;
  if (rows < 0 || cols < 0 || rlim < 0 || clim < 0 || (rows > 0 && cols > 0 && (!X || !out)) ||
      ldo < cols || ldx < (trans ? rlim : clim))
    return fail(ctx, CUR_EINVAL, "bad arguments");
  CK(cudaSetDevice(ctx->device));
  return gather(ctx, X, false, ldx, trans != 0, ridx, cidx, rows, cols, rlim, clim, out, ldo);
}

int cur_step_sketch_q(cur_ctx* ctx, const double* G, int64_t c, const float* A, int64_t m,
                      int64_t n, int64_t lda, int digits, double* Y, double* sumsq_host) {
  if (!ctx) return CUR_EINVAL;
  if (!G || !A || !Y || c < 1 || m < 1 || n < 1 || lda < n)
    return fail(ctx, CUR_EINVAL, "bad arguments");
  TRY(check_precision_form(ctx, digits, A, lda, CUR_F32, c));
  CK(cudaSetDevice(ctx->device));
  TRY(ensure(ctx, B_STATUS, sizeof(DevStatus)));
  CK(cudaMemsetAsync(ctx->buf[B_STATUS].p, 0, sizeof(DevStatus), ctx->stream));
  TRY(sketch_q(ctx, digits, G, c, A, m, n, lda, Y, 0, B_STEP_PARTS, B_STEP_TC));
  TRY(read_status(ctx));
  if (sumsq_host) *sumsq_host = ctx->st_host->scalar[0];
  return CUR_OK;
}

int cur_step_sketch_fx(cur_ctx* ctx, const double* G, int64_t c, const double* A, int64_t m,
                       int64_t n, int64_t lda, double* Y, double* sumsq_host) {
  if (!ctx) return CUR_EINVAL;
  if (!G || !A || !Y || c < 1 || m < 1 || n < 1 || lda < n)
    return fail(ctx, CUR_EINVAL, "bad arguments");
  TRY(check_fx_form(ctx, A, lda, CUR_F64));
  CK(cudaSetDevice(ctx->device));
  TRY(ensure(ctx, B_STATUS, sizeof(DevStatus)));
  CK(cudaMemsetAsync(ctx->buf[B_STATUS].p, 0, sizeof(DevStatus), ctx->stream));
  TRY(sketch_fx(ctx, G, c, A, m, n, lda, Y, 0, B_STEP_PARTS, B_STEP_FX));
  TRY(read_status(ctx));
  if (sumsq_host) *sumsq_host = ctx->st_host->scalar[0];
  return CUR_OK;
}

int cur_test_wait_timeout(cur_ctx* ctx, int which, int nblocks, double budget_ms) {
  if (!ctx) return CUR_EINVAL;
  if ((which != 0 && which != 1) || nblocks < 1 || nblocks > ctx->num_sms || !(budget_ms > 0.0) ||
      budget_ms > 5000.0)
    return fail(ctx, CUR_EINVAL, "bad arguments");
  CK(cudaSetDevice(ctx->device));
  TRY(ensure(ctx, B_STATUS, sizeof(DevStatus)));
  TRY(ensure(ctx, B_STEP_PARTS, sizeof(GridBar) + 256));
  CK(cudaMemsetAsync(ctx->buf[B_STATUS].p, 0, sizeof(DevStatus), ctx->stream));
  int khz = 0;
  CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device));
  const long long budget = (long long)(budget_ms * (double)(khz > 0 ? khz : 2000000));
  CK(launch_timeout_check(env_of(ctx), which, nblocks, budget, bp<GridBar>(ctx, B_STEP_PARTS),
                          dstat(ctx)));
  return read_status(ctx);
}

int cur_step_lupp(cur_ctx* ctx, const double* X, int64_t ldx, int64_t nr, int64_t ncand,
                  int64_t steps, uint8_t* mask, int64_t* piv) {
  if (!ctx) return CUR_EINVAL;
  if (!X || !mask || !piv || nr < 1 || ncand < 1 || ldx < ncand || steps < 0 || steps > nr ||
      steps > ncand)
    return fail(ctx, CUR_EINVAL, "bad arguments");
  CK(cudaSetDevice(ctx->device));
  TRY(ensure(ctx, B_STATUS, sizeof(DevStatus)));
  CK(cudaMemsetAsync(ctx->buf[B_STATUS].p, 0, sizeof(DevStatus), ctx->stream));
  TRY(lupp_call(ctx, B_STEP_LUPP, X, ldx, nr, ncand, steps, mask, piv));
  return read_status(ctx);
}

int cur_step_pinv(cur_ctx* ctx, const double* M, int64_t p, int64_t q, int64_t ldm, double thr,
                  double* X, int64_t* rank_host) {
  if (!ctx) return CUR_EINVAL;
  if (!M || !X || p < 1 || q < 1 || ldm < q) return fail(ctx, CUR_EINVAL, "bad arguments");
  if (p > kMaxCoreRank) return fail(ctx, CUR_EINVAL, "p > 16384 is not supported by the core solve");
  CK(cudaSetDevice(ctx->device));
  TRY(ensure(ctx, B_STATUS, sizeof(DevStatus)));
  CK(cudaMemsetAsync(ctx->buf[B_STATUS].p, 0, sizeof(DevStatus), ctx->stream));
  LaunchEnv env = env_of(ctx);
  const int T = team_core(env, p, q) ? core_qr_grid(env, p) : 0;
  if (T > 0) {  // the same kernels as the core of cur_run at this size
    const size_t wb = core_qr_work_bytes(p, q, T);
    TRY(ensure(ctx, B_TEAMCORE, wb + 256));
    double* W = bp<double>(ctx, B_TEAMCORE);
    int64_t* rk = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(W) + wb);
    // column-major M: W[col * p + i] = M(i, col)
    TRY(gather(ctx, M, false, ldm, true, nullptr, nullptr, q, p, q, p, W, p));
    CK(launch_core_qr(env, W, p, q, thr < 0 ? -1.0 : thr, X, p, W, T, dstat(ctx), rk));
    ctx->launches += 1;
    TRY(read_status(ctx));
    if (rank_host) CK(cudaMemcpy(rank_host, rk, sizeof(int64_t), cudaMemcpyDeviceToHost));
    return CUR_OK;
  }
  TRY(pinv_call(ctx, B_STEP_QR, M, p, q, ldm, thr < 0 ? 0 : 1, thr, nullptr, X, p));
  TRY(read_status(ctx));
  if (rank_host) {
    QrcpWork w;
    qrcp_carve(ctx->buf[B_STEP_QR].p, p, q, qrcp_grid(env, p, q), &w);
    CK(cudaMemcpy(rank_host, w.rank, sizeof(int64_t), cudaMemcpyDeviceToHost));
  }
  return CUR_OK;
}

}  // extern "C"
