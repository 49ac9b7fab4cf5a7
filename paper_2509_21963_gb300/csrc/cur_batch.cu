// cur_batch.cu -- C ABI of the batched engine (include/cur_batch.h): job
// validation, output and scratch sizing, the largest-work-first queue order,
// graph capture of the persistent launch, and the team-size autotuner.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/cur.h"
#include "../../include/cur_batch.h"
#include "batch.cuh"
#include "ctx.cuh"

using namespace cur;

struct cur_batch {
  cur_ctx* ctx = nullptr;
  bool a_f32 = false;
  int64_t njobs = 0;
  std::vector<BatchJobDev> jobs;
  std::vector<int> order;
  BatchDims dims{};
  // device memory owned by the batch
  void* outputs = nullptr;   // jobs, order, out records, I, J, U, rho history, queue, status
  size_t outputs_bytes = 0;
  char* team_scratch = nullptr;
  size_t team_alloc = 0;
  char* cta_scratch = nullptr;
  size_t cta_alloc = 0;
  BatchParams P{};
  BatchOutDev* out_host = nullptr;  // pinned
  // schedule
  int threads = 256;
  int team = 1;
  int tile_n = 8;            // outputs per thread and pass of the residual products (4 or 8)
  int team_big = 0;          // 0: one team class
  int nbig = 0;
  int64_t big_cut = 0;
  int grid = 0;
  std::vector<double> work;  // estimated work per job, in queue order
  cudaStream_t bstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_tried = false;
  bool launched = false;
  bool have_results = false;
};

namespace {

int bfail(cur_ctx* ctx, int code, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  return ctx_fail_v(ctx, code, msg);
}

#define BCK(expr)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      cudaGetLastError();                                                                   \
      return bfail(ctx, CUR_ECUDA, "%s failed: %s (%d)", #expr, cudaGetErrorString(e_),     \
                   (int)e_);                                                                \
    }                                                                                       \
  } while (0)

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

LaunchEnv benv(cur_batch* b) { return LaunchEnv{b->bstream, b->ctx->num_sms, b->ctx->device}; }

int reserve(cur_ctx* ctx, size_t bytes) {
  if (ctx->budget && ctx->held + bytes > ctx->budget)
    return bfail(ctx, CUR_EBUDGET, "batch memory of %zu bytes exceeds the HBM budget of %zu bytes",
                 ctx->held + bytes, ctx->budget);
  ctx->held += bytes;
  return CUR_OK;
}

void release(cur_ctx* ctx, size_t bytes) { ctx->held -= std::min(ctx->held, bytes); }

int dev_alloc(cur_ctx* ctx, void** p, size_t bytes) {
  int s = reserve(ctx, bytes);
  if (s != CUR_OK) return s;
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release(ctx, bytes);
    *p = nullptr;
    return bfail(ctx, CUR_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  return CUR_OK;
}

void drop_graph(cur_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->graph_tried = false;
}

// (Re)size the team and CTA scratch for a schedule: nbig teams of team_big
// CTAs serving the queue positions [0, big_cut) first (nbig = 0: none), and
// as many teams of `team` CTAs as the remaining co-resident CTAs allow.
int plan_schedule(cur_batch* b, int team, int team_big = 0, int nbig = 0, int64_t big_cut = 0) {
  cur_ctx* ctx = b->ctx;
  LaunchEnv env = benv(b);
  const size_t panel = batch_panel_bytes(b->dims.R);
  const int max_ctas = batch_max_ctas(env, b->threads, b->a_f32, panel);
  if (max_ctas < 1) return bfail(ctx, CUR_ECUDA, "the batch kernel cannot be resident on this GPU");
  if (team < 1 || team > 32 || team > max_ctas)
    return bfail(ctx, CUR_EINVAL, "team size %d outside 1..%d", team, std::min(32, max_ctas));
  if (nbig < 0 || (nbig > 0 && (team_big < 1 || team_big > 32 ||
                                (int64_t)nbig * team_big + team > max_ctas)))
    return bfail(ctx, CUR_EINVAL, "%d big teams of %d CTAs leave no room for a team of %d (%d CTAs)",
                 nbig, team_big, team, max_ctas);
  if (nbig == 0) { team_big = 0; big_cut = 0; }
  big_cut = std::max<int64_t>(0, std::min<int64_t>(big_cut, b->njobs));
  const int bigctas = nbig * team_big;
  const int teams = nbig + (max_ctas - bigctas) / team;
  const int grid = bigctas + ((max_ctas - bigctas) / team) * team;
  BatchLayout L = batch_layout_dev(b->dims, team);
  size_t tb = al256(L.team_bytes), cb = al256(L.cta_bytes);
  if (nbig > 0) {
    BatchLayout Lb = batch_layout_dev(b->dims, team_big);
    tb = std::max(tb, al256(Lb.team_bytes));
    cb = std::max(cb, al256(Lb.cta_bytes));
  }
  const size_t need_t = tb * (size_t)teams, need_c = cb * (size_t)grid;
  BCK(cudaStreamSynchronize(b->bstream));
  if (need_t > b->team_alloc) {
    if (b->team_scratch) { cudaFree(b->team_scratch); release(ctx, b->team_alloc); }
    b->team_scratch = nullptr;
    b->team_alloc = 0;
    int s = dev_alloc(ctx, (void**)&b->team_scratch, need_t);
    if (s != CUR_OK) return s;
    b->team_alloc = need_t;
  }
  if (need_c > b->cta_alloc) {
    if (b->cta_scratch) { cudaFree(b->cta_scratch); release(ctx, b->cta_alloc); }
    b->cta_scratch = nullptr;
    b->cta_alloc = 0;
    int s = dev_alloc(ctx, (void**)&b->cta_scratch, need_c);
    if (s != CUR_OK) return s;
    b->cta_alloc = need_c;
  }
  // barriers start at zero; every team's header is re-zeroed here and stays
  // consistent across launches (a completed barrier leaves its counter at a
  // multiple of the team size)
  BCK(cudaMemsetAsync(b->team_scratch, 0, need_t, b->bstream));
  BCK(cudaStreamSynchronize(b->bstream));
  b->team = team;
  b->team_big = team_big;
  b->nbig = nbig;
  b->big_cut = big_cut;
  b->grid = grid;
  b->P.team = team;
  b->P.tile_n = b->tile_n;
  b->P.team_big = team_big;
  b->P.nbig = nbig;
  b->P.big_cut = big_cut;
  b->P.team_scratch = b->team_scratch;
  b->P.team_bytes = tb;
  b->P.cta_scratch = b->cta_scratch;
  b->P.cta_bytes = cb;
  b->P.panel_bytes = panel;
  drop_graph(b);
  return CUR_OK;
}

// The launch sequence: queue head and status to zero, the kernel, the
// per-job records to pinned host memory.
cudaError_t enqueue(cur_batch* b) {
  cudaError_t e = cudaMemsetAsync(b->P.next, 0, 2 * sizeof(unsigned long long), b->bstream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->P.st, 0, sizeof(DevStatus), b->bstream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->P.prof, 0, sizeof(unsigned long long) * kBatchPhases, b->bstream);
  if (e == cudaSuccess) e = launch_batch(benv(b), b->P, b->grid, b->threads, b->a_f32);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->out_host, b->P.out, sizeof(BatchOutDev) * (size_t)b->njobs,
                        cudaMemcpyDeviceToHost, b->bstream);
  return e;
}

void try_capture(cur_batch* b) {
  b->graph_tried = true;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->bstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaError_t e = enqueue(b);
  cudaError_t e2 = cudaStreamEndCapture(b->bstream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return;
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    cudaGetLastError();
    ex = nullptr;
  }
  cudaGraphDestroy(g);
  b->gexec = ex;
}

double work_estimate(const BatchJobDev& j) {
  const double r = (double)j.rmax;
  return r * r * ((double)j.m + (double)j.n + 4.3 * r) + 2.0 * j.c * (double)j.m * (double)j.n;
}

}  // namespace

extern "C" {

int cur_batch_create(cur_ctx* ctx, const cur_batch_job* jobs, int64_t njobs, int dtype,
                     cur_batch** out) {
  if (!out) return bfail(ctx, CUR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctx) return CUR_EINVAL;
  if (!jobs || njobs < 1) return bfail(ctx, CUR_EINVAL, "empty batch");
  if (njobs > (int64_t)1 << 30) return bfail(ctx, CUR_EINVAL, "too many jobs");
  if (dtype != CUR_F64 && dtype != CUR_F32) return bfail(ctx, CUR_EINVAL, "dtype %d", dtype);
  cur_batch* b = new cur_batch();
  b->ctx = ctx;
  b->a_f32 = dtype == CUR_F32;
  b->njobs = njobs;
  b->jobs.resize((size_t)njobs);
  int64_t off_ij = 0, off_u = 0, off_h = 0;
  BatchDims d{1, 1, 1, 1, 1};
  for (int64_t k = 0; k < njobs; ++k) {
    const cur_batch_job& s = jobs[k];
    BatchJobDev& j = b->jobs[(size_t)k];
    int c = s.sketch_size == 0 ? (int)std::floor(1.1 * s.block_size) : s.sketch_size;
    const char* why = nullptr;
    if (!s.A) why = "A is NULL";
    else if (s.m < 1 || s.n < 1) why = "m and n must be >= 1";
    else if (s.lda < s.n) why = "lda < n";
    else if (!(s.tol > 0.0)) why = "tol must be > 0";
    else if (s.block_size < 1 || s.block_size > kBatchMaxB) why = "block_size outside 1..64";
    else if (c < s.block_size || c > kBatchMaxC) why = "sketch_size outside b..128";
    if (why) {
      delete b;
      return bfail(ctx, CUR_EINVAL, "job %lld: %s", (long long)k, why);
    }
    j.A = s.A;
    j.m = s.m;
    j.n = s.n;
    j.lda = s.lda;
    j.tol = s.tol;
    j.b = s.block_size;
    j.c = c;
    j.seed = s.seed;
    const int64_t mn = std::min(s.m, s.n);
    j.rmax = (s.max_rank <= 0 || s.max_rank > mn) ? mn : s.max_rank;
    j.off_ij = off_ij;
    j.off_j = off_ij;
    j.ws = nullptr;
    j.off_u = off_u;
    j.off_hist = off_h;
    off_ij += j.rmax;
    off_u += j.rmax * j.rmax;
    off_h += (j.rmax + j.b - 1) / j.b;
    d.M = std::max(d.M, j.m);
    d.N = std::max(d.N, j.n);
    d.C = std::max(d.C, (int64_t)j.c);
    d.B = std::max(d.B, (int64_t)j.b);
    d.R = std::max(d.R, j.rmax);
  }
  b->dims = d;
  b->order.resize((size_t)njobs);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::vector<double> w((size_t)njobs);
  for (int64_t k = 0; k < njobs; ++k) w[(size_t)k] = work_estimate(b->jobs[(size_t)k]);
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int x, int y) { return w[(size_t)x] > w[(size_t)y]; });
  b->work.resize((size_t)njobs);
  for (int64_t k = 0; k < njobs; ++k) b->work[(size_t)k] = w[(size_t)b->order[(size_t)k]];

  // one allocation for everything the size of which depends only on the jobs
  size_t o = 0;
  auto put = [&](size_t bytes) { size_t at = o; o += al256(bytes); return at; };
  const size_t o_jobs = put(sizeof(BatchJobDev) * (size_t)njobs);
  const size_t o_order = put(sizeof(int) * (size_t)njobs);
  const size_t o_out = put(sizeof(BatchOutDev) * (size_t)njobs);
  const size_t o_I = put(8 * (size_t)off_ij);
  const size_t o_J = put(8 * (size_t)off_ij);
  const size_t o_U = put(8 * (size_t)off_u);
  const size_t o_h = put(8 * (size_t)off_h);
  const size_t o_next = put(2 * sizeof(unsigned long long));   // big and small queue heads
  const size_t o_st = put(sizeof(DevStatus));
  const size_t o_prof = put(sizeof(unsigned long long) * kBatchPhases);
  b->outputs_bytes = o;
  int s = CUR_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) { cudaGetLastError(); delete b; return bfail(ctx, CUR_ECUDA, "cudaSetDevice"); }
  s = dev_alloc(ctx, &b->outputs, o);
  if (s != CUR_OK) { delete b; return s; }
  if (cudaStreamCreateWithFlags(&b->bstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost((void**)&b->out_host, sizeof(BatchOutDev) * (size_t)njobs) != cudaSuccess) {
    cudaGetLastError();
    cur_batch_free(b);
    return bfail(ctx, CUR_ENOMEM, "stream, event or pinned buffer creation failed");
  }
  char* base = static_cast<char*>(b->outputs);
  b->P.jobs = reinterpret_cast<BatchJobDev*>(base + o_jobs);
  b->P.order = reinterpret_cast<int*>(base + o_order);
  b->P.njobs = njobs;
  b->P.out = reinterpret_cast<BatchOutDev*>(base + o_out);
  b->P.Iout = reinterpret_cast<int64_t*>(base + o_I);
  b->P.Jout = reinterpret_cast<int64_t*>(base + o_J);
  b->P.Uout = reinterpret_cast<double*>(base + o_U);
  b->P.rho_hist = reinterpret_cast<double*>(base + o_h);
  b->P.hist_len = off_h;
  b->P.next = reinterpret_cast<unsigned long long*>(base + o_next);
  b->P.next_small = b->P.next + 1;
  b->P.st = reinterpret_cast<DevStatus*>(base + o_st);
  b->P.prof = reinterpret_cast<unsigned long long*>(base + o_prof);
  b->P.dims = d;
  cudaError_t e = cudaMemcpyAsync((void*)b->P.jobs, b->jobs.data(),
                                  sizeof(BatchJobDev) * (size_t)njobs, cudaMemcpyHostToDevice,
                                  b->bstream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void*)b->P.order, b->order.data(), sizeof(int) * (size_t)njobs,
                        cudaMemcpyHostToDevice, b->bstream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->bstream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cur_batch_free(b);
    return bfail(ctx, CUR_ECUDA, "batch upload failed: %s", cudaGetErrorString(e));
  }
  // default schedule: a team of 8 CTAs when the largest job is big enough to
  // use them, otherwise one CTA per job
  const double wmax = w[(size_t)b->order[0]];
  s = plan_schedule(b, wmax > 5e9 ? 8 : 1);
  if (s != CUR_OK) { cur_batch_free(b); return s; }
  *out = b;
  return CUR_OK;
}

void cur_batch_free(cur_batch* b) {
  if (!b) return;
  cur_ctx* ctx = b->ctx;
  if (b->bstream) cudaStreamSynchronize(b->bstream);
  drop_graph(b);
  if (b->outputs) { cudaFree(b->outputs); release(ctx, b->outputs_bytes); }
  if (b->team_scratch) { cudaFree(b->team_scratch); release(ctx, b->team_alloc); }
  if (b->cta_scratch) { cudaFree(b->cta_scratch); release(ctx, b->cta_alloc); }
  if (b->out_host) cudaFreeHost(b->out_host);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->bstream) cudaStreamDestroy(b->bstream);
  cudaGetLastError();
  delete b;
}

int cur_batch_set_team(cur_batch* b, int team) {
  if (!b) return CUR_EINVAL;
  if (team == 0) return CUR_OK;
  return plan_schedule(b, team);
}

int cur_batch_set_classes(cur_batch* b, int team, int team_big, int nbig, int64_t big_cut) {
  if (!b) return CUR_EINVAL;
  return plan_schedule(b, team, team_big, nbig, big_cut);
}

int cur_batch_set_tile(cur_batch* b, int tile_n) {
  if (!b) return CUR_EINVAL;
  if (tile_n != 4 && tile_n != 8) return bfail(b->ctx, CUR_EINVAL, "tile_n must be 4 or 8");
  if (tile_n != b->tile_n) {
    b->tile_n = tile_n;
    b->P.tile_n = tile_n;
    drop_graph(b);
  }
  return CUR_OK;
}

int cur_batch_get_tile(const cur_batch* b, int* tile_n) {
  if (!b || !tile_n) return CUR_EINVAL;
  *tile_n = b->tile_n;
  return CUR_OK;
}

int cur_batch_get_classes(const cur_batch* b, int* team_big, int* nbig, int64_t* big_cut) {
  if (!b) return CUR_EINVAL;
  if (team_big) *team_big = b->team_big;
  if (nbig) *nbig = b->nbig;
  if (big_cut) *big_cut = b->big_cut;
  return CUR_OK;
}

int cur_batch_get_schedule(const cur_batch* b, int* team, int* grid, int* teams, int* graph) {
  if (!b) return CUR_EINVAL;
  if (team) *team = b->team;
  if (grid) *grid = b->grid;
  if (teams) *teams = b->nbig + (b->grid - b->nbig * b->team_big) / b->team;
  if (graph) *graph = b->gexec ? 1 : 0;
  return CUR_OK;
}

int cur_batch_launch(cur_batch* b) {
  if (!b) return CUR_EINVAL;
  cur_ctx* ctx = b->ctx;
  BCK(cudaSetDevice(ctx->device));
  BCK(cudaEventRecord(b->ev_in, ctx->stream));
  BCK(cudaStreamWaitEvent(b->bstream, b->ev_in, 0));
  if (!b->graph_tried) try_capture(b);
  if (b->gexec) {
    BCK(cudaGraphLaunch(b->gexec, b->bstream));
  } else {
    BCK(enqueue(b));
  }
  BCK(cudaEventRecord(b->ev_out, b->bstream));
  BCK(cudaStreamWaitEvent(ctx->stream, b->ev_out, 0));
  b->launched = true;
  b->have_results = false;
  ctx->launches += 1;
  return CUR_OK;
}

int cur_batch_wait(cur_batch* b) {
  if (!b) return CUR_EINVAL;
  cur_ctx* ctx = b->ctx;
  if (!b->launched) return bfail(ctx, CUR_EINVAL, "no launch to wait for");
  BCK(cudaStreamSynchronize(b->bstream));
  DevStatus st;
  BCK(cudaMemcpy(&st, b->P.st, sizeof(st), cudaMemcpyDeviceToHost));
  b->launched = false;
  if (st.err != 0) {  // a team may have stopped inside a barrier: reset the headers
    cudaMemsetAsync(b->team_scratch, 0, b->team_alloc, b->bstream);
    cudaStreamSynchronize(b->bstream);
    cudaGetLastError();
  }
  if (st.err == kDevTimeout)
    return bfail(ctx, CUR_ETIMEOUT, "a team barrier of the batch kernel exceeded its cycle budget");
  if (st.err != 0) return bfail(ctx, CUR_ECUDA, "batch kernel device status %d", st.err);
  b->have_results = true;
  return CUR_OK;
}

int cur_batch_run(cur_batch* b) {
  int s = cur_batch_launch(b);
  if (s != CUR_OK) return s;
  return cur_batch_wait(b);
}

// Timed launches per candidate team size in cur_batch_tune (the fastest counts).
constexpr int kTuneReps = 2;

int cur_batch_tune(cur_batch* b, const int* candidates, int ncand, int* best_team,
                   double* best_ms) {
  if (!b) return CUR_EINVAL;
  cur_ctx* ctx = b->ctx;
  static const int kDefault[] = {1, 2, 4, 8, 16};
  if (!candidates) { candidates = kDefault; ncand = 5; }
  if (ncand < 1) return bfail(ctx, CUR_EINVAL, "no candidate team sizes");
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  const int max_ctas = batch_max_ctas(benv(b), b->threads, b->a_f32, batch_panel_bytes(b->dims.R));
  // Candidate schedules: one class of each candidate size, then, on top of the
  // best of those, big-team classes (team_big in {8, 16} above it, 1 or 2 big
  // teams) whose queue share is the big teams' share of the CTAs, counted in
  // estimated work from the largest job down.
  struct Cand { int team, team_big, nbig; int64_t cut; int tile; };
  std::vector<Cand> cands;
  for (int k = 0; k < ncand; ++k)
    if (candidates[k] >= 1 && candidates[k] <= 32 && candidates[k] <= max_ctas)
      cands.push_back({candidates[k], 0, 0, 0, 8});
  const size_t nsingle = cands.size();
  size_t tile_from = (size_t)-1;   // index after the last schedule candidate (set below)
  double wsum = 0.0;
  for (double x : b->work) wsum += x;
  int best = -1;
  float best_t = 0.f;
  int s = CUR_OK;
  for (size_t k = 0; k < cands.size() && s == CUR_OK; ++k) {
    const Cand cd = cands[k];
    b->tile_n = cd.tile;
    s = plan_schedule(b, cd.team, cd.team_big, cd.nbig, cd.cut);
    if (s != CUR_OK) break;
    // capture the candidate's graph before timing (host-side work that would
    // otherwise leave the GPU idle inside the timed interval), then keep the
    // fastest of kTuneReps graph launches
    try_capture(b);
    float cand = -1.f;
    for (int rep = 0; rep < kTuneReps && s == CUR_OK; ++rep) {
      if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) { s = CUR_ECUDA; break; }
      s = cur_batch_launch(b);
      if (s != CUR_OK) break;
      if (cudaEventRecord(e1, ctx->stream) != cudaSuccess) { s = CUR_ECUDA; break; }
      s = cur_batch_wait(b);
      if (s != CUR_OK) break;
      float ms = 0.f;
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      if (cand < 0.f || ms < cand) cand = ms;
    }
    if (s != CUR_OK) break;
    if (best < 0 || cand < best_t) { best = (int)k; best_t = cand; }
    if (k + 1 == nsingle && best >= 0) {   // the big-team classes
      const int ts = cands[(size_t)best].team;
      for (int tbig : {8, 16})
        for (int nb : {1, 2}) {
          if (b->njobs < 2 || tbig <= ts || nb * tbig + ts > max_ctas) continue;
          const double share = wsum * (double)(nb * tbig) / (double)max_ctas;
          int64_t cut = 0;
          double acc = 0.0;
          while (cut < b->njobs && (cut == 0 || acc < share)) acc += b->work[(size_t)cut++];
          if (cut >= b->njobs) cut = b->njobs - 1;
          cands.push_back({ts, tbig, nb, cut, 8});
        }
      tile_from = cands.size();
    }
    if (k + 1 == tile_from && best >= 0) {   // the other product tile on the best schedule
      Cand c4 = cands[(size_t)best];
      c4.tile = 4;
      cands.push_back(c4);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != CUR_OK) return s;
  if (best < 0) return bfail(ctx, CUR_EINVAL, "no candidate team size fits this GPU");
  const Cand bc = cands[(size_t)best];
  if (best + 1 != (int)cands.size()) {
    b->tile_n = bc.tile;
    s = plan_schedule(b, bc.team, bc.team_big, bc.nbig, bc.cut);
    if (s != CUR_OK) return s;
    s = cur_batch_run(b);  // results of the chosen schedule
    if (s != CUR_OK) return s;
  }
  if (best_team) *best_team = bc.team;
  if (best_ms) *best_ms = best_t;
  return CUR_OK;
}

int cur_batch_phase_cycles(const cur_batch* b, double* cycles, int nphase) {
  if (!b || !cycles || nphase < 1) return CUR_EINVAL;
  cur_ctx* ctx = b->ctx;
  if (!b->have_results) return ctx_fail_v(ctx, CUR_EINVAL, "no completed run");
  unsigned long long v[kBatchPhases];
  BCK(cudaMemcpy(v, b->P.prof, sizeof(v), cudaMemcpyDeviceToHost));
  for (int k = 0; k < nphase && k < kBatchPhases; ++k) cycles[k] = (double)v[k];
  return CUR_OK;
}

int cur_batch_job_cycles(const cur_batch* b, int64_t job, int64_t* cycles) {
  if (!b || job < 0 || job >= b->njobs || !cycles) return CUR_EINVAL;
  if (!b->have_results) return ctx_fail_v(b->ctx, CUR_EINVAL, "no completed run");
  *cycles = b->out_host[job].cycles;
  return CUR_OK;
}

int cur_batch_job_result(const cur_batch* b, int64_t job, int64_t* rank, int64_t* iters,
                         double* rho, int* status) {
  if (!b || job < 0 || job >= b->njobs) return CUR_EINVAL;
  if (!b->have_results) return ctx_fail_v(b->ctx, CUR_EINVAL, "no completed run");
  const BatchOutDev& o = b->out_host[job];
  if (rank) *rank = o.rank;
  if (iters) *iters = o.iters;
  if (rho) *rho = o.rho;
  if (status) *status = o.status;
  return CUR_OK;
}

const int64_t* cur_batch_I(const cur_batch* b, int64_t job) {
  if (!b || job < 0 || job >= b->njobs) return nullptr;
  return b->P.Iout + b->jobs[(size_t)job].off_ij;
}

const int64_t* cur_batch_J(const cur_batch* b, int64_t job) {
  if (!b || job < 0 || job >= b->njobs) return nullptr;
  return b->P.Jout + b->jobs[(size_t)job].off_j;
}

const double* cur_batch_U(const cur_batch* b, int64_t job) {
  if (!b || job < 0 || job >= b->njobs) return nullptr;
  return b->P.Uout + b->jobs[(size_t)job].off_u;
}

const double* cur_batch_rho_history(const cur_batch* b, int64_t job) {
  if (!b || job < 0 || job >= b->njobs) return nullptr;
  return b->P.rho_hist + b->jobs[(size_t)job].off_hist;
}

int cur_batch_copy_job(const cur_batch* b, int64_t job, int64_t* I, int64_t* J, double* U,
                       double* rho_history) {
  if (!b || job < 0 || job >= b->njobs) return CUR_EINVAL;
  cur_ctx* ctx = b->ctx;
  if (!b->have_results) return ctx_fail_v(ctx, CUR_EINVAL, "no completed run");
  const int64_t r = b->out_host[job].rank;
  const BatchJobDev& j = b->jobs[(size_t)job];
  if (r > 0) {
    if (I) BCK(cudaMemcpy(I, b->P.Iout + j.off_ij, 8 * (size_t)r, cudaMemcpyDeviceToHost));
    if (J) BCK(cudaMemcpy(J, b->P.Jout + j.off_j, 8 * (size_t)r, cudaMemcpyDeviceToHost));
    if (U) BCK(cudaMemcpy(U, b->P.Uout + j.off_u, 8 * (size_t)(r * r), cudaMemcpyDeviceToHost));
  }
  const int64_t it = b->out_host[job].iters;
  if (rho_history && it > 0)
    BCK(cudaMemcpy(rho_history, b->P.rho_hist + j.off_hist, 8 * (size_t)it,
                   cudaMemcpyDeviceToHost));
  return CUR_OK;
}

}  // extern "C"
