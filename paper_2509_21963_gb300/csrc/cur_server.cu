// cur_server.cu -- serving form (include/cur_server.h): request FIFO,
// admission by HBM footprint into a first-fit arena, waves of admitted
// requests launched as cluster-per-request kernels on several streams, a
// scheduler thread that retires waves and returns their scratch at once.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/cur.h"
#include "../../include/cur_batch.h"
#include "../../include/cur_server.h"
#include "arena.h"
#include "batch.cuh"
#include "ctx.cuh"

using namespace cur;

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

enum ReqState { kPending = 0, kAdmitted = 1, kRunning = 2, kDone = 3 };

struct Req {
  uint64_t id = 0;
  cur_batch_job job{};
  int a_on_host = 0;
  int c = 0;
  int64_t rmax = 0;
  size_t scratch_bytes = 0, out_bytes = 0, a_bytes = 0;
  size_t scratch_off = 0, out_off = 0, a_off = 0;
  size_t off_I = 0, off_J = 0, off_U = 0, off_h = 0;  // byte offsets in the arena
  BatchOutDev out{};
  double t_submit = 0, t_admit = 0, t_done = 0;
  int state = kPending;
  bool big = false;  // runs alone on the whole GPU through the single-matrix path
  std::string err;   // why a large request failed (its lane context's message)
};

struct Wave {
  int stream = 0;
  cudaEvent_t ev = nullptr;
  std::vector<Req*> reqs;
  size_t desc_off = 0, desc_bytes = 0;
};

// One worker for large requests: a private context (own stream) and thread.
struct BigLane {
  cur_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  std::thread th;
  std::condition_variable cv;
  Req* job = nullptr;
  bool quit = false;
};

constexpr int kMaxWave = 2048;
constexpr int kBackfill = 16;
constexpr size_t kDescPool = 64ull << 20;

}  // namespace

struct cur_server {
  cur_ctx* ctx = nullptr;
  std::vector<BigLane*> lanes;       // workers of the large-request path
  int64_t big_elements = 0;          // m * n at or above which a request is large
  bool a_f32 = true;
  int team = 4;
  std::vector<cudaStream_t> streams;
  cudaStream_t readback = nullptr;
  int next_stream = 0;
  char* arena_base = nullptr;
  Arena arena;
  char* desc_base = nullptr;
  Arena desc;
  DevStatus* st = nullptr;
  unsigned long long* prof = nullptr;
  std::vector<BatchOutDev> out_stage;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<Req*> pending;
  std::vector<Req*> ready;
  std::vector<Wave> inflight;
  std::unordered_map<uint64_t, Req*> reqs;
  uint64_t next_id = 1;
  int64_t n_submitted = 0, n_admitted = 0, n_completed = 0, n_waves = 0, n_launches = 0;
  int worker_status = CUR_OK;
  std::string worker_err;
};

namespace {

int sfail(cur_ctx* ctx, int code, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  return ctx_fail_v(ctx, code, msg);
}

void release_scratch(cur_server* s, Req* r) {
  if (r->scratch_bytes) s->arena.release(r->scratch_off, r->scratch_bytes);
  if (r->a_bytes) s->arena.release(r->a_off, r->a_bytes);
  r->scratch_bytes = r->a_bytes = 0;
}

bool try_admit(cur_server* s, Req* r) {
  size_t so = 0, oo = 0, ao = 0;
  if (r->scratch_bytes && !s->arena.alloc(r->scratch_bytes, &so)) return false;
  if (!s->arena.alloc(r->out_bytes, &oo)) {
    if (r->scratch_bytes) s->arena.release(so, r->scratch_bytes);
    return false;
  }
  if (r->a_bytes && !s->arena.alloc(r->a_bytes, &ao)) {
    if (r->scratch_bytes) s->arena.release(so, r->scratch_bytes);
    s->arena.release(oo, r->out_bytes);
    return false;
  }
  r->scratch_off = so;
  r->out_off = oo;
  r->a_off = ao;
  const size_t rm = (size_t)r->rmax;
  r->off_I = oo;
  r->off_J = oo + al256(8 * rm);
  r->off_U = r->off_J + al256(8 * rm);
  r->off_h = r->off_U + al256(8 * rm * rm);
  return true;
}

void fail_worker(cur_server* s, cudaError_t e, const char* what) {
  if (s->worker_status == CUR_OK) {
    s->worker_status = CUR_ECUDA;
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    s->worker_err = buf;
  }
}

// Launch every admitted request as one wave on the next stream.
void launch_wave(cur_server* s) {
  const int n = (int)std::min<size_t>(s->ready.size(), kMaxWave);
  Wave w;
  w.stream = s->next_stream;
  s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
  w.desc_bytes = (sizeof(BatchJobDev) + sizeof(BatchOutDev)) * (size_t)n + 256;
  if (!s->desc.alloc(w.desc_bytes, &w.desc_off)) return;  // retry after a wave retires
  cudaStream_t st = s->streams[(size_t)w.stream];
  std::vector<BatchJobDev> jobs((size_t)n);
  for (int k = 0; k < n; ++k) {
    Req* r = s->ready[(size_t)k];
    BatchJobDev& j = jobs[(size_t)k];
    j.A = r->job.A;
    j.lda = r->job.lda;
    if (r->a_on_host) {
      const size_t es = s->a_f32 ? 4 : 8;
      cudaError_t e = cudaMemcpy2DAsync(s->arena_base + r->a_off, (size_t)r->job.n * es, r->job.A,
                                        (size_t)r->job.lda * es, (size_t)r->job.n * es,
                                        (size_t)r->job.m, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) fail_worker(s, e, "copy of a host request");
      j.A = s->arena_base + r->a_off;
      j.lda = r->job.n;
    }
    j.m = r->job.m;
    j.n = r->job.n;
    j.tol = r->job.tol;
    j.b = r->job.block_size;
    j.c = r->c;
    j.seed = r->job.seed;
    j.rmax = r->rmax;
    j.off_ij = (int64_t)(r->off_I / 8);
    j.off_j = (int64_t)(r->off_J / 8);
    j.off_u = (int64_t)(r->off_U / 8);
    j.off_hist = (int64_t)(r->off_h / 8);
    j.ws = s->arena_base + r->scratch_off;
    r->state = kRunning;
    w.reqs.push_back(r);
  }
  s->ready.erase(s->ready.begin(), s->ready.begin() + n);
  char* d = s->desc_base + w.desc_off;
  BatchParams P{};
  P.jobs = reinterpret_cast<BatchJobDev*>(d);
  P.out = reinterpret_cast<BatchOutDev*>(d + al256(sizeof(BatchJobDev) * (size_t)n));
  P.njobs = n;
  P.Iout = reinterpret_cast<int64_t*>(s->arena_base);
  P.Jout = reinterpret_cast<int64_t*>(s->arena_base);
  P.Uout = reinterpret_cast<double*>(s->arena_base);
  P.rho_hist = reinterpret_cast<double*>(s->arena_base);
  P.st = s->st;
  P.prof = s->prof;
  P.panel_bytes = kBatchMaxPanelBytes;
  P.team = s->team;
  cudaError_t e = cudaMemcpyAsync((void*)P.jobs, jobs.data(), sizeof(BatchJobDev) * (size_t)n,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = launch_serve(LaunchEnv{st, s->ctx->num_sms, s->ctx->device}, P, s->team, s->a_f32);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(w.ev, st);
  if (e != cudaSuccess) {
    fail_worker(s, e, "wave launch");
    if (w.ev) cudaEventDestroy(w.ev);
    w.ev = nullptr;
  }
  s->n_waves += 1;
  s->n_launches += w.ev ? 1 : 0;
  s->inflight.push_back(w);
}

void finish_wave(cur_server* s, Wave& w, cudaError_t q) {
  const size_t n = w.reqs.size();
  if (q == cudaSuccess && w.ev) {
    s->out_stage.resize(n);
    const char* d = s->desc_base + w.desc_off;
    const BatchOutDev* dout =
        reinterpret_cast<const BatchOutDev*>(d + al256(sizeof(BatchJobDev) * n));
    cudaError_t e = cudaMemcpyAsync(s->out_stage.data(), dout, sizeof(BatchOutDev) * n,
                                    cudaMemcpyDeviceToHost, s->readback);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->readback);
    if (e != cudaSuccess) fail_worker(s, e, "wave readback");
    else q = cudaSuccess;
  } else if (q != cudaSuccess) {
    fail_worker(s, q, "wave execution");
  }
  const double t = now_ms();
  for (size_t k = 0; k < n; ++k) {
    Req* r = w.reqs[k];
    if (s->worker_status == CUR_OK) {
      r->out = s->out_stage[k];
    } else {
      r->out = BatchOutDev{};
      r->out.status = CUR_ECUDA;
    }
    r->t_done = t;
    r->state = kDone;
    release_scratch(s, r);
    s->n_completed += 1;
  }
  s->desc.release(w.desc_off, w.desc_bytes);
  if (w.ev) cudaEventDestroy(w.ev);
  w.ev = nullptr;
}

// Run one large request alone through the single-matrix path (cur_run_opts
// on the private context), then copy its I, J, U and rho history into the
// request's output block.  Called with the lock released and no wave in flight.
// Returns the number of kernels the request launched.
int64_t run_big(cur_server* s, BigLane* ln, Req* r) {
  const size_t es = s->a_f32 ? 4 : 8;
  const void* A = r->job.A;
  int64_t lda = r->job.lda;
  cudaError_t e = cudaSuccess;
  if (r->a_on_host) {
    e = cudaMemcpy2DAsync(s->arena_base + r->a_off, (size_t)r->job.n * es, r->job.A,
                          (size_t)r->job.lda * es, (size_t)r->job.n * es, (size_t)r->job.m,
                          cudaMemcpyHostToDevice, ln->stream);
    A = s->arena_base + r->a_off;
    lda = r->job.n;
  }
  cur_opts o{};
  o.max_rank = r->rmax;
  cur_result* res = nullptr;
  int st = e == cudaSuccess ? cur_run_opts(ln->ctx, A, r->job.m, r->job.n, lda,
                                           s->a_f32 ? CUR_F32 : CUR_F64, r->job.tol,
                                           r->job.block_size, r->c, r->job.seed, &o, &res)
                            : CUR_ECUDA;
  r->out = BatchOutDev{};
  int64_t launches = 0;
  if (res) {
    launches = cur_result_kernel_launches(res);
    const int64_t k = cur_result_rank(res), it = cur_result_iterations(res);
    r->out.rank = k;
    r->out.iters = it;
    r->out.rho = cur_result_err(res);
    r->out.normY = cur_result_sketch_norm(res);
    r->out.status = cur_result_status(res);
    char* base = s->arena_base;
    if (k > 0) {
      e = cudaMemcpyAsync(base + r->off_I, cur_result_I(res), 8 * (size_t)k,
                          cudaMemcpyDeviceToDevice, ln->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + r->off_J, cur_result_J(res), 8 * (size_t)k,
                            cudaMemcpyDeviceToDevice, ln->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + r->off_U, cur_result_U(res), 8 * (size_t)(k * k),
                            cudaMemcpyDeviceToDevice, ln->stream);
    }
    const double* h = cur_result_rho_history(res);
    if (e == cudaSuccess && it > 0 && h)
      e = cudaMemcpyAsync(base + r->off_h, h, 8 * (size_t)it, cudaMemcpyHostToDevice,
                          ln->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ln->stream);
    cur_result_free(res);
    if (e != cudaSuccess) {
      r->out.status = CUR_ECUDA;
      r->err = cudaGetErrorString(e);
      cudaGetLastError();
    }
  } else {
    r->out.status = st == CUR_OK ? CUR_ECUDA : st;
    r->err = e != cudaSuccess ? cudaGetErrorString(e) : cur_last_error(ln->ctx);
    cudaGetLastError();
  }
  return launches;
}

void admit(cur_server* s) {
  int skipped = 0;
  for (auto it = s->pending.begin(); it != s->pending.end() && skipped <= kBackfill;) {
    Req* r = *it;
    if (try_admit(s, r)) {
      r->state = kAdmitted;
      r->t_admit = now_ms();
      s->ready.push_back(r);
      s->n_admitted += 1;
      it = s->pending.erase(it);
    } else {
      ++it;
      ++skipped;
    }
  }
}

bool lanes_busy(const cur_server* s) {
  for (const BigLane* ln : s->lanes)
    if (ln->job) return true;
  return false;
}

BigLane* idle_lane(cur_server* s) {
  for (BigLane* ln : s->lanes)
    if (!ln->job) return ln;
  return nullptr;
}

// A large-request worker: runs one request at a time through cur_run_opts on
// its own context.  Several lanes overlap their requests' launch and host-sync
// gaps; their cooperative kernels each wait only on their own CTAs, so one
// lane's kernel at worst queues behind another's for the length of a kernel.
void lane_main(cur_server* s, BigLane* ln) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    ln->cv.wait(lk, [&] { return ln->job != nullptr || ln->quit; });
    if (!ln->job) return;
    Req* r = ln->job;
    lk.unlock();
    const int64_t launches = run_big(s, ln, r);
    lk.lock();
    s->n_launches += launches;
    r->t_done = now_ms();
    r->state = kDone;
    if (r->a_bytes) s->arena.release(r->a_off, r->a_bytes);
    r->a_bytes = 0;
    s->n_completed += 1;
    ln->job = nullptr;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

void worker_main(cur_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool progressed = false;
    for (size_t k = 0; k < s->inflight.size();) {
      Wave& w = s->inflight[k];
      cudaError_t q = w.ev ? cudaEventQuery(w.ev) : cudaErrorUnknown;
      if (q == cudaErrorNotReady) { ++k; continue; }
      finish_wave(s, w, q);
      s->inflight.erase(s->inflight.begin() + (long)k);
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    admit(s);
    // large requests at the head of the ready list go to idle lanes once the
    // waves in flight have drained (no wave runs beside a large request)
    auto big_it = std::find_if(s->ready.begin(), s->ready.end(), [](Req* q) { return q->big; });
    if (big_it != s->ready.end()) {
      if (big_it == s->ready.begin()) {
        BigLane* ln;
        while (s->inflight.empty() && !s->ready.empty() && s->ready.front()->big &&
               (ln = idle_lane(s)) != nullptr) {
          Req* r = s->ready.front();
          s->ready.erase(s->ready.begin());
          r->state = kRunning;
          ln->job = r;
          s->n_waves += 1;
          ln->cv.notify_one();
          progressed = true;
        }
      } else if (!lanes_busy(s)) {
        // small requests ahead of the large one go out as one wave first
        const size_t nsmall = (size_t)(big_it - s->ready.begin());
        std::vector<Req*> rest(big_it, s->ready.end());
        s->ready.resize(nsmall);
        launch_wave(s);
        const bool launched = s->ready.empty();
        s->ready.insert(s->ready.end(), rest.begin(), rest.end());
        if (launched) progressed = true;
      }
    } else if (!s->ready.empty() && !lanes_busy(s)) {
      const size_t before = s->ready.size();
      launch_wave(s);
      if (s->ready.size() != before) progressed = true;
    }
    const bool busy = lanes_busy(s);
    if (s->stop && s->pending.empty() && s->ready.empty() && s->inflight.empty() && !busy) break;
    if (!progressed) {
      if (s->inflight.empty() && s->ready.empty() && (s->pending.empty() || s->stop)) {
        if (s->stop && !busy) break;
        s->cv_work.wait(lk);
      } else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(100));
        lk.lock();
      }
    }
  }
  s->cv_done.notify_all();
}

Req* find(cur_server* s, uint64_t ticket) {
  auto it = s->reqs.find(ticket);
  return it == s->reqs.end() ? nullptr : it->second;
}

}  // namespace

extern "C" {

int cur_server_create(cur_ctx* ctx, size_t hbm_budget, int dtype, int team, int streams,
                      int64_t big_elements, int big_lanes, cur_server** out) {
  if (!out) return sfail(ctx, CUR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctx) return CUR_EINVAL;
  if (dtype != CUR_F32 && dtype != CUR_F64) return sfail(ctx, CUR_EINVAL, "dtype %d", dtype);
  if (team < 1 || team > 8) return sfail(ctx, CUR_EINVAL, "team %d outside 1..8", team);
  if (streams < 1 || streams > 16) return sfail(ctx, CUR_EINVAL, "streams %d outside 1..16", streams);
  if (big_lanes < 1 || big_lanes > 4) return sfail(ctx, CUR_EINVAL, "big_lanes %d outside 1..4", big_lanes);
  if (hbm_budget < ((size_t)1 << 20)) return sfail(ctx, CUR_EINVAL, "budget below 1 MiB");
  if (cudaSetDevice(ctx->device) != cudaSuccess) { cudaGetLastError(); return sfail(ctx, CUR_ECUDA, "cudaSetDevice"); }
  const bool f32 = dtype == CUR_F32;
  if (serve_max_clusters(LaunchEnv{nullptr, ctx->num_sms, ctx->device}, team, f32,
                         kBatchMaxPanelBytes) < 1)
    return sfail(ctx, CUR_EINVAL, "clusters of %d CTAs of the serving kernel do not fit on this GPU",
                 team);
  if (ctx->budget && ctx->held + hbm_budget + kDescPool > ctx->budget)
    return sfail(ctx, CUR_EBUDGET, "server budget exceeds the context's HBM budget");
  cur_server* s = new cur_server();
  s->ctx = ctx;
  s->a_f32 = f32;
  s->team = team;
  s->big_elements = big_elements > 0 ? big_elements : 0;
  cudaError_t e = cudaMalloc((void**)&s->arena_base, hbm_budget);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->desc_base, kDescPool);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->st, sizeof(DevStatus) + 256);
  if (e == cudaSuccess) {
    s->prof = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(s->st) + 128);
    e = cudaMemset(s->st, 0, sizeof(DevStatus) + 256);
  }
  for (int k = 0; k < streams && e == cudaSuccess; ++k) {
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) s->streams.push_back(st);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->readback, cudaStreamNonBlocking);
  for (int k = 0; k < big_lanes && e == cudaSuccess; ++k) {
    BigLane* ln = new BigLane();
    s->lanes.push_back(ln);
    e = cudaStreamCreateWithFlags(&ln->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && cur_create(&ln->ctx, ctx->device, ln->stream, 0) != CUR_OK)
      e = cudaErrorMemoryAllocation;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    cur_server_free(s);
    return sfail(ctx, CUR_ENOMEM, "server allocation failed: %s", cudaGetErrorString(e));
  }
  ctx->held += hbm_budget + kDescPool;
  s->arena.init(hbm_budget);
  s->desc.init(kDescPool);
  for (BigLane* ln : s->lanes) ln->th = std::thread(lane_main, s, ln);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return CUR_OK;
}

void cur_server_free(cur_server* s) {
  if (!s) return;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->stop = true;
      // requests never admitted are dropped
      for (Req* r : s->pending) { r->state = kDone; r->out.status = CUR_ECUDA; }
      s->pending.clear();
    }
    s->cv_work.notify_all();
    s->worker.join();
  }
  {
    std::lock_guard<std::mutex> g(s->mu);
    for (BigLane* ln : s->lanes) {
      ln->quit = true;
      ln->cv.notify_all();
    }
  }
  for (BigLane* ln : s->lanes)
    if (ln->th.joinable()) ln->th.join();
  for (auto& kv : s->reqs) delete kv.second;
  if (s->arena_base) {
    cudaFree(s->arena_base);
    s->ctx->held -= std::min(s->ctx->held, s->arena.cap + kDescPool);
  }
  if (s->desc_base) cudaFree(s->desc_base);
  if (s->st) cudaFree(s->st);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  if (s->readback) cudaStreamDestroy(s->readback);
  for (BigLane* ln : s->lanes) {
    if (ln->ctx) cur_free(ln->ctx);
    if (ln->stream) cudaStreamDestroy(ln->stream);
    delete ln;
  }
  cudaGetLastError();
  delete s;
}

int cur_server_submit(cur_server* s, const cur_batch_job* job, int a_on_host, uint64_t* ticket) {
  if (!s || !job || !ticket) return CUR_EINVAL;
  cur_ctx* ctx = s->ctx;
  const int c = job->sketch_size == 0 ? (int)std::floor(1.1 * job->block_size) : job->sketch_size;
  const char* why = nullptr;
  if (!job->A) why = "A is NULL";
  else if (job->m < 1 || job->n < 1) why = "m and n must be >= 1";
  else if (job->lda < job->n) why = "lda < n";
  else if (!(job->tol > 0.0)) why = "tol must be > 0";
  else if (job->block_size < 1 || job->block_size > kBatchMaxB) why = "block_size outside 1..64";
  else if (c < job->block_size || c > kBatchMaxC) why = "sketch_size outside b..128";
  if (why) return sfail(ctx, CUR_EINVAL, "request: %s", why);
  Req* r = new Req();
  r->job = *job;
  r->a_on_host = a_on_host ? 1 : 0;
  r->c = c;
  const int64_t mn = std::min(job->m, job->n);
  r->rmax = (job->max_rank <= 0 || job->max_rank > mn) ? mn : job->max_rank;
  const BatchDims d{job->m, job->n, c, job->block_size, r->rmax};
  r->big = s->big_elements > 0 && job->m * job->n >= s->big_elements;
  // a large request's scratch lives in the private context's workspace
  r->scratch_bytes = r->big ? 0 : serve_job_scratch_bytes(d, s->team);
  const size_t rm = (size_t)r->rmax;
  r->out_bytes = 2 * al256(8 * rm) + al256(8 * rm * rm) +
                 al256(8 * (size_t)((r->rmax + job->block_size - 1) / job->block_size));
  r->a_bytes = a_on_host ? (size_t)job->m * (size_t)job->n * (s->a_f32 ? 4 : 8) : 0;
  const size_t total = al256(r->scratch_bytes) + al256(r->out_bytes) + al256(r->a_bytes);
  if (total > s->arena.cap) {
    delete r;
    return sfail(ctx, CUR_EBUDGET, "request footprint %zu bytes exceeds the server budget %zu",
                 total, s->arena.cap);
  }
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->worker_status != CUR_OK) {
      delete r;
      return sfail(ctx, s->worker_status, "server failed: %s", s->worker_err.c_str());
    }
    r->id = s->next_id++;
    r->t_submit = now_ms();
    s->reqs[r->id] = r;
    s->pending.push_back(r);
    s->n_submitted += 1;
    *ticket = r->id;
  }
  s->cv_work.notify_all();
  return CUR_OK;
}

int cur_server_poll(cur_server* s, uint64_t ticket, int* done) {
  if (!s || !done) return CUR_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  Req* r = find(s, ticket);
  if (!r) return ctx_fail_v(s->ctx, CUR_EINVAL, "unknown ticket");
  *done = r->state == kDone ? 1 : 0;
  return CUR_OK;
}

int cur_server_wait(cur_server* s, uint64_t ticket, double timeout_s) {
  if (!s) return CUR_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  Req* r = find(s, ticket);
  if (!r) return ctx_fail_v(s->ctx, CUR_EINVAL, "unknown ticket");
  auto pred = [&] { return r->state == kDone; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, pred);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
    return ctx_fail_v(s->ctx, CUR_ETIMEOUT, "request still running");
  }
  if (s->worker_status != CUR_OK)
    return sfail(s->ctx, s->worker_status, "server failed: %s", s->worker_err.c_str());
  return CUR_OK;
}

int cur_server_drain(cur_server* s) {
  if (!s) return CUR_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] {
    return (s->pending.empty() && s->ready.empty() && s->inflight.empty() && !lanes_busy(s)) ||
           s->worker_status != CUR_OK;
  });
  if (s->worker_status != CUR_OK)
    return sfail(s->ctx, s->worker_status, "server failed: %s", s->worker_err.c_str());
  return CUR_OK;
}

int cur_server_result(cur_server* s, uint64_t ticket, int64_t* rank, int64_t* iters, double* rho,
                      int* status, double* latency_ms, double* queue_ms) {
  if (!s) return CUR_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  Req* r = find(s, ticket);
  if (!r) return ctx_fail_v(s->ctx, CUR_EINVAL, "unknown ticket");
  if (r->state != kDone) return ctx_fail_v(s->ctx, CUR_EINVAL, "request not completed");
  if (rank) *rank = r->out.rank;
  if (iters) *iters = r->out.iters;
  if (rho) *rho = r->out.rho;
  if (status) *status = r->out.status;
  if (latency_ms) *latency_ms = r->t_done - r->t_submit;
  if (queue_ms) *queue_ms = r->t_admit - r->t_submit;
  if (!r->err.empty()) ctx_fail_v(s->ctx, CUR_OK, r->err.c_str());
  return CUR_OK;
}

int cur_server_copy(cur_server* s, uint64_t ticket, int64_t* I, int64_t* J, double* U,
                    double* rho_history) {
  if (!s) return CUR_EINVAL;
  cur_ctx* ctx = s->ctx;
  Req* r;
  {
    std::lock_guard<std::mutex> g(s->mu);
    r = find(s, ticket);
    if (!r) return ctx_fail_v(ctx, CUR_EINVAL, "unknown ticket");
    if (r->state != kDone) return ctx_fail_v(ctx, CUR_EINVAL, "request not completed");
  }
  if (r->out.status == CUR_ECUDA) return ctx_fail_v(ctx, CUR_ECUDA, "request failed");
  const size_t k = (size_t)r->out.rank, it = (size_t)r->out.iters;
  const char* base = s->arena_base;
  cudaError_t e = cudaSuccess;
  if (k && I) e = cudaMemcpy(I, base + r->off_I, 8 * k, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && k && J) e = cudaMemcpy(J, base + r->off_J, 8 * k, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && k && U) e = cudaMemcpy(U, base + r->off_U, 8 * k * k, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && it && rho_history)
    e = cudaMemcpy(rho_history, base + r->off_h, 8 * it, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sfail(ctx, CUR_ECUDA, "result copy: %s", cudaGetErrorString(e));
  return CUR_OK;
}

int cur_server_release(cur_server* s, uint64_t ticket) {
  if (!s) return CUR_EINVAL;
  {
    std::lock_guard<std::mutex> g(s->mu);
    Req* r = find(s, ticket);
    if (!r) return ctx_fail_v(s->ctx, CUR_EINVAL, "unknown ticket");
    if (r->state != kDone) return ctx_fail_v(s->ctx, CUR_EINVAL, "request not completed");
    s->arena.release(r->out_off, r->out_bytes);
    s->reqs.erase(ticket);
    delete r;
  }
  s->cv_work.notify_all();  // freed memory may admit pending requests
  return CUR_OK;
}

int cur_server_get_stats(cur_server* s, cur_server_stats* o) {
  if (!s || !o) return CUR_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  o->submitted = s->n_submitted;
  o->admitted = s->n_admitted;
  o->completed = s->n_completed;
  o->waves = s->n_waves;
  o->launches = s->n_launches;
  o->bytes_in_use = s->arena.used;
  o->bytes_peak = s->arena.peak;
  o->budget = s->arena.cap;
  o->pending = (int64_t)s->pending.size();
  o->in_flight = (int64_t)(s->ready.size());
  for (const Wave& w : s->inflight) o->in_flight += (int64_t)w.reqs.size();
  for (const BigLane* ln : s->lanes) o->in_flight += ln->job ? 1 : 0;
  return CUR_OK;
}

}  // extern "C"
