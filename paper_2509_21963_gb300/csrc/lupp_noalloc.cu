// lupp_noalloc.cu -- LUPP index selection for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside another
// framework's memory pool or arena, allocation-free real-time or embedded
// loops, and setups whose allocator must not be re-entered mid-run.  For
// them, cur_step_lupp_noalloc runs the same selection kernel as
// cur_step_lupp, but takes its scratch (the working copy of the candidate
// matrix, the per-CTA publication slots, the grid-barrier word and the status
// word) from one file-scope device array of fixed size instead of a context
// workspace.  Every GPU that loads this library holds that array until the
// process exits.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/cur_steps.h"
#include "cur_internal.cuh"

// Scratch capacity: 16 MiB.  It holds nr * ncand doubles of working copy plus
// 2 * grid * lupp_slot_stride(nr) doubles of slots, e.g. 55 x 20000 or 50 x 20000.
constexpr size_t kNoAllocBytes = 16u << 20;

// The scratch itself: shared by every call on a device, keeps the last call's
// contents (the status and barrier words are cleared by each call).
static __device__ __align__(256) unsigned char g_lupp_scratch[kNoAllocBytes];

namespace {

constexpr size_t kHeaderBytes = 256;   // DevStatus + GridBar, 256-byte aligned
constexpr int kMaxDevices = 64;

// Device address of g_lupp_scratch per device, resolved once with that device
// current (the host-side name of the array is only a stand-in).
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

void put_err(char* err, size_t len, const char* msg) {
  if (err && len) {
    strncpy(err, msg, len - 1);
    err[len - 1] = '\0';
  }
}

size_t round_up(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" int cur_step_lupp_noalloc(int device, void* cuda_stream, const double* X, int64_t ldx,
                                     int64_t nr, int64_t ncand, int64_t steps, uint8_t* mask,
                                     int64_t* piv, char* err, size_t err_len) {
  using namespace cur;
  if (!X || !mask || !piv || nr < 1 || ncand < 1 || ldx < ncand || steps < 0 || steps > nr ||
      steps > ncand) {
    put_err(err, err_len, "cur_step_lupp_noalloc: bad arguments");
    return CUR_EINVAL;
  }
  if (device < 0 || device >= kMaxDevices) {
    put_err(err, err_len, "cur_step_lupp_noalloc: device index out of range");
    return CUR_EINVAL;
  }
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    put_err(err, err_len, cudaGetErrorString(e));
    return CUR_ECUDA;
  }
  LaunchEnv env;
  env.stream = static_cast<cudaStream_t>(cuda_stream);
  env.device = device;
  e = cudaDeviceGetAttribute(&env.num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    put_err(err, err_len, cudaGetErrorString(e));
    return CUR_ECUDA;
  }
  const int grid = lupp_grid(env, nr, ncand);
  const size_t slot_bytes =
      round_up(sizeof(double) * 2 * (size_t)grid * (size_t)lupp_slot_stride(nr));
  const size_t w_bytes = round_up(sizeof(double) * (size_t)nr * (size_t)ncand);
  if (kHeaderBytes + slot_bytes + w_bytes > kNoAllocBytes) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "cur_step_lupp_noalloc: needs %zu bytes of scratch (nr %lld x ncand %lld), "
             "the fixed maximum is %zu bytes",
             kHeaderBytes + slot_bytes + w_bytes, (long long)nr, (long long)ncand, kNoAllocBytes);
    put_err(err, err_len, msg);
    return CUR_EINVAL;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
      e = cudaGetSymbolAddress(&g_addr[device], g_lupp_scratch);
      if (e != cudaSuccess) {
        g_addr[device] = nullptr;
        put_err(err, err_len, cudaGetErrorString(e));
        return CUR_ECUDA;
      }
    }
    base = g_addr[device];
  }
  unsigned char* p = static_cast<unsigned char*>(base);
  DevStatus* st = reinterpret_cast<DevStatus*>(p);
  LuppWork w;
  w.bar = reinterpret_cast<GridBar*>(p + 128);
  w.slot_val = reinterpret_cast<double*>(p + kHeaderBytes);
  w.W = reinterpret_cast<double*>(p + kHeaderBytes + slot_bytes);
  w.max_grid = grid;
  // the status word must start at zero (the barrier is cleared by launch_lupp)
  e = cudaMemsetAsync(st, 0, sizeof(DevStatus), env.stream);
  if (e == cudaSuccess) e = launch_lupp(env, X, ldx, nr, ncand, steps, mask, piv, w, grid, st);
  DevStatus host_st;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&host_st, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, env.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(env.stream);
  if (e != cudaSuccess) {
    put_err(err, err_len, cudaGetErrorString(e));
    return CUR_ECUDA;
  }
  // the same mapping of the device status as the workspace entry point
  if (host_st.err == kDevTimeout) {
    put_err(err, err_len, "cur_step_lupp_noalloc: grid barrier exceeded its cycle budget");
    return CUR_ETIMEOUT;
  }
  if (host_st.err == kDevNoCandidate) {
    put_err(err, err_len, "cur_step_lupp_noalloc: fewer eligible candidates than steps");
    return CUR_EINVAL;
  }
  if (host_st.err != 0) {
    char msg[96];
    snprintf(msg, sizeof(msg), "cur_step_lupp_noalloc: device status %d", host_st.err);
    put_err(err, err_len, msg);
    return CUR_ECUDA;
  }
  put_err(err, err_len, "");
  return CUR_OK;
}
