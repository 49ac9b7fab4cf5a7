// ctx.cuh -- the library context shared by the translation units that
// implement the C ABI (cur_api.cu: single decompositions; cur_batch.cu: the
// batched engine).
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "../../include/cur.h"
#include "cur_internal.cuh"

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

enum BufId {
  B_OMEGA, B_S, B_LUPPW, B_SROWT, B_G1, B_G2, B_N, B_NP, B_SJK, B_T1, B_PARTS, B_SPLITK,
  B_LT, B_RT, B_I, B_J, B_MASKC, B_MASKR, B_QRSMALL, B_QRBIG, B_CORE, B_STATUS, B_AHOST,
  B_STEP_QR, B_STEP_LUPP, B_STEP_PARTS, B_TC, B_STEP_TC, B_TEAMCORE, B_FX, B_STEP_FX,
  B_PLT, B_PRT, B_QP, B_STEP_RP, B_STEP_RQ, B_PS, B_PNP, B_PRK, B_PT1, B_COUNT
};

struct cur_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  size_t held = 0;
  int num_sms = 0;
  std::string err;
  DevBuf buf[B_COUNT];
  cur::DevStatus* st_host = nullptr;  // pinned mirror of the device status block
  // phase timing (opts->timing): events recorded at phase boundaries
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_phase;      // phase that starts at event i (-1: none)
  bool timing = false;
  int64_t launches = 0;           // kernel launches of the current run
  // host-input runs: a copy stream and per-row-block events (created on demand)
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> copy_ev;
  // a second compute stream: the sketch matrix is generated there while the
  // column-scale pass of the FP64 tensor-core sketch reads A (created on demand)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t side_ev[2] = {nullptr, nullptr};
  // device blocks of freed results (U, I, J), reused by later runs
  std::vector<std::pair<void*, size_t>> result_pool;
};

namespace cur {
// Record `msg` as the context's last error and return `code`.
int ctx_fail_v(cur_ctx* ctx, int code, const char* msg);
}  // namespace cur
