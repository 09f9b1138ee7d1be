// Per-stage device timing: CUDA events recorded on the launching stream around
// each stage while profiling is enabled, resolved into per-stage totals when
// read.  Off by default; when off, a scope costs one relaxed atomic load and
// an NVTX range named after the stage (a no-op unless a tool is attached).
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstring>
#include <mutex>

#include "litho_internal.h"

namespace litho {

namespace {

const char* kStageNames[kStageCount] = {"mask_spectrum", "stage1_fft", "stage2_fft", "stage1_gemm_operands",
                                        "stage2_gemm",   "resist",     "ilt_forward", "ilt_backward",
                                        "ilt_reduce",    "upsample",   "upsample_resist", "contours",
                                        "epe",           "raster"};

struct Rec {
  int stage, launches;
  cudaEvent_t a, b;
};

std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Rec> g_pending;
std::vector<cudaEvent_t> g_pool;
double g_ms[kStageCount];
long long g_launches[kStageCount];

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void resolve_locked() {
  for (auto& r : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      g_ms[r.stage] += ms;
      g_launches[r.stage] += r.launches;
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_pending.clear();
}

}  // namespace

ProfScope::ProfScope(int stage, cudaStream_t st, int launches) : stage_(stage), st_(st), launches_(launches) {
  nvtxRangePushA(kStageNames[stage]);
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t a = get_event();
  if (a && cudaEventRecord(a, st_) != cudaSuccess) {
    g_pool.push_back(a);
    a = nullptr;
  }
  a_ = a;
}

ProfScope::~ProfScope() {
  nvtxRangePop();
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = get_event();
  if (b && cudaEventRecord(b, st_) == cudaSuccess) {
    g_pending.push_back(Rec{stage_, launches_, static_cast<cudaEvent_t>(a_), b});
  } else {
    g_pool.push_back(static_cast<cudaEvent_t>(a_));
  }
}

}  // namespace litho

using namespace litho;

extern "C" {

litho_status litho_profile_enable(int on) {
  g_on.store(on != 0);
  return LITHO_OK;
}

void litho_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked();
  std::memset(g_ms, 0, sizeof(g_ms));
  std::memset(g_launches, 0, sizeof(g_launches));
}

litho_status litho_profile_read(int max_stages, char* names, double* total_ms, long long* launches, int* count) {
  if (!count || (max_stages > 0 && (!names || !total_ms || !launches))) {
    set_error("null argument");
    return LITHO_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked();
  int n = 0;
  for (int s = 0; s < kStageCount && n < max_stages; ++s) {
    if (g_launches[s] == 0) continue;
    std::strncpy(names + 32 * n, kStageNames[s], 31);
    names[32 * n + 31] = 0;
    total_ms[n] = g_ms[s];
    launches[n] = g_launches[s];
    ++n;
  }
  *count = n;
  return LITHO_OK;
}

}  // extern "C"
