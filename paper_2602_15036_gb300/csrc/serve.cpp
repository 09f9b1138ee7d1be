// Continuous-batching request server (litho_serve_*).
//
// Requests (one clip each: an aerial image, or one ILT gradient step) arrive
// at any time.  A scheduler thread admits queued requests whenever a slot
// (one non-blocking CUDA stream) is free and the request's device footprint
// fits in what the HBM budget has left; a request that does not fit yet is
// skipped so that smaller ones behind it can start (no head-of-line
// blocking), except that the oldest request, once skipped many times, holds
// admission until it fits (no starvation).  Admitted work is enqueued on the
// slot's stream: stream-ordered allocation, host-to-device copy from pinned
// staging, the imaging or gradient kernels, device-to-host copy, stream-
// ordered free, and a host callback that records completion.  Requests on
// different slots overlap on the device.  Kernel sets are built once per
// (optics, n, pixel, defocus, k) on a builder thread and stay resident; a
// request whose kernels are still being built waits without blocking others.
// All device kernels are deterministic, so a result is bit-identical whether
// the request ran alone or in a mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "litho_internal.h"

namespace litho {
namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kQueued = 0, kRunning, kDone, kCancelled, kFailed };

struct KernelEntry {
  litho_kernels* h = nullptr;
  bool building = false, failed = false;
  litho_status status = LITHO_OK;
  std::string err;
  litho_optics optics{};
  std::vector<double> custom;
  int n = 0, k = 0;
  double pixel = 0, z = 0;
  size_t bytes = 0;
};

struct Req {
  uint64_t ticket = 0;
  litho_request r{};
  std::vector<double> custom;
  std::string key;
  int state = kQueued;
  litho_status result = LITHO_OK;
  std::string err;
  size_t footprint = 0;
  int skipped = 0;
  double t_submit = 0, t_done = 0;
  int slot = -1;
  litho_server* srv = nullptr;
  bool in_pinned = false, out_pinned = false;  // caller buffers usable for DMA directly
};

// True for page-locked (cudaHostAlloc / cudaHostRegister) host memory.
bool is_pinned(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

struct Slot {
  cudaStream_t stream = nullptr;
  bool busy = false;
  char* pinned = nullptr;
  size_t pinned_bytes = 0;
};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

std::string kernel_key(const litho_request& r, const std::vector<double>& custom) {
  char buf[512];
  const litho_optics& o = r.optics;
  snprintf(buf, sizeof(buf), "%a|%a|%a|%d|%d|%a|%a|%a|%a|%d|%a|%a|%d", o.wavelength_nm, o.na, o.n_medium, o.kind,
           o.src_grid, o.sigma_in, o.sigma_out, o.pole_sigma, o.pole_radius, r.n, r.pixel_nm, r.defocus_nm, r.k);
  std::string s(buf);
  for (double w : custom) {
    snprintf(buf, sizeof(buf), "|%a", w);
    s += buf;
  }
  return s;
}

// Device bytes of one request (inputs, output, workspace) for a kernel set shape.
size_t request_bytes(const litho_request& r, int crop) {
  litho_kernels shape;
  shape.n = r.n;
  shape.crop = crop;
  shape.n_focus = 1;
  shape.k = r.k;
  shape.pixel_nm = r.pixel_nm;
  shape.nc = coarse_grid(crop, r.n, false);  // as the kernel upload computes them
  shape.nc_tc = coarse_grid(crop, r.n, true);
  const size_t nn = size_t(r.n) * r.n;
  size_t ws = 0;
  if (r.kind == LITHO_REQ_IMAGE) {
    litho_aerial_workspace_size(&shape, 1, static_cast<litho_precision>(r.precision), &ws);
    return up256(nn * 4) + up256(nn * 4) + up256(ws);
  }
  litho_ilt_workspace_size(&shape, 1, &ws, nullptr);
  return 3 * up256(nn * 4) + up256(ws);
}

}  // namespace
}  // namespace litho

struct litho_server {
  size_t budget = 0;
  int max_slots = 0, max_queue = 0, device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::thread sched, builder;
  bool stop = false;
  std::deque<litho::Req*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<litho::Req>> reqs;
  std::vector<litho::Slot> slots;
  std::map<std::string, litho::KernelEntry> cache;
  std::deque<std::string> build_queue;
  size_t in_use = 0, high_water = 0, cache_bytes = 0;
  int running = 0;
  uint64_t next_ticket = 1, submitted = 0, completed = 0, rejected = 0, cancelled = 0;
  std::vector<double> latencies;
  double first_submit = -1.0, last_done = 0.0, pixels = 0.0;
  std::atomic<int> fault_mask{0};
};

namespace litho {
namespace {

void finish_locked(litho_server* s, Req* q, int state, litho_status st, const char* msg) {
  q->state = state;
  q->result = st;
  if (msg) q->err = msg;
  q->t_done = now_ms();
  if (q->slot >= 0) {
    s->slots[q->slot].busy = false;
    s->running--;
    s->in_use -= q->footprint;
    q->slot = -1;
  }
  if (state == kDone) {
    s->completed++;
    s->latencies.push_back(q->t_done - q->t_submit);
    s->last_done = q->t_done;
    s->pixels += double(q->r.n) * q->r.n;
  }
  s->cv.notify_all();
}

void CUDART_CB on_done(void* arg) {
  Req* q = static_cast<Req*>(arg);
  litho_server* s = q->srv;
  // The slot stays busy until finish_locked, so its staging buffer is ours here.
  Slot& sl = s->slots[q->slot];
  const size_t nn = size_t(q->r.n) * q->r.n;
  const size_t in_bytes = nn * 4 * (q->r.kind == LITHO_REQ_ILT_STEP ? 2 : 1);
  if (!q->out_pinned) std::memcpy(q->r.output_host, sl.pinned + up256(in_bytes), nn * 4);
  if (q->r.kind == LITHO_REQ_ILT_STEP && q->r.loss_host)
    std::memcpy(q->r.loss_host, sl.pinned + up256(in_bytes) + up256(nn * 4), sizeof(double));
  std::lock_guard<std::mutex> lk(s->mu);
  finish_locked(s, q, kDone, LITHO_OK, nullptr);
}

constexpr double kInjectedDelayMs = 200.0;  // the injected slow request's device delay

// Enqueues an admitted request on its slot's stream (called without the lock).
litho_status launch(litho_server* s, Req* q, litho_kernels* h, std::string* err) {
  Slot& sl = s->slots[q->slot];
  const litho_request& r = q->r;
  const size_t nn = size_t(r.n) * r.n;
  const bool ilt = r.kind == LITHO_REQ_ILT_STEP;
  const size_t in_bytes = nn * 4 * (ilt ? 2 : 1);
  const size_t stage = up256(in_bytes) + up256(nn * 4) + 256;
  if (sl.pinned_bytes < stage) {
    if (sl.pinned) cudaFreeHost(sl.pinned);
    sl.pinned = nullptr;
    sl.pinned_bytes = 0;
    if (cudaMallocHost(&sl.pinned, stage) != cudaSuccess) {
      *err = "pinned staging allocation failed";
      return LITHO_ENOMEM;
    }
    sl.pinned_bytes = stage;
  }
  // Pinned caller buffers are copied by DMA directly; pageable ones go through
  // the slot's pinned staging buffer.
  q->in_pinned = is_pinned(r.input_host) && (!ilt || is_pinned(r.target_host));
  q->out_pinned = is_pinned(r.output_host);
  if (!q->in_pinned) {
    std::memcpy(sl.pinned, r.input_host, nn * 4);
    if (ilt) std::memcpy(sl.pinned + nn * 4, r.target_host, nn * 4);
  }
  const size_t dev_bytes = q->footprint;
  void* d = nullptr;
  if (s->fault_mask.load() & 1) {
    s->fault_mask.fetch_and(~1);
    *err = "injected device allocation failure";
    return LITHO_ENOMEM;
  }
  if (s->fault_mask.load() & 2) {  // a slow request: a fixed device delay before its work
    s->fault_mask.fetch_and(~2);
    if (launch_delay(sl.stream, kInjectedDelayMs) != cudaSuccess) {
      *err = "delay launch failed";
      return LITHO_ECUDA;
    }
  }
  if (cudaMallocAsync(&d, dev_bytes, sl.stream) != cudaSuccess) {
    cudaGetLastError();
    *err = "device allocation failed";
    return LITHO_ENOMEM;
  }
  char* base = static_cast<char*>(d);
  float* d_in = reinterpret_cast<float*>(base);
  float* d_tg = ilt ? reinterpret_cast<float*>(base + up256(nn * 4)) : nullptr;
  float* d_out = reinterpret_cast<float*>(base + up256(nn * 4) * (ilt ? 2 : 1));
  char* ws = base + up256(nn * 4) * (ilt ? 3 : 2);
  const size_t ws_bytes = dev_bytes - up256(nn * 4) * (ilt ? 3 : 2);
  litho_status st = LITHO_OK;
  auto fail = [&](litho_status code, const char* what) {
    *err = what;
    cudaFreeAsync(d, sl.stream);
    return code;
  };
  if (q->in_pinned) {
    if (cudaMemcpyAsync(d_in, r.input_host, nn * 4, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess ||
        (ilt && cudaMemcpyAsync(d_tg, r.target_host, nn * 4, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess))
      return fail(LITHO_ECUDA, "host-to-device copy failed");
  } else if (cudaMemcpyAsync(d_in, sl.pinned, in_bytes, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess) {
    return fail(LITHO_ECUDA, "host-to-device copy failed");
  }
  if (ilt) {
    st = litho_ilt_grad(h, d_in, d_tg, 1, r.dose, r.mask_steep, r.resist_steep, r.threshold, r.sigma_nm,
                        static_cast<litho_precision>(LITHO_PREC_FFT32 | LITHO_GRID_COARSE), d_out, nullptr, ws,
                        ws_bytes, sl.stream);
  } else {
    st = litho_aerial(h, d_in, 1, r.dose, static_cast<litho_precision>(r.precision), d_out, ws, ws_bytes, sl.stream);
  }
  if (st != LITHO_OK) return fail(st, litho_last_error());
  if (cudaMemcpyAsync(q->out_pinned ? static_cast<void*>(r.output_host) : sl.pinned + up256(in_bytes), d_out, nn * 4,
                      cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
    return fail(LITHO_ECUDA, "device-to-host copy failed");
  if (ilt) {
    double* loss_dev = ilt_loss_device(h, 1, ws, ws_bytes);
    if (cudaMemcpyAsync(sl.pinned + up256(in_bytes) + up256(nn * 4), loss_dev, sizeof(double),
                        cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
      return fail(LITHO_ECUDA, "device-to-host copy failed");
  }
  cudaFreeAsync(d, sl.stream);
  if (cudaLaunchHostFunc(sl.stream, on_done, q) != cudaSuccess) {
    *err = "cudaLaunchHostFunc failed";
    return LITHO_ECUDA;
  }
  return LITHO_OK;
}

void scheduler(litho_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    if (s->stop && s->running == 0) break;
    bool admitted = false;
    if (!s->stop) {
      int free_slot = -1;
      for (int i = 0; i < s->max_slots; ++i)
        if (!s->slots[i].busy) {
          free_slot = i;
          break;
        }
      for (auto it = s->queue.begin(); it != s->queue.end() && free_slot >= 0;) {
        Req* q = *it;
        KernelEntry& ke = s->cache[q->key];
        if (ke.failed) {
          it = s->queue.erase(it);
          finish_locked(s, q, kFailed, ke.status, ke.err.c_str());
          continue;
        }
        if (!ke.h) {
          if (!ke.building) {
            ke.building = true;
            ke.optics = q->r.optics;
            ke.custom = q->custom;
            ke.optics.custom_w = ke.custom.empty() ? nullptr : ke.custom.data();
            ke.n = q->r.n;
            ke.k = q->r.k;
            ke.pixel = q->r.pixel_nm;
            ke.z = q->r.defocus_nm;
            s->build_queue.push_back(q->key);
            s->cv.notify_all();
          }
          ++it;
          continue;
        }
        if (s->in_use + q->footprint > s->budget - std::min(s->budget, s->cache_bytes)) {
          const bool oldest = (it == s->queue.begin());
          if (oldest && ++q->skipped > 64) break;  // hold admission for the oldest request
          ++it;
          continue;
        }
        it = s->queue.erase(it);
        q->state = kRunning;
        q->slot = free_slot;
        s->slots[free_slot].busy = true;
        s->running++;
        s->in_use += q->footprint;
        s->high_water = std::max(s->high_water, s->in_use + s->cache_bytes);
        litho_kernels* h = ke.h;
        lk.unlock();
        std::string err;
        litho_status st = launch(s, q, h, &err);
        lk.lock();
        if (st != LITHO_OK) finish_locked(s, q, kFailed, st, err.c_str());
        admitted = true;
        break;
      }
    }
    if (!admitted) s->cv.wait_for(lk, std::chrono::milliseconds(20));
  }
}

void kernel_builder(litho_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv.wait(lk, [&] { return s->stop || !s->build_queue.empty(); });
    if (s->stop) break;
    const std::string key = s->build_queue.front();
    s->build_queue.pop_front();
    KernelEntry& ke = s->cache[key];
    litho_optics o = ke.optics;
    const int n = ke.n, k = ke.k;
    const double pixel = ke.pixel, z = ke.z;
    lk.unlock();
    litho_kernels* h = nullptr;
    litho_status st = litho_make_kernels(&o, n, pixel, &z, 1, k, &h);
    std::string err = st == LITHO_OK ? "" : litho_last_error();
    lk.lock();
    KernelEntry& e2 = s->cache[key];
    e2.building = false;
    if (st == LITHO_OK) {
      e2.h = h;
      e2.bytes = size_t(h->crop) * h->crop * h->k * 8 + size_t(h->n) * 8 + size_t(h->k) * 4;
      s->cache_bytes += e2.bytes;
    } else {
      e2.failed = true;
      e2.status = st;
      e2.err = err;
    }
    s->cv.notify_all();
  }
}

}  // namespace
}  // namespace litho

using namespace litho;

extern "C" {

litho_status litho_serve_create(size_t hbm_budget_bytes, int max_slots, int max_queue, litho_server** out) {
  if (!out || max_slots < 1 || max_slots > 64 || max_queue < 1 || hbm_budget_bytes == 0) {
    set_error("need out != NULL, 1 <= max_slots <= 64, max_queue >= 1, budget > 0");
    return LITHO_EINVAL;
  }
  *out = nullptr;
  auto s = std::make_unique<litho_server>();
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->max_queue = max_queue;
  LITHO_TRY_CUDA(cudaGetDevice(&s->device));
  // Keep memory freed by cudaFreeAsync in the device pool instead of returning
  // it to the driver at every synchronisation: re-mapping it costs far more
  // than a request's kernels.
  cudaMemPool_t pool;
  LITHO_TRY_CUDA(cudaDeviceGetDefaultMemPool(&pool, s->device));
  uint64_t keep = ~0ull;
  LITHO_TRY_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  s->slots.resize(max_slots);
  // Pinned staging sized up front for the largest request (2048^2 ILT step:
  // theta, target, gradient), so no slot ever reallocates it: cudaFreeHost
  // and cudaMallocHost both wait for the whole device.
  const size_t nn = size_t(2048) * 2048;
  const size_t stage = up256(nn * 4 * 2) + up256(nn * 4) + 256;
  for (auto& sl : s->slots) {
    LITHO_TRY_CUDA(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
    LITHO_TRY_CUDA(cudaMallocHost(&sl.pinned, stage));
    sl.pinned_bytes = stage;
  }
  litho_server* raw = s.release();
  raw->sched = std::thread(scheduler, raw);
  raw->builder = std::thread(kernel_builder, raw);
  *out = raw;
  return LITHO_OK;
}

litho_status litho_serve_submit(litho_server* s, const litho_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) {
    set_error("null argument");
    return LITHO_EINVAL;
  }
  const litho_request& r = *req;
  const bool pow2 = r.n >= 32 && r.n <= 2048 && (r.n & (r.n - 1)) == 0;
  if (!pow2 || r.k < 1 || r.k > 1024 || !(r.pixel_nm > 0) || !std::isfinite(r.defocus_nm) || !r.input_host ||
      !r.output_host || (r.kind != LITHO_REQ_IMAGE && r.kind != LITHO_REQ_ILT_STEP) ||
      (r.kind == LITHO_REQ_ILT_STEP && !r.target_host) || (r.precision & ~(0xFF | LITHO_GRID_COARSE)) != 0 ||
      (r.precision & 0xFF) > LITHO_PREC_FP16) {
    set_error("invalid request fields");
    std::lock_guard<std::mutex> lk(s->mu);
    s->rejected++;
    return LITHO_EINVAL;
  }
  SourcePoints src;
  std::string why;
  if (!sample_source(r.optics, &src, &why)) {
    set_error("%s", why.c_str());
    std::lock_guard<std::mutex> lk(s->mu);
    s->rejected++;
    return LITHO_EINVAL;
  }
  auto q = std::make_unique<Req>();
  q->r = r;
  if (r.kind == LITHO_REQ_ILT_STEP) q->r.precision = LITHO_PREC_FFT32;
  if (r.optics.kind == LITHO_SRC_CUSTOM && r.optics.custom_w)
    q->custom.assign(r.optics.custom_w, r.optics.custom_w + size_t(r.optics.src_grid) * r.optics.src_grid);
  q->r.optics.custom_w = q->custom.empty() ? nullptr : q->custom.data();
  const int crop = band_crop(r.optics, src, r.n, r.pixel_nm);
  q->footprint = request_bytes(q->r, crop);
  q->key = kernel_key(q->r, q->custom);
  q->srv = s;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    set_error("server is shutting down");
    return LITHO_ECANCELED;
  }
  if (q->footprint > s->budget) {
    set_error("request needs %zu device bytes, above the whole budget of %zu", q->footprint, s->budget);
    s->rejected++;
    return LITHO_EINVAL;
  }
  if (int(s->queue.size()) >= s->max_queue) {
    set_error("queue full (%d waiting)", s->max_queue);
    s->rejected++;
    return LITHO_EBUSY;
  }
  q->ticket = s->next_ticket++;
  q->t_submit = now_ms();
  if (s->first_submit < 0) s->first_submit = q->t_submit;
  *ticket = q->ticket;
  s->queue.push_back(q.get());
  s->reqs[q->ticket] = std::move(q);
  s->submitted++;
  s->cv.notify_all();
  return LITHO_OK;
}

litho_status litho_serve_poll(litho_server* s, uint64_t ticket, int timeout_ms) {
  if (!s) {
    set_error("null server");
    return LITHO_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("unknown ticket %llu", (unsigned long long)ticket);
    return LITHO_EINVAL;
  }
  Req* q = it->second.get();
  auto finished = [&] { return q->state == kDone || q->state == kCancelled || q->state == kFailed; };
  if (!finished() && timeout_ms > 0) s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished);
  if (q->state == kDone) return LITHO_OK;
  if (q->state == kCancelled) return LITHO_ECANCELED;
  if (q->state == kFailed) {
    set_error("%s", q->err.c_str());
    return q->result;
  }
  set_error("request %llu still %s", (unsigned long long)ticket, q->state == kQueued ? "queued" : "running");
  return LITHO_ETIMEOUT;
}

litho_status litho_serve_cancel(litho_server* s, uint64_t ticket) {
  if (!s) return LITHO_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("unknown ticket");
    return LITHO_EINVAL;
  }
  Req* q = it->second.get();
  if (q->state == kQueued) {
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), q));
    s->cancelled++;
    finish_locked(s, q, kCancelled, LITHO_ECANCELED, "cancelled");
    return LITHO_OK;
  }
  if (q->state == kCancelled) return LITHO_OK;
  if (q->state == kRunning) {
    set_error("request is running");
    return LITHO_EBUSY;
  }
  set_error("request already finished");
  return LITHO_EINVAL;
}

litho_status litho_serve_stats(litho_server* s, litho_serve_stats_t* out) {
  if (!s || !out) return LITHO_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->rejected = s->rejected;
  out->cancelled = s->cancelled;
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) {
    if (l.empty()) return 0.0;
    const double pos = p * (l.size() - 1);
    const size_t i = size_t(pos);
    const double f = pos - double(i);
    return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
  };
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  const double span = s->last_done - s->first_submit;
  out->mpx_per_s = (span > 0 && s->completed) ? s->pixels / (span * 1e-3) / 1e6 : 0.0;
  out->hbm_high_water = s->high_water;
  int built = 0;
  for (auto& kv : s->cache) built += kv.second.h != nullptr;
  out->kernel_sets_cached = built;
  return LITHO_OK;
}

litho_status litho_serve_stats_reset(litho_server* s) {
  if (!s) return LITHO_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->latencies.clear();
  s->submitted = s->completed = s->rejected = s->cancelled = 0;
  s->first_submit = -1.0;
  s->last_done = 0.0;
  s->pixels = 0.0;
  s->high_water = s->in_use + s->cache_bytes;
  return LITHO_OK;
}

litho_status litho_serve_inject_fault(litho_server* s, int fault_mask) {
  if (!s) return LITHO_EINVAL;
  s->fault_mask.store(fault_mask);
  return LITHO_OK;
}

void litho_serve_destroy(litho_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    while (!s->queue.empty()) {
      Req* q = s->queue.front();
      s->queue.pop_front();
      s->cancelled++;
      finish_locked(s, q, kCancelled, LITHO_ECANCELED, "server destroyed");
    }
    s->cv.notify_all();
  }
  if (s->sched.joinable()) s->sched.join();
  if (s->builder.joinable()) s->builder.join();
  for (auto& sl : s->slots) {
    if (sl.stream) {
      cudaStreamSynchronize(sl.stream);
      cudaStreamDestroy(sl.stream);
    }
    if (sl.pinned) cudaFreeHost(sl.pinned);
  }
  for (auto& kv : s->cache)
    if (kv.second.h) litho_free_kernels(kv.second.h);
  delete s;
}

}  // extern "C"
