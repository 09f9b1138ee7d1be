// Continuous-batching request server (litho_serve_*).
//
// Requests (one clip each: an aerial image, or one ILT gradient step) arrive
// at any time.  A scheduler thread admits queued work whenever a slot (one
// non-blocking CUDA stream) is free and the work's device footprint fits in
// what the HBM budget has left; a request that does not fit yet is skipped so
// that smaller ones behind it can start (no head-of-line blocking), except
// that the oldest request, once skipped many times, holds admission until it
// fits (no starvation).
//
// Batching: the admitted request takes with it every queued request that
// can share its launches: the same kernel set (optics, n, pixel, defocus, k),
// kind, precision and scalar parameters (dose; the ILT step's resist and
// sigmoid constants), in arrival order, up to kMaxBatch clips and kMaxBatchWork
// pixels (ILT steps counted twice), while the batch's footprint fits the budget and its pageable
// buffers fit the slot's pinned staging.  So requests that arrived while the
// GPU was busy run as one grouped call (litho_aerial / litho_ilt_grad on b
// clips), which images the clips in shared launches.  A batch is enqueued on
// its slot's stream: stream-ordered allocation, host-to-device copies (pinned
// caller buffers by DMA, pageable ones through the slot's pinned staging),
// the grouped imaging or gradient call, device-to-host copies, stream-ordered
// free, and one host callback that completes every request of the batch.
// Batches on different slots overlap on the device.  Kernel sets are built
// once per key on a builder thread and stay resident; a request whose
// kernels are still being built waits without blocking others.  The grouped
// calls give each clip the same result as the clip imaged alone, bit for
// bit, and all device kernels are deterministic, so a request's result does
// not depend on what it ran with.
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
  std::string key;   // kernel set
  std::string bkey;  // batch: kernel set, kind, precision, scalar parameters
  int crop = 0;
  int state = kQueued;
  litho_status result = LITHO_OK;
  std::string err;
  size_t footprint = 0;  // alone
  int skipped = 0;
  double t_submit = 0, t_done = 0;
  int slot = -1;
  bool in_pinned = false, out_pinned = false;  // caller buffers usable for DMA directly
  size_t stage_in = 0, stage_out = 0;          // offsets in the slot's pinned staging
};

constexpr int kMaxBatch = 64;  // clips per batch
// Work per batch, in pixels with an ILT step counting twice (it images and
// back-propagates): 8 image clips of 2048^2.  Larger batches would leave one
// slot with seconds of work while the others run dry.
constexpr double kMaxBatchWork = 8.0 * 2048.0 * 2048.0;
double work_px(const litho_request& r) { return double(r.n) * r.n * (r.kind == LITHO_REQ_ILT_STEP ? 2.0 : 1.0); }
// Batches of at most this much work run on their slot's high-priority stream:
// the GPU dispatches their thread blocks ahead of the waiting blocks of large
// requests, so small requests are not held behind them.
constexpr double kSmallBatchWork = 2.0 * 1024.0 * 1024.0;

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
  cudaStream_t stream = nullptr;      // the running batch's stream: one of the two below
  cudaStream_t lo = nullptr, hi = nullptr;  // low and high stream priority
  bool busy = false;
  char* pinned = nullptr;
  size_t pinned_bytes = 0;
  std::vector<Req*> batch;  // the requests running on this slot
  size_t footprint = 0;     // device bytes of the batch
  litho_server* srv = nullptr;
  int index = 0;
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

std::string batch_key(const litho_request& r, const std::string& kernel_key) {
  char buf[256];
  snprintf(buf, sizeof(buf), "#%d|%d|%a", r.kind, r.precision, r.dose);
  std::string s = kernel_key + buf;
  if (r.kind == LITHO_REQ_ILT_STEP) {
    snprintf(buf, sizeof(buf), "|%a|%a|%a|%a", r.sigma_nm, r.threshold, r.mask_steep, r.resist_steep);
    s += buf;
  }
  return s;
}

// The precision code the batch's call takes (ILT steps run on the coarse grid).
int call_precision(const litho_request& r) {
  return r.kind == LITHO_REQ_ILT_STEP ? int(LITHO_PREC_FFT32 | LITHO_GRID_COARSE) : r.precision;
}

// Workspace bytes of the grouped call for b clips, for a kernel set shape.
size_t workspace_bytes(const litho_request& r, int crop, int b) {
  litho_kernels shape;
  shape.n = r.n;
  shape.crop = crop;
  shape.n_focus = 1;
  shape.k = r.k;
  shape.pixel_nm = r.pixel_nm;
  shape.nc = coarse_grid(crop, r.n, false);  // as the kernel upload computes them
  shape.nc_tc = coarse_grid(crop, r.n, true);
  size_t ws = 0;
  if (r.kind == LITHO_REQ_IMAGE)
    litho_aerial_workspace_size(&shape, b, static_cast<litho_precision>(r.precision), &ws);
  else
    litho_ilt_workspace_size(&shape, b, &ws, nullptr);
  return ws;
}

// Device bytes of a batch of b clips: inputs [b][n][n] (and targets for ILT),
// outputs [b][n][n], workspace.
size_t batch_bytes(const litho_request& r, int crop, int b) {
  const size_t plane = up256(size_t(b) * r.n * r.n * 4);
  return plane * (r.kind == LITHO_REQ_ILT_STEP ? 3 : 2) + up256(workspace_bytes(r, crop, b));
}

// Pinned staging bytes a request needs when its buffers are pageable.
size_t staging_bytes(const Req* q) {
  const size_t nn4 = size_t(q->r.n) * q->r.n * 4;
  const bool ilt = q->r.kind == LITHO_REQ_ILT_STEP;
  size_t b = 0;
  if (!q->in_pinned) b += up256(nn4 * (ilt ? 2 : 1));
  if (!q->out_pinned) b += up256(nn4);
  if (ilt) b += 256;  // the loss
  return b;
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
  size_t reserved = 0;  // bytes reserved in the default memory pool at creation
  int running = 0;
  uint64_t next_ticket = 1, submitted = 0, completed = 0, rejected = 0, cancelled = 0;
  uint64_t batches = 0;  // batches launched in the statistics window
  int max_batch = 0;     // largest batch (clips) in the window
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
  q->slot = -1;
  if (state == kDone) {
    s->completed++;
    s->latencies.push_back(q->t_done - q->t_submit);
    s->last_done = q->t_done;
    s->pixels += double(q->r.n) * q->r.n;
  }
  s->cv.notify_all();
}

// Frees a slot whose batch has finished (or failed to launch).
void release_slot_locked(litho_server* s, Slot& sl) {
  sl.busy = false;
  sl.batch.clear();
  s->running--;
  s->in_use -= sl.footprint;
  sl.footprint = 0;
  s->cv.notify_all();
}

void CUDART_CB on_batch_done(void* arg) {
  Slot* sl = static_cast<Slot*>(arg);
  litho_server* s = sl->srv;
  // The slot stays busy until release_slot_locked, so its batch and staging are ours here.
  for (Req* q : sl->batch) {
    const size_t nn = size_t(q->r.n) * q->r.n;
    if (!q->out_pinned) std::memcpy(q->r.output_host, sl->pinned + q->stage_out, nn * 4);
    if (q->r.kind == LITHO_REQ_ILT_STEP && q->r.loss_host)
      std::memcpy(q->r.loss_host, sl->pinned + q->stage_out + (q->out_pinned ? 0 : up256(nn * 4)), sizeof(double));
  }
  std::lock_guard<std::mutex> lk(s->mu);
  for (Req* q : sl->batch) finish_locked(s, q, kDone, LITHO_OK, nullptr);
  release_slot_locked(s, *sl);
}

constexpr double kInjectedDelayMs = 200.0;  // the injected slow request's device delay

// Enqueues an admitted batch on its slot's stream (called without the lock).
// fault: the injected fault bits this batch takes (see litho_serve_inject_fault).
litho_status launch(litho_server* s, Slot& sl, litho_kernels* h, int fault, std::string* err) {
  const litho_request& r = sl.batch[0]->r;
  const int b = int(sl.batch.size());
  const size_t nn = size_t(r.n) * r.n;
  const bool ilt = r.kind == LITHO_REQ_ILT_STEP;
  // pageable buffers go through the slot's pinned staging (sized at admission)
  size_t off = 0;
  for (Req* q : sl.batch) {
    q->stage_in = off;
    if (!q->in_pinned) {
      std::memcpy(sl.pinned + off, q->r.input_host, nn * 4);
      if (ilt) std::memcpy(sl.pinned + off + nn * 4, q->r.target_host, nn * 4);
      off += up256(nn * 4 * (ilt ? 2 : 1));
    }
    q->stage_out = off;
    off += (q->out_pinned ? 0 : up256(nn * 4)) + (ilt ? 256 : 0);
  }
  if (off > sl.pinned_bytes) {  // admission keeps batches within the staging; a guard, not a path
    *err = "pinned staging too small for the batch";
    return LITHO_ENOMEM;
  }
  if (fault & 1) {
    *err = "injected device allocation failure";
    return LITHO_ENOMEM;
  }
  if ((fault & 2) && launch_delay(sl.stream, kInjectedDelayMs) != cudaSuccess) {  // a slow batch
    *err = "delay launch failed";
    return LITHO_ECUDA;
  }
  void* d = nullptr;
  if (cudaMallocAsync(&d, sl.footprint, sl.stream) != cudaSuccess) {
    cudaGetLastError();
    *err = "device allocation failed";
    return LITHO_ENOMEM;
  }
  const size_t plane = up256(size_t(b) * nn * 4);
  char* base = static_cast<char*>(d);
  float* d_in = reinterpret_cast<float*>(base);
  float* d_tg = ilt ? reinterpret_cast<float*>(base + plane) : nullptr;
  float* d_out = reinterpret_cast<float*>(base + plane * (ilt ? 2 : 1));
  char* ws = base + plane * (ilt ? 3 : 2);
  const size_t ws_bytes = sl.footprint - plane * (ilt ? 3 : 2);
  auto fail = [&](litho_status code, const char* what) {
    *err = what;
    cudaFreeAsync(d, sl.stream);
    return code;
  };
  for (int i = 0; i < b; ++i) {
    const Req* q = sl.batch[i];
    const void* src_in = q->in_pinned ? static_cast<const void*>(q->r.input_host) : sl.pinned + q->stage_in;
    if (cudaMemcpyAsync(d_in + i * nn, src_in, nn * 4, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
      return fail(LITHO_ECUDA, "host-to-device copy failed");
    if (ilt) {
      const void* src_tg =
          q->in_pinned ? static_cast<const void*>(q->r.target_host) : sl.pinned + q->stage_in + nn * 4;
      if (cudaMemcpyAsync(d_tg + i * nn, src_tg, nn * 4, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
        return fail(LITHO_ECUDA, "host-to-device copy failed");
    }
  }
  litho_status st;
  if (ilt)
    st = litho_ilt_grad(h, d_in, d_tg, b, r.dose, r.mask_steep, r.resist_steep, r.threshold, r.sigma_nm,
                        static_cast<litho_precision>(call_precision(r)), d_out, nullptr, ws, ws_bytes, sl.stream);
  else
    st = litho_aerial(h, d_in, b, r.dose, static_cast<litho_precision>(r.precision), d_out, ws, ws_bytes, sl.stream);
  if (st != LITHO_OK) return fail(st, litho_last_error());
  const double* loss_dev = ilt ? ilt_loss_device(h, b, ws, ws_bytes) : nullptr;
  for (int i = 0; i < b; ++i) {
    const Req* q = sl.batch[i];
    void* dst = q->out_pinned ? static_cast<void*>(q->r.output_host) : sl.pinned + q->stage_out;
    if (cudaMemcpyAsync(dst, d_out + i * nn, nn * 4, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
      return fail(LITHO_ECUDA, "device-to-host copy failed");
    if (ilt && cudaMemcpyAsync(sl.pinned + q->stage_out + (q->out_pinned ? 0 : up256(nn * 4)), loss_dev + i,
                               sizeof(double), cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
      return fail(LITHO_ECUDA, "device-to-host copy failed");
  }
  cudaFreeAsync(d, sl.stream);
  if (cudaLaunchHostFunc(sl.stream, on_batch_done, &sl) != cudaSuccess) {
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
        const size_t avail = s->budget - std::min(s->budget, s->cache_bytes);
        if (s->in_use + q->footprint > avail) {
          const bool oldest = (it == s->queue.begin());
          if (oldest && ++q->skipped > 64) break;  // hold admission for the oldest request
          ++it;
          continue;
        }
        Slot& sl = s->slots[free_slot];
        // an injected fault applies to a batch of this request alone
        const int fault = s->fault_mask.exchange(0);
        std::vector<Req*> batch{q};
        size_t fp = q->footprint, staging = staging_bytes(q);
        double work = work_px(q->r);
        if (!fault) {
          for (auto jt = std::next(it); jt != s->queue.end() && int(batch.size()) < kMaxBatch; ++jt) {
            Req* q2 = *jt;
            if (q2->bkey != q->bkey) continue;
            if (work + work_px(q2->r) > kMaxBatchWork) break;
            const size_t fp2 = batch_bytes(q->r, q->crop, int(batch.size()) + 1);
            if (s->in_use + fp2 > avail) break;
            const size_t st2 = staging + staging_bytes(q2);
            if (st2 > sl.pinned_bytes) continue;
            batch.push_back(q2);
            fp = fp2;
            staging = st2;
            work += work_px(q2->r);
          }
        }
        for (Req* m : batch) {
          s->queue.erase(std::find(s->queue.begin(), s->queue.end(), m));
          m->state = kRunning;
          m->slot = free_slot;
        }
        sl.busy = true;
        sl.batch = batch;
        sl.footprint = fp;
        sl.stream = work <= kSmallBatchWork ? sl.hi : sl.lo;
        s->running++;
        s->in_use += fp;
        s->high_water = std::max(s->high_water, s->in_use + s->cache_bytes);
        s->batches++;
        s->max_batch = std::max(s->max_batch, int(batch.size()));
        litho_kernels* h = ke.h;
        lk.unlock();
        std::string err;
        litho_status st = launch(s, sl, h, fault, &err);
        lk.lock();
        if (st != LITHO_OK) {
          for (Req* m : sl.batch) finish_locked(s, m, kFailed, st, err.c_str());
          release_slot_locked(s, sl);
        }
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
  for (int i = 0; i < max_slots; ++i) {
    s->slots[i].srv = s.get();
    s->slots[i].index = i;
  }
  // Pinned staging sized up front for the largest request (2048^2 ILT step:
  // theta, target, gradient), so no slot ever reallocates it: cudaFreeHost
  // and cudaMallocHost both wait for the whole device.
  const size_t nn = size_t(2048) * 2048;
  const size_t stage = up256(nn * 4 * 2) + up256(nn * 4) + 256;
  int prio_lo = 0, prio_hi = 0;  // numerically lower is higher priority
  LITHO_TRY_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
  for (auto& sl : s->slots) {
    LITHO_TRY_CUDA(cudaStreamCreateWithPriority(&sl.lo, cudaStreamNonBlocking, prio_lo));
    LITHO_TRY_CUDA(cudaStreamCreateWithPriority(&sl.hi, cudaStreamNonBlocking, prio_hi));
    sl.stream = sl.lo;
    LITHO_TRY_CUDA(cudaMallocHost(&sl.pinned, stage));
    sl.pinned_bytes = stage;
  }
  // Reserve the budget in the pool now (at most half of the free memory): the
  // scheduler thread allocates each batch with cudaMallocAsync, and a pool
  // that must grow maps memory inside that call, which holds up every later
  // admission.  One allocation and its free leave the pages mapped in the
  // pool (release threshold above), so batches are carved from them.
  size_t free_b = 0, total_b = 0;
  LITHO_TRY_CUDA(cudaMemGetInfo(&free_b, &total_b));
  s->reserved = std::min(hbm_budget_bytes, free_b / 2);
  if (s->reserved > 0) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, s->reserved, s->slots[0].stream) == cudaSuccess) {
      LITHO_TRY_CUDA(cudaFreeAsync(p, s->slots[0].stream));
      LITHO_TRY_CUDA(cudaStreamSynchronize(s->slots[0].stream));
    } else {
      cudaGetLastError();  // the reservation is an optimisation: carry on without it
      s->reserved = 0;
    }
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
  q->crop = band_crop(r.optics, src, r.n, r.pixel_nm);
  q->footprint = batch_bytes(q->r, q->crop, 1);
  q->key = kernel_key(q->r, q->custom);
  q->bkey = batch_key(q->r, q->key);
  // pinned caller buffers are copied by DMA directly; pageable ones through the slot's staging
  q->in_pinned = is_pinned(r.input_host) && (r.kind != LITHO_REQ_ILT_STEP || is_pinned(r.target_host));
  q->out_pinned = is_pinned(r.output_host);
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
  out->batches = s->batches;
  out->max_batch = s->max_batch;
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
  s->batches = 0;
  s->max_batch = 0;
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
    for (cudaStream_t st : {sl.lo, sl.hi}) {
      if (!st) continue;
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    if (sl.pinned) cudaFreeHost(sl.pinned);
  }
  for (auto& kv : s->cache)
    if (kv.second.h) litho_free_kernels(kv.second.h);
  if (s->reserved) {  // hand the reservation back to the device
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
  }
  delete s;
}

}  // extern "C"
