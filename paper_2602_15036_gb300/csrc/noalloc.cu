// litho_aerial_noalloc: the FP32 aerial-image path with its scratch in a
// fixed, library-owned device array instead of caller- or library-allocated
// memory.
//
// Who needs it: callers that must not allocate device memory at call time.
// cudaMalloc can stall until the whole device is idle and can fail under
// memory pressure, and cudaFree always waits for the device; a host
// application that owns every device allocation through its own pool (for
// example an OPC engine that budgets HBM per job), or a latency-critical loop
// that cannot afford such a stall, cannot take either.  This entry point
// performs no allocation at all: the caller passes the mask and the output,
// and the intermediate spectra and stage-1 fields live in `g_scratch` below.
//
// The array is a file-scope __device__ object, so every GPU on which the
// library is loaded reserves kScratchBytes for it until the process exits.
// Host code cannot use the symbol's name as a device address; the device
// address is looked up once per device with cudaGetSymbolAddress.
#include <cmath>
#include <mutex>

#include "litho_internal.h"

namespace litho {

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Bytes of g_scratch one clip needs: row spectrum [N][C], crop spectrum
// [C][C] and the stage-1 fields of all planes and kernels [F*K][N][C].
size_t clip_bytes(const litho_kernels* h) {
  const size_t N = h->n, C = h->crop, FK = size_t(h->n_focus) * h->k;
  return up256(N * C * sizeof(float2)) + up256(C * C * sizeof(float2)) + up256(FK * N * C * sizeof(float2));
}

// Device address of g_scratch on the current device, looked up on first use.
litho_status scratch_address(void** out) {
  int dev = 0;
  LITHO_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d beyond the %d devices litho_aerial_noalloc tracks", dev, kMaxDevices);
    return LITHO_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    LITHO_TRY_CUDA(cudaGetSymbolAddress(&p, g_scratch));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return LITHO_OK;
}

}  // namespace

}  // namespace litho

using namespace litho;

extern "C" {

size_t litho_aerial_noalloc_max_bytes(void) { return kScratchBytes; }

litho_status litho_aerial_noalloc(const litho_kernels* h, const float* mask_dev, int b, double dose,
                                  float* intensity_dev, void* stream) {
  if (!h || !mask_dev || !intensity_dev) {
    set_error("null argument");
    return LITHO_EINVAL;
  }
  if (b < 1) {
    set_error("b must be >= 1");
    return LITHO_EINVAL;
  }
  if (!std::isfinite(dose)) {
    set_error("dose must be finite");
    return LITHO_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(mask_dev) & 15) != 0 || (reinterpret_cast<uintptr_t>(intensity_dev) & 15) != 0) {
    set_error("mask and intensity must be 16-byte aligned");
    return LITHO_EINVAL;
  }
  // The kernel set's tables live on h->device and the scratch address is
  // looked up on the current device: both must be the same GPU.
  int cur = 0;
  LITHO_TRY_CUDA(cudaGetDevice(&cur));
  if (cur != h->device) {
    set_error("litho_aerial_noalloc: the current device is %d but the kernel set lives on device %d; make that "
              "device current first",
              cur, h->device);
    return LITHO_EINVAL;
  }
  const size_t need = clip_bytes(h);
  if (need > kScratchBytes) {
    set_error("litho_aerial_noalloc: this kernel set needs %zu bytes of scratch per clip (N=%d, crop=%d, "
              "%d focus planes x %d kernels) but the fixed scratch array holds %zu; use litho_aerial with a "
              "workspace instead",
              need, h->n, h->crop, h->n_focus, h->k, kScratchBytes);
    return LITHO_EINVAL;
  }
  void* base = nullptr;
  litho_status s = scratch_address(&base);
  if (s != LITHO_OK) return s;
  const size_t N = h->n, C = h->crop;
  const int F = h->n_focus, K = h->k;
  // Every byte of the three regions is written before it is read within each
  // clip, so nothing carries over from an earlier call and nothing is cleared.
  char* p = static_cast<char*>(base);
  float2* rowbuf = reinterpret_cast<float2*>(p);
  float2* mhat = reinterpret_cast<float2*>(p + up256(N * C * sizeof(float2)));
  float2* t1 = reinterpret_cast<float2*>(p + up256(N * C * sizeof(float2)) + up256(C * C * sizeof(float2)));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int clip = 0; clip < b; ++clip) {
    const float* m = mask_dev + size_t(clip) * N * N;
    float* img = intensity_dev + size_t(clip) * F * N * N;
    LITHO_TRY_CUDA(launch_mask_spectrum(m, 1, int(N), int(C), h->d_tw, rowbuf, mhat, st));
    LITHO_TRY_CUDA(launch_stage1_fft(mhat, h->d_phi, F * K, int(N), int(C), h->d_tw, t1, st));
    LITHO_TRY_CUDA(launch_stage2_fft(t1, h->d_lambda, K, int(N), int(C), float(dose), h->d_tw, img, F,
                                     (long long)K * N * C, (long long)N * N, st));
  }
  return LITHO_OK;
}

}  // extern "C"
