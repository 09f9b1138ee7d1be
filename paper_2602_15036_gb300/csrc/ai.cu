// Input channels of the AI initialiser (paper Eq. (9)) and its
// lithography-consistency images (Eqs. (15)-(17)).
//
// Eq. (9), as read here: X[c] = (Z_t, I0 / max I0, (dI/dM - min) / (max - min))
// with I0 the aerial image of the target at one focus plane, dI/dM the
// gradient of the plane's total intensity with respect to the mask pixels
// (the adjoint of Eq. (4) applied to ones, as litho_intensity_vjp computes
// it; both channels come from one set of stage-1 fields, see ai_channels)
// and the extremes taken over the whole batch (a constant channel maps to 0).
// Eqs. (15)-(17): Z_round = [G (x) Z_t >= tau_round] with the resist's
// periodic Gaussian, Z_print = [I >= tau_print], L_litho = sum |Z_print -
// Z_round| per clip (an integer count, reduced in a fixed order).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "litho_internal.h"

namespace litho {

namespace {

constexpr int kReduceBlocks = 304, kReduceThreads = 256;

// Per-block minimum and maximum of channel `ch` of X[b][3][nn]: block
// (x, clip) scans its share of the clip's channel (16-byte loads when nn is a
// multiple of 4); partials [b][gridDim.x].
__global__ void __launch_bounds__(kReduceThreads) k_minmax(const float* __restrict__ x, int b, size_t nn, int ch,
                                                           float2* __restrict__ part) {
  __shared__ float smin[kReduceThreads], smax[kReduceThreads];
  float lo = FLT_MAX, hi = -FLT_MAX;
  const float* src = x + (size_t(blockIdx.y) * 3 + ch) * nn;
  const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  if (nn % 4 == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    for (size_t i = t0; i < nn / 4; i += stride) {
      const float4 v = s4[i];
      lo = fminf(lo, fminf(fminf(v.x, v.y), fminf(v.z, v.w)));
      hi = fmaxf(hi, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
    }
  } else {
    for (size_t i = t0; i < nn; i += stride) {
      lo = fminf(lo, src[i]);
      hi = fmaxf(hi, src[i]);
    }
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int o = kReduceThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + o]);
      smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[size_t(blockIdx.y) * gridDim.x + blockIdx.x] = make_float2(smin[0], smax[0]);
}

// Channel ch of every clip: v -> (v - lo) * s, with lo and s from the
// `nparts` block partials (mode 0: lo = 0, s = 1/max; mode 1: lo = min,
// s = 1/(max - min); s = 0 when the range is empty).  Block (x, clip).
__global__ void k_normalize(float* __restrict__ x, int b, size_t nn, int ch, const float2* __restrict__ part,
                            int nparts, int mode) {
  __shared__ float smin[kReduceThreads], smax[kReduceThreads];
  float lo = FLT_MAX, hi = -FLT_MAX;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
    lo = fminf(lo, part[k].x);
    hi = fmaxf(hi, part[k].y);
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int o = kReduceThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + o]);
      smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + o]);
    }
    __syncthreads();
  }
  lo = mode == 0 ? 0.f : smin[0];
  hi = smax[0];
  const float s = hi > lo ? 1.0f / (hi - lo) : 0.f;
  float* dst = x + (size_t(blockIdx.y) * 3 + ch) * nn;
  const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  if (nn % 4 == 0) {
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (size_t i = t0; i < nn / 4; i += stride) {
      float4 v = d4[i];
      v.x = (v.x - lo) * s;
      v.y = (v.y - lo) * s;
      v.z = (v.z - lo) * s;
      v.w = (v.w - lo) * s;
      d4[i] = v;
    }
  } else {
    for (size_t i = t0; i < nn; i += stride) dst[i] = (dst[i] - lo) * s;
  }
}

__global__ void k_copy_channel(const float* __restrict__ src, float* __restrict__ x, int b, size_t nn, int ch) {
  const size_t total = size_t(b) * nn;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    x[(i / nn) * 3 * nn + size_t(ch) * nn + i % nn] = src[i];
}

__global__ void k_threshold(const float* __restrict__ img, size_t count, float thr, uint8_t* __restrict__ z) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    z[i] = img[i] >= thr ? 1 : 0;
}

// Number of pixels where the two 0/1 prints differ, per clip (grid y): each
// block counts 16-byte pieces (the XOR of two 0/1 bytes is one bit) and adds
// its count to the clip's total with an integer atomic (exact, so the result
// does not depend on the order).  out must be zero on entry.
constexpr int kL1Blocks = 64;
__global__ void __launch_bounds__(kReduceThreads) k_l1_count(const uint4* __restrict__ a, const uint4* __restrict__ b,
                                                             size_t pieces, unsigned long long* __restrict__ out) {
  __shared__ unsigned long long s[kReduceThreads];
  const size_t base = size_t(blockIdx.y) * pieces;
  unsigned long long c = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < pieces; i += (size_t)gridDim.x * blockDim.x) {
    const uint4 x = a[base + i], y = b[base + i];
    c += __popc(x.x ^ y.x) + __popc(x.y ^ y.y) + __popc(x.z ^ y.z) + __popc(x.w ^ y.w);
  }
  s[threadIdx.x] = c;
  __syncthreads();
  for (int o = kReduceThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out + blockIdx.y, s[0]);
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

}  // namespace litho

using namespace litho;

extern "C" {

litho_status litho_ai_inputs_workspace_size(const litho_kernels* h, int b, size_t* bytes) {
  if (!h || !bytes || b < 1) {
    set_error("null argument or b < 1");
    return LITHO_EINVAL;
  }
  *bytes = up256(ai_channels_bytes(h, b)) + up256(size_t(std::max(kReduceBlocks, b)) * sizeof(float2));
  return LITHO_OK;
}

litho_status litho_ai_inputs(const litho_kernels* h, const float* target_dev, int b, double dose, int focus,
                             litho_precision prec, float* x_dev, void* workspace_dev, size_t workspace_bytes,
                             void* stream) {
  if (!h || !target_dev || !x_dev || !workspace_dev || b < 1 || b > 65535) {
    set_error("null argument or b outside [1, 65535]");
    return LITHO_EINVAL;
  }
  if (focus < 0 || focus >= h->n_focus || !std::isfinite(dose)) {
    set_error("focus must index a plane of the kernel set; dose finite");
    return LITHO_EINVAL;
  }
  if ((int(prec) & ~LITHO_GRID_COARSE) != LITHO_PREC_FFT32) {
    set_error("litho_ai_inputs implements the FP32 FFT path only (LITHO_PREC_FFT32, optionally | LITHO_GRID_COARSE)");
    return LITHO_EUNSUPPORTED;
  }
  size_t need = 0;
  litho_status s = litho_ai_inputs_workspace_size(h, b, &need);
  if (s != LITHO_OK) return s;
  if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace_dev) & 255) != 0) {
    set_error("workspace must be 256-byte aligned and hold %zu bytes (%zu given)", need, workspace_bytes);
    return workspace_bytes < need ? LITHO_ENOMEM : LITHO_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nn = size_t(h->n) * h->n;
  float2* part = reinterpret_cast<float2*>(static_cast<char*>(workspace_dev) + up256(ai_channels_bytes(h, b)));
  {
    ProfScope ps(kStageIltForward, st, 1);
    k_copy_channel<<<512, 256, 0, st>>>(target_dev, x_dev, b, nn, 0);
    LITHO_TRY_CUDA(cudaGetLastError());
  }
  s = ai_channels(h, target_dev, b, dose, focus, (int(prec) & LITHO_GRID_COARSE) != 0, x_dev, workspace_dev, st);
  if (s != LITHO_OK) return s;
  ProfScope ps(kStageIltReduce, st, 4);
  const int per_clip = std::max(1, kReduceBlocks / b);  // partials per clip: at most kReduceBlocks in all
  for (int ch = 1; ch <= 2; ++ch) {
    k_minmax<<<dim3(per_clip, b), kReduceThreads, 0, st>>>(x_dev, b, nn, ch, part);
    k_normalize<<<dim3(std::max(1, 1216 / b), b), kReduceThreads, 0, st>>>(x_dev, b, nn, ch, part, per_clip * b,
                                                                          ch == 1 ? 0 : 1);
  }
  LITHO_TRY_CUDA(cudaGetLastError());
  return LITHO_OK;
}

litho_status litho_print_images(const float* target_dev, const float* intensity_dev, int b, int n, double pixel_nm,
                                double sigma_round_nm, double tau_round, double tau_print, uint8_t* z_round_dev,
                                uint8_t* z_print_dev, int64_t* loss_dev, float* blur_dev, void* stream) {
  if (!target_dev || !intensity_dev || !z_round_dev || !z_print_dev || !blur_dev || b < 1 || n < 32 || n % 32) {
    set_error("null argument, b < 1, or n not a multiple of 32");
    return LITHO_EINVAL;
  }
  if (!std::isfinite(tau_round) || !std::isfinite(tau_print)) {
    set_error("thresholds must be finite");
    return LITHO_EINVAL;
  }
  if (((reinterpret_cast<uintptr_t>(z_round_dev) | reinterpret_cast<uintptr_t>(z_print_dev)) & 15) != 0) {
    set_error("z_round_dev and z_print_dev must be 16-byte aligned");
    return LITHO_EINVAL;
  }
  ResistTaps taps;
  std::string why;
  if (!resist_taps(sigma_round_nm, pixel_nm, &taps, &why)) {
    set_error("%s", why.c_str());
    return LITHO_EINVAL;
  }
  if (2 * taps.radius >= n) {
    set_error("blur radius must be below n/2");
    return LITHO_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nn = size_t(n) * n;
  ProfScope ps(kStageResist, st, loss_dev ? 3 : 2);
  LITHO_TRY_CUDA(launch_resist(target_dev, b, n, taps, float(tau_round), blur_dev, z_round_dev, st));
  k_threshold<<<1024, 256, 0, st>>>(intensity_dev, size_t(b) * nn, float(tau_print), z_print_dev);
  if (loss_dev) {
    LITHO_TRY_CUDA(cudaMemsetAsync(loss_dev, 0, size_t(b) * sizeof(int64_t), st));
    k_l1_count<<<dim3(kL1Blocks, b), kReduceThreads, 0, st>>>(
        reinterpret_cast<const uint4*>(z_print_dev), reinterpret_cast<const uint4*>(z_round_dev), nn / 16,
        reinterpret_cast<unsigned long long*>(loss_dev));
  }
  LITHO_TRY_CUDA(cudaGetLastError());
  return LITHO_OK;
}

}  // extern "C"
