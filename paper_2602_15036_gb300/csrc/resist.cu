// Resist model (paper Eq. (5)): I_blur = g (x) I with a periodic, separable,
// normalised Gaussian g[j] ~ exp(-(j p)^2 / (2 s^2)), |j| <= R = ceil(4 s / p),
// then printed = [I_blur >= T] (ties print, as the ">=" of Eqs. (16)-(17)).
//
// One pass over HBM: each CTA loads a (32 + 2R) x (32 + 2R) tile with a
// periodic halo into shared memory, blurs rows into a second tile, blurs
// columns from it and writes I_blur (f32) and printed (u8) once.  For the
// common radii (R <= 12) the radius is a template parameter: the taps live in
// registers, the tap loops unroll and each thread blurs four consecutive
// column outputs from a register window; larger radii take a loop version.
#include <cmath>

#include "litho_internal.h"

namespace litho {

namespace {

constexpr int TX = 32, TY = 32, BY = 8, RPT = TY / BY;  // RPT: column outputs per thread

template <int R>  // R >= 0: compile-time radius; R < 0: taps.radius at run time
__global__ void __launch_bounds__(TX * BY) k_resist(const float* __restrict__ img, int n, ResistTaps taps, float thr,
                                                    float* __restrict__ iblur, uint8_t* __restrict__ printed) {
  extern __shared__ float sm[];
  const int r = R >= 0 ? R : taps.radius;
  const int hw = TX + 2 * r, hh = TY + 2 * r;
  float* tile = sm;            // [hh][hw]
  float* rows = sm + hh * hw;  // [hh][TX]
  const int plane = blockIdx.z, x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const float* src = img + (size_t)plane * n * n;
  const bool pow2 = (n & (n - 1)) == 0;
  for (int ty = threadIdx.y; ty < hh; ty += BY) {
    int gy = y0 + ty - r;
    gy = pow2 ? (gy & (n - 1)) : (gy + n) % n;
    const float* srow = src + (size_t)gy * n;
    for (int tx = threadIdx.x; tx < hw; tx += TX) {
      int gx = x0 + tx - r;
      gx = pow2 ? (gx & (n - 1)) : (gx + n) % n;
      tile[ty * hw + tx] = __ldg(srow + gx);
    }
  }
  __syncthreads();
  const int x = threadIdx.x;
  // rows[ty][x] = sum_a g[a] tile[ty][x + r - a]
  if constexpr (R >= 0) {
    float g[2 * R + 1];
#pragma unroll
    for (int a = 0; a <= 2 * R; ++a) g[a] = taps.g[a];
    for (int ty = threadIdx.y; ty < hh; ty += BY) {
      const float* t = tile + ty * hw + x + R;
      float acc = 0.f;
#pragma unroll
      for (int a = -R; a <= R; ++a) acc = fmaf(g[a + R], t[-a], acc);
      rows[ty * TX + x] = acc;
    }
    __syncthreads();
    const int yy = threadIdx.y * RPT;
    float win[RPT + 2 * R];
#pragma unroll
    for (int j = 0; j < RPT + 2 * R; ++j) win[j] = rows[(yy + j) * TX + x];
    float* dst = iblur + (size_t)plane * n * n;
    uint8_t* pr = printed ? printed + (size_t)plane * n * n : nullptr;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int a = -R; a <= R; ++a) acc = fmaf(g[a + R], win[i + R - a], acc);
      const size_t o = (size_t)(y0 + yy + i) * n + x0 + x;
      dst[o] = acc;
      if (pr) pr[o] = acc >= thr ? 1 : 0;
    }
  } else {
    for (int ty = threadIdx.y; ty < hh; ty += BY) {
      const float* t = tile + ty * hw + x + r;
      float acc = 0.f;
      for (int a = -r; a <= r; ++a) acc = fmaf(taps.g[a + r], t[-a], acc);
      rows[ty * TX + x] = acc;
    }
    __syncthreads();
    float* dst = iblur + (size_t)plane * n * n;
    uint8_t* pr = printed ? printed + (size_t)plane * n * n : nullptr;
    for (int yy = threadIdx.y; yy < TY; yy += BY) {
      const float* c = rows + (yy + r) * TX + x;
      float acc = 0.f;
      for (int a = -r; a <= r; ++a) acc = fmaf(taps.g[a + r], c[-a * TX], acc);
      const size_t o = (size_t)(y0 + yy) * n + x0 + x;
      dst[o] = acc;
      if (pr) pr[o] = acc >= thr ? 1 : 0;
    }
  }
}

template <int R>
cudaError_t launch_r(const float* img, int planes, int n, const ResistTaps& taps, float thr, float* iblur,
                     uint8_t* printed, cudaStream_t st) {
  const int r = taps.radius;
  const size_t sm = sizeof(float) * ((TY + 2 * r) * (TX + 2 * r) + (TY + 2 * r) * TX);
  cudaError_t e = cudaFuncSetAttribute(k_resist<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_resist<R><<<dim3(n / TX, n / TY, planes), dim3(TX, BY), sm, st>>>(img, n, taps, thr, iblur, printed);
  return cudaGetLastError();
}

}  // namespace

bool resist_taps(double sigma_nm, double pixel_nm, ResistTaps* t, std::string* why) {
  if (!(sigma_nm > 0.0) || !(pixel_nm > 0.0)) {
    *why = "sigma_nm and pixel_nm must be > 0";
    return false;
  }
  const int r = int(std::ceil(4.0 * sigma_nm / pixel_nm));
  if (r > kMaxResistRadius) {
    *why = "resist blur radius ceil(4 sigma / pixel) above 64 pixels";
    return false;
  }
  double g[2 * kMaxResistRadius + 1], sum = 0.0;
  for (int j = -r; j <= r; ++j) {
    g[j + r] = std::exp(-(j * pixel_nm) * (j * pixel_nm) / (2.0 * sigma_nm * sigma_nm));
    sum += g[j + r];
  }
  t->radius = r;
  for (int j = 0; j < 2 * r + 1; ++j) t->g[j] = float(g[j] / sum);
  return true;
}

cudaError_t launch_resist(const float* img, int planes, int n, const ResistTaps& taps, float threshold, float* iblur,
                          uint8_t* printed, cudaStream_t st) {
  if (n % TX != 0 || n % TY != 0 || 2 * taps.radius >= n) return cudaErrorInvalidValue;
  switch (taps.radius) {
#define R_CASE(R) \
  case R: return launch_r<R>(img, planes, n, taps, threshold, iblur, printed, st);
    R_CASE(1) R_CASE(2) R_CASE(3) R_CASE(4) R_CASE(5) R_CASE(6) R_CASE(7) R_CASE(8) R_CASE(9) R_CASE(10)
    R_CASE(11) R_CASE(12)
#undef R_CASE
    default: return launch_r<-1>(img, planes, n, taps, threshold, iblur, printed, st);
  }
}

}  // namespace litho
