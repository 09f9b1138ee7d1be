// Resist model (paper Eq. (5)): I_blur = g (x) I with a periodic, separable,
// normalised Gaussian g[j] ~ exp(-(j p)^2 / (2 s^2)), |j| <= R = ceil(4 s / p),
// then printed = [I_blur >= T] (ties print, as the ">=" of Eqs. (16)-(17)).
//
// One pass over HBM, by strips: a CTA takes 32 columns by SH rows (128 when
// n allows, else 32).  Its threads load the strip and its periodic halo into
// shared memory together, the warps blur its rows horizontally into a
// shared strip of SH + 2R rows; then each thread
// blurs its column over a register window of SH/8 + 2R rows and writes
// I_blur (f32) and printed (u8), a warp writing whole 128-byte rows.  Reads
// are 1 + 2R/32 horizontal and 1 + 2R/SH vertical per pixel (the halos of
// neighbouring strips, which run side by side, mostly hit L2).  For the
// common radii (R <= 12) the radius is a template parameter (taps in
// registers, unrolled loops); larger radii take a loop version.
#include <cmath>

#include "litho_internal.h"

namespace litho {

namespace {

constexpr int SW = 32, SWARPS = 8;  // strip width, warps per CTA

template <int R, int SH>  // R >= 0: compile-time radius; R < 0: taps.radius at run time
__global__ void __launch_bounds__(32 * SWARPS) k_resist(const float* __restrict__ img, int n, ResistTaps taps,
                                                        float thr, float* __restrict__ iblur,
                                                        uint8_t* __restrict__ printed) {
  constexpr int PER = SH / SWARPS;  // output rows per thread
  extern __shared__ float sm[];
  const int r = R >= 0 ? R : taps.radius;
  const int rows_in = SH + 2 * r, wi = SW + 2 * r;
  float* tile = sm;                 // [rows_in][wi] the strip and its periodic halo
  float* hb = sm + rows_in * wi;    // [rows_in][SW] horizontally blurred rows
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int plane = blockIdx.z, x0 = blockIdx.x * SW, y0 = blockIdx.y * SH;
  const float* src = img + (size_t)plane * n * n;
  const bool pow2 = (n & (n - 1)) == 0;
  float g[R >= 0 ? 2 * R + 1 : 1];
  if constexpr (R >= 0) {
#pragma unroll
    for (int a = 0; a <= 2 * R; ++a) g[a] = taps.g[a];
  }
  // all threads load the tile at once (consecutive threads, consecutive x)
  for (int i = threadIdx.x; i < rows_in * wi; i += blockDim.x) {
    const int ry = i / wi, rx = i - ry * wi;
    int gy = y0 + ry - r, gx = x0 + rx - r;
    gy = pow2 ? (gy & (n - 1)) : (gy + n) % n;
    gx = pow2 ? (gx & (n - 1)) : (gx + n) % n;
    tile[i] = __ldg(src + (size_t)gy * n + gx);
  }
  __syncthreads();
  // rows: hb[ry][x] = sum_a g[a] I[y0 + ry - r][x0 + x - a]
  for (int ry = warp; ry < rows_in; ry += SWARPS) {
    const float* t = tile + ry * wi + lane + r;
    float acc = 0.f;
    if constexpr (R >= 0) {
#pragma unroll
      for (int a = -R; a <= R; ++a) acc = fmaf(g[a + R], t[-a], acc);
    } else {
      for (int a = -r; a <= r; ++a) acc = fmaf(taps.g[a + r], t[-a], acc);
    }
    hb[ry * SW + lane] = acc;
  }
  __syncthreads();
  // columns: rows y0 + warp PER ... of column x0 + lane
  const int yy = warp * PER;
  float* dst = iblur + (size_t)plane * n * n;
  uint8_t* pr = printed ? printed + (size_t)plane * n * n : nullptr;
  if constexpr (R >= 0) {
    float win[PER + 2 * R];
#pragma unroll
    for (int j = 0; j < PER + 2 * R; ++j) win[j] = hb[(yy + j) * SW + lane];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int a = -R; a <= R; ++a) acc = fmaf(g[a + R], win[i + R - a], acc);
      const size_t o = (size_t)(y0 + yy + i) * n + x0 + lane;
      dst[o] = acc;
      if (pr) pr[o] = acc >= thr ? 1 : 0;
    }
  } else {
    for (int i = 0; i < PER; ++i) {
      const float* c = hb + (yy + i + r) * SW + lane;
      float acc = 0.f;
      for (int a = -r; a <= r; ++a) acc = fmaf(taps.g[a + r], c[-a * SW], acc);
      const size_t o = (size_t)(y0 + yy + i) * n + x0 + lane;
      dst[o] = acc;
      if (pr) pr[o] = acc >= thr ? 1 : 0;
    }
  }
}

template <int R, int SH>
cudaError_t launch_rs(const float* img, int planes, int n, const ResistTaps& taps, float thr, float* iblur,
                      uint8_t* printed, cudaStream_t st) {
  const int r = taps.radius;
  const size_t sm = sizeof(float) * ((SH + 2 * r) * (SW + 2 * r) + (SH + 2 * r) * SW);
  cudaError_t e = cudaFuncSetAttribute(k_resist<R, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_resist<R, SH><<<dim3(n / SW, n / SH, planes), 32 * SWARPS, sm, st>>>(img, n, taps, thr, iblur, printed);
  return cudaGetLastError();
}

template <int R>
cudaError_t launch_r(const float* img, int planes, int n, const ResistTaps& taps, float thr, float* iblur,
                     uint8_t* printed, cudaStream_t st) {
  return n % 128 == 0 ? launch_rs<R, 128>(img, planes, n, taps, thr, iblur, printed, st)
                      : launch_rs<R, 32>(img, planes, n, taps, thr, iblur, printed, st);
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
  if (n % SW != 0 || 2 * taps.radius >= n) return cudaErrorInvalidValue;
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
