// Stage 2 of the FP32 path for 1024-point rows, one warp per row, and for
// 512-point rows, two rows per warp (paper
// Eq. (4): I(y, x) = dose sum_k lam_k |sum_u T_k(y, u) e^{+2 pi i u x / N}|^2).
//
// The 1024-point inverse transform of a row is two radix-32 passes
// (1024 = 32 x 32, Stockham order, as in fft_common.cuh):
//   pass 1: lane l takes x[l + 32 r], r < 32, and forms their 32-point DFT in
//           registers; output q lands at position 32 l + q;
//   pass 2: lane l takes the values at l + 32 r, multiplies them by
//           w^(r l) (w = e^{+2 pi i / 1024}) and forms their 32-point DFT;
//           output q is the sample x = l + 32 q.
// The only exchange between the passes is one write and one read of the row
// through a padded shared-memory buffer (element i at i + i/32, so that both
// the write, lanes at stride 33, and the read, lanes consecutive, are free of
// bank conflicts).  The kernel loop runs inside the warp: each lane keeps
// lam_k |E_k|^2 of its 32 samples in registers across all kernels of the
// plane and writes them once, coalesced.  Compared with the three-pass
// block kernel this halves the shared-memory traffic per row, whose pipe was
// that kernel's bound.
//
// A row whose band occupies at most a quarter of the indices on each side
// (crop / 2 <= 256) takes the banded first pass: inputs r in [8, 24) are
// zero, neither loaded nor added.
//
// Each warp copies the next kernel's band row (crop complex values) into its
// staging buffer with 16-byte cp.async as soon as the current row has been
// read into registers, so the copy runs while the current row is
// transformed: the load latency is hidden without holding the values in
// registers (the 32-point transforms already take most of them).
#include <cmath>

#include "fft_common.cuh"
#include "litho_internal.h"

namespace litho {

namespace {

constexpr int kN = 1024, kR = 32;
constexpr int kRowLd = kN + kN / kR;  // padded row buffer of one warp

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory"); }

// SPEC: instead of the image row, its forward transform cropped to the c2
// frequencies |u| < c2/2 (index u + c2/2 of row y of plane p in `spec`, plane
// stride 1024 c2), as the first step of the exact Fourier interpolation:
// the row x = lane + 32 q is already where the four-step forward transform
// wants it (pass 1 over q, twiddle e^{-2 pi i lane u1 / 1024}, exchange,
// pass 2 over the lanes, output u1 + 32 u2 in lane u1).
template <bool BANDED, int kWarps, bool FOLDED, bool SPEC>
__global__ void __launch_bounds__(32 * kWarps, 1)
    k_stage2_w32(const float2* __restrict__ t1, const float* __restrict__ lam, int nk, int crop, float dose,
                 const float2* __restrict__ tw2_g, float* __restrict__ img, long long t1_plane, long long img_plane,
                 int lam_period, float2* __restrict__ spec, int c2) {
  extern __shared__ float4 smem_raw[];
  float2* tw2 = reinterpret_cast<float2*>(smem_raw);  // w^(r l) at (r - 1) 32 + l
  float2* rowbuf = tw2 + (kR - 1) * kR;                // [kWarps][kRowLd]
  float2* stage0 = rowbuf + kWarps * kRowLd;           // [kWarps][crop]
  for (int i = threadIdx.x; i < (kR - 1) * kR; i += blockDim.x) tw2[i] = tw2_g[i];
  __syncthreads();
  const int lane = threadIdx.x % 32, wp = threadIdx.x / 32;
  const int y = blockIdx.x * kWarps + wp, plane = blockIdx.y, half = crop / 2;
  if (y >= kN) return;  // no barrier below
  const float2* base = t1 + plane * t1_plane + (size_t)y * crop;
  const float* lp = lam + (plane % lam_period) * nk;
  float2* buf = rowbuf + wp * kRowLd;
  float2* stage = stage0 + (size_t)wp * crop;
  // band row of kernel j into the staging buffer: crop / 2 pieces of 16 bytes
  auto fetch = [&](int j) {
    const float2* src = base + (size_t)j * kN * crop;
    for (int i = lane; i < crop / 2; i += 32) cp_async16(stage + 2 * i, src + 2 * i);
    cp_async_commit();
  };
  float acc[kR];
#pragma unroll
  for (int q = 0; q < kR; ++q) acc[q] = 0.f;
  fetch(0);
  for (int j = 0; j < nk; ++j) {
    cp_async_wait<0>();
    __syncwarp();  // row j visible to every lane
    const float l = __ldg(lp + j);
    const float2* row = stage;
    float2 v[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      if (BANDED && r >= kR / 4 && r < 3 * kR / 4) {
        v[r] = make_float2(0.f, 0.f);  // not read by the banded network
      } else {
        const int idx = lane + kR * r;
        const int c = (r < kR / 2 ? idx : idx - kN) + half;  // crop column of frequency index idx
        v[r] = (c >= 0 && c < crop) ? row[c] : make_float2(0.f, 0.f);
      }
    }
    __syncwarp();  // every lane has read row j: the buffer takes row j + 1 during the transform
    if (j + 1 < nk) fetch(j + 1);
    if (l == 0.f) continue;  // a zero kernel (beyond the rank): uniform across the warp
    dft32<+1, BANDED>(v);
#pragma unroll
    for (int q = 0; q < kR; ++q) buf[lane * (kR + 1) + q] = v[q];  // position 32 lane + q, padded
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      v[r] = buf[lane + (kR + 1) * r];  // position lane + 32 r, padded
      if (r > 0) v[r] = cmul(v[r], tw2[(r - 1) * kR + lane]);
    }
    __syncwarp();  // every lane has read buf before the next kernel's pass 1 writes it
    dft32<+1, false>(v);
#pragma unroll
    for (int q = 0; q < kR; ++q)
      acc[q] = FOLDED ? fmaf(v[q].x, v[q].x, fmaf(v[q].y, v[q].y, acc[q]))  // sqrt(lam) is in the field
                      : fmaf(l, fmaf(v[q].x, v[q].x, v[q].y * v[q].y), acc[q]);
  }
  if constexpr (SPEC) {
    float2 v[kR];
#pragma unroll
    for (int q = 0; q < kR; ++q) v[q] = make_float2(dose * acc[q], 0.f);
    dft32<-1, false>(v);
#pragma unroll
    for (int u1 = 0; u1 < kR; ++u1) {
      float2 x = v[u1];
      if (u1 > 0) {
        const float2 w = tw2[(u1 - 1) * kR + lane];
        x = cmul(x, make_float2(w.x, -w.y));
      }
      buf[lane * (kR + 1) + u1] = x;  // position (u1, lane), padded
    }
    __syncwarp();
#pragma unroll
    for (int l = 0; l < kR; ++l) v[l] = buf[lane + (kR + 1) * l];
    dft32<-1, false>(v);
    float2* srow = spec + (size_t)plane * kN * c2 + (size_t)y * c2;
    const int h2 = c2 / 2;
#pragma unroll
    for (int u2 = 0; u2 < kR; ++u2) {
      const int u = lane + kR * u2, us = u < kN / 2 ? u : u - kN;
      if (us >= -h2 && us < h2) srow[us + h2] = v[u2];
    }
  } else {
    float* out = img + plane * img_plane + (size_t)y * kN;
#pragma unroll
    for (int q = 0; q < kR; ++q) out[lane + kR * q] = dose * acc[q];
  }
}

template <bool BANDED, int kWarps, bool FOLDED, bool SPEC>
cudaError_t launch_w32_k(const float2* t1, const float* lam, int nk, int crop, float dose, const float2* tw2,
                         float* img, int planes, long long t1_plane, long long img_plane, int lam_period,
                         cudaStream_t st, float2* spec, int c2) {
  const dim3 grid((kN + kWarps - 1) / kWarps, planes);
  const size_t sm = sizeof(float2) * ((kR - 1) * kR + kWarps * kRowLd + size_t(kWarps) * crop);
  cudaError_t e = smem_attrs(k_stage2_w32<BANDED, kWarps, FOLDED, SPEC>, sm);
  if (e != cudaSuccess) return e;
  k_stage2_w32<BANDED, kWarps, FOLDED, SPEC><<<grid, 32 * kWarps, sm, st>>>(t1, lam, nk, crop, dose, tw2, img,
                                                                            t1_plane, img_plane, lam_period, spec, c2);
  return cudaGetLastError();
}

template <int kWarps>
cudaError_t launch_w32_t(const float2* t1, const float* lam, int nk, int crop, float dose, const float2* tw2,
                         float* img, int planes, long long t1_plane, long long img_plane, int lam_period,
                         cudaStream_t st, bool folded, float2* spec, int c2) {
  const bool banded = crop / 2 <= kN / 4;  // the band leaves indices [N/4, 3N/4) empty
#define W32(B, F, S) \
  launch_w32_k<B, kWarps, F, S>(t1, lam, nk, crop, dose, tw2, img, planes, t1_plane, img_plane, lam_period, st, spec, c2)
  if (spec) {
    if (banded) return folded ? W32(true, true, true) : W32(true, false, true);
    return folded ? W32(false, true, true) : W32(false, false, true);
  }
  if (banded) return folded ? W32(true, true, false) : W32(true, false, false);
  return folded ? W32(false, true, false) : W32(false, false, false);
#undef W32
}

// The same stage 2 for 512-point rows, two rows per warp (512 = 16 x 32):
// lane l takes x[l + 32 r] of both rows for the first (radix-16) pass; in the
// second (radix-32) pass lanes 0-15 take row A and lanes 16-31 row B, lane j
// applying w^(r j) to positions j + 16 r and forming the 32-point DFT whose
// output q is the sample x = j + 16 q.  One padded exchange (i + i/16) per
// row and kernel; lam |E|^2 accumulates in registers.  The second-pass
// twiddles are the first 31 x 16 entries of the kernel set's 512-point
// table (w^(r j), r in [1, 32), j in [0, 16)).
constexpr int kW512Warps = 8, kW512Buf = 512 + 32;

template <bool BANDED>
__global__ void __launch_bounds__(32 * kW512Warps, 2)
    k_stage2_w512(const float2* __restrict__ t1, const float* __restrict__ lam, int nk, int crop, float dose,
                  const float2* __restrict__ tw_g, float* __restrict__ img, long long t1_plane, long long img_plane,
                  int lam_period) {
  constexpr int N = 512;
  extern __shared__ float4 smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);  // (r - 1) 16 + j
  float2* bufs = tw + 31 * 16;                        // [warp][2 rows][kW512Buf]
  float2* stage0 = bufs + kW512Warps * 2 * kW512Buf;  // [warp][2 rows][crop]
  for (int i = threadIdx.x; i < 31 * 16; i += blockDim.x) tw[i] = tw_g[i];
  __syncthreads();
  const int lane = threadIdx.x % 32, wp = threadIdx.x / 32, half = crop / 2;
  const int y0 = (blockIdx.x * kW512Warps + wp) * 2, plane = blockIdx.y;
  if (y0 >= N) return;  // no block barrier below
  float2* buf = bufs + wp * 2 * kW512Buf;
  float2* stage = stage0 + (size_t)wp * 2 * crop;
  const float* lp = lam + (plane % lam_period) * nk;
  const float2* base = t1 + plane * t1_plane + (size_t)y0 * crop;
  const int rsel = lane / 16, jj = lane % 16;
  auto fetch = [&](int k) {  // band rows y0, y0 + 1 of kernel k
    const float2* src = base + (size_t)k * N * crop;
    for (int i = lane; i < crop; i += 32) cp_async16(stage + 2 * i, src + 2 * i);
    cp_async_commit();
  };
  float acc[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) acc[q] = 0.f;
  fetch(0);
  for (int k = 0; k < nk; ++k) {
    cp_async_wait<0>();
    __syncwarp();
    float2 a[2][16];
#pragma unroll
    for (int row = 0; row < 2; ++row) {
      const float2* band = stage + row * crop;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if (BANDED && r >= 4 && r < 12) {
          a[row][r] = make_float2(0.f, 0.f);
        } else {
          const int idx = lane + 32 * r;
          const int c = (r < 8 ? idx : idx - N) + half;
          a[row][r] = (c >= 0 && c < crop) ? band[c] : make_float2(0.f, 0.f);
        }
      }
    }
    __syncwarp();  // both rows are in registers: the staging buffer takes kernel k + 1
    if (k + 1 < nk) fetch(k + 1);
    const float l = __ldg(lp + k);
    if (l == 0.f) continue;  // a zero kernel (beyond the rank): uniform across the warp
#pragma unroll
    for (int row = 0; row < 2; ++row) {
      dft_reg<16, +1, BANDED>(a[row]);
#pragma unroll
      for (int q = 0; q < 16; ++q) buf[row * kW512Buf + pad16(16 * lane + q)] = a[row][q];
    }
    __syncwarp();
    float2 v[32];
    const float2* rb = buf + rsel * kW512Buf;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      v[r] = rb[pad16(jj + 16 * r)];
      if (r > 0) v[r] = cmul(v[r], tw[(r - 1) * 16 + jj]);
    }
    __syncwarp();  // the row buffers are free for the next kernel
    dft32<+1, false>(v);
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = fmaf(l, fmaf(v[q].x, v[q].x, v[q].y * v[q].y), acc[q]);
  }
  float* out = img + plane * img_plane + (size_t)(y0 + rsel) * N;
#pragma unroll
  for (int q = 0; q < 32; ++q) out[jj + 16 * q] = dose * acc[q];
}

}  // namespace

// crop: even (16-byte row pieces) and at most 512 (staging buffers within shared memory)
bool stage2_w32_supported(int n, int crop) { return n == kN && crop >= 2 && crop <= kN / 2 && crop % 2 == 0; }

void stage2_w32_table(float2* out) {
  for (int r = 1; r < kR; ++r)
    for (int l = 0; l < kR; ++l) {
      const double a = 2.0 * 3.14159265358979323846 * double(r * l) / double(kN);
      out[(r - 1) * kR + l] = make_float2(float(std::cos(a)), float(std::sin(a)));
    }
}

bool stage2_w512_supported(int n, int crop) { return n == 512 && crop >= 2 && crop <= 256 && crop % 2 == 0; }

cudaError_t launch_stage2_w512(const float2* t1, const float* lam, int nk, int n, int crop, float dose,
                               const float2* tw512, float* img, int planes, long long t1_plane, long long img_plane,
                               int lam_period, cudaStream_t st) {
  if (!stage2_w512_supported(n, crop) || !tw512) return cudaErrorInvalidValue;
  if (lam_period <= 0) lam_period = planes;
  const dim3 grid(512 / (2 * kW512Warps), planes);
  const size_t sm = sizeof(float2) * (31 * 16 + kW512Warps * 2 * (size_t(kW512Buf) + crop));
  if (crop / 2 <= 128) {  // the band leaves indices [N/4, 3N/4) empty
    cudaError_t e = smem_attrs(k_stage2_w512<true>, sm);
    if (e != cudaSuccess) return e;
    k_stage2_w512<true><<<grid, 32 * kW512Warps, sm, st>>>(t1, lam, nk, crop, dose, tw512, img, t1_plane, img_plane,
                                                           lam_period);
  } else {
    cudaError_t e = smem_attrs(k_stage2_w512<false>, sm);
    if (e != cudaSuccess) return e;
    k_stage2_w512<false><<<grid, 32 * kW512Warps, sm, st>>>(t1, lam, nk, crop, dose, tw512, img, t1_plane,
                                                            img_plane, lam_period);
  }
  return cudaGetLastError();
}

cudaError_t launch_stage2_w32(const float2* t1, const float* lam, int nk, int n, int crop, float dose,
                              const float2* tw2, float* img, int planes, long long t1_plane, long long img_plane,
                              int lam_period, cudaStream_t st, bool folded, float2* spec, int c2) {
  if (!stage2_w32_supported(n, crop) || !tw2) return cudaErrorInvalidValue;
  if (spec && (c2 < 2 || c2 > kN || c2 % 2 != 0)) return cudaErrorInvalidValue;
  if (lam_period <= 0) lam_period = planes;
  // 12 warps per CTA: one CTA of 384 threads fits the SM's registers (about 160 per thread);
  // measured on the 2048^2 workload's 1024-point rows: 5.90 ms per step against 6.29 with 8
  // warps and 6.04 with 16 (128 registers)
  return launch_w32_t<12>(t1, lam, nk, crop, dose, tw2, img, planes, t1_plane, img_plane, lam_period, st, folded,
                          spec, c2);
}

}  // namespace litho
