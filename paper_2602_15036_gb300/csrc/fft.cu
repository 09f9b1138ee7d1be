// FFT-based kernels: mask spectrum (crop), stage 1 (band multiply + inverse
// transform over v), and stage 2 of the FP32 path (inverse transform over u
// fused with the lam_k |E_k|^2 accumulation over all kernels).
//
// Paper Section III.A: the object spectrum O(f) of Eq. (1) (thin-mask reading:
// the mask's DFT), and the SOCS image of Eq. (4), I = sum_k lam_k |O (x) phi_k|^2,
// evaluated as E_k = IDFT(M . Phi_k) restricted to the C x C band crop.
//
// Data layout (all row-major, x fastest):
//   mask    [b][N][N] f32
//   rowbuf  [b][N][C] c64   row DFT of the mask, crop columns only
//   mhat    [b][C][C] c64   N^-2 DFT(m) on the crop, [v][u]
//   t1      [j][N][C] c64   stage-1 field T_j[y][u] = sum_v mhat[v][u] Phi_j[v][u] e^{2 pi i v y/N}
//   img     [plane][N][N] f32
#include <algorithm>

#include "fft_common.cuh"
#include "litho_internal.h"
#include "stage1.cuh"

namespace litho {

namespace {

__device__ __forceinline__ int freq_of(int idx, int n) { return idx < n / 2 ? idx : idx - n; }

// ---- mask spectrum, pass 1: two real rows per complex transform ----------------------------
// z = m[y0] + i m[y1]; Z = DFT(z); X(u) = (Z(u) + conj Z(-u))/2, Y(u) = (Z(u) - conj Z(-u))/(2i).
template <int N>
__global__ void __launch_bounds__(Plan<N>::NT) k_mask_rows(const float* __restrict__ m, int crop,
                                                            const float2* __restrict__ tw_g,
                                                            float2* __restrict__ rowbuf, int pairs_per_cta) {
  extern __shared__ float2 smem[];
  float2* tw = smem;
  float2* buf = smem + N;
  float2* zc = smem + N + PadLen<N>::value;  // Z(u) for u in [-C/2, C/2], index u + C/2 (crop + 1 <= N + 1 entries)
  load_twiddles<N>(tw, tw_g);
  __syncthreads();
  const int b = blockIdx.y, t = threadIdx.x, half = crop / 2;
  constexpr int R0 = Plan<N>::R[0], NB0 = N / R0;
  static_assert(PassShape<N, Plan<N>::NT, R0>::PER == 1, "one first-pass butterfly per thread");
  // this thread's first-pass inputs (columns t + r N/R0 of both rows) of a pair, loaded one pair ahead
  float2 nxt[R0];
  auto prefetch = [&](int pr) {
    const float* r0 = m + ((size_t)b * N + 2 * pr) * N;
#pragma unroll
    for (int r = 0; r < R0; ++r)
      nxt[r] = t < NB0 ? make_float2(__ldg(r0 + t + r * NB0), __ldg(r0 + N + t + r * NB0)) : make_float2(0.f, 0.f);
  };
  const int pr0 = blockIdx.x * pairs_per_cta, pr1 = min(N / 2, (blockIdx.x + 1) * pairs_per_cta);
  if (pr0 < pr1) prefetch(pr0);
  // pairs [pr0, pr1): the next pair's first pass writes buf only after a
  // barrier that follows this pair's reads of zc
  for (int pr = pr0; pr < pr1; ++pr) {
    const int y0 = 2 * pr;
    float2 cur[R0];
#pragma unroll
    for (int r = 0; r < R0; ++r) cur[r] = nxt[r];
    auto load = [&](int, int r, int) { return cur[r]; };
    auto use = [&](int, int, int idx, float2 v) {
      const int u = freq_of(idx, N);
      if (u >= -half && u <= half) zc[u + half] = v;
      if (u == -N / 2 && half == N / 2) zc[crop] = v;  // crop == N: Z(N/2) is Z(-N/2)
    };
    // once the first pass has consumed this pair, the next pair's loads go out
    auto after_first = [&]() {
      if (pr + 1 < pr1) prefetch(pr + 1);
    };
    fft_load_use<N, -1, decltype(load), decltype(use), false>(buf, tw, t, load, use, after_first);
    __syncthreads();
    float2* o0 = rowbuf + ((size_t)b * N + y0) * crop;
    float2* o1 = o0 + crop;
    for (int c = t; c < crop; c += blockDim.x) {
      const float2 zp = zc[c], zm = zc[crop - c];
      o0[c] = make_float2(0.5f * (zp.x + zm.x), 0.5f * (zp.y - zm.y));
      o1[c] = make_float2(0.5f * (zp.y + zm.y), -0.5f * (zp.x - zm.x));
    }
  }
}


// ---- mask spectrum, pass 2: column DFTs of the crop columns, crop rows kept ------------------
// With `gain` (per crop index, real and even in the frequency), the stored
// value is S (1 + i gain[v] gain[u]): an image whose spectrum is S comes out
// of the inverse transform as I + i (g (x) I) for the separable filter with
// transfer function gain (x) gain, because both I and g (x) I are real.
template <int N>
__global__ void __launch_bounds__(Plan<N>::NT * ColW<N>::W) k_mask_cols(const float2* __restrict__ rowbuf, int crop,
                                                                         const float2* __restrict__ tw_g,
                                                                         const float* __restrict__ gain,
                                                                         float2* __restrict__ mhat, int gain_real) {
  constexpr int W = ColW<N>::W, NT = Plan<N>::NT, LD = ColLD<N>::value;
  extern __shared__ float2 smem[];
  float2* tw = smem;
  float2* buf = smem + N;
  load_twiddles<N>(tw, tw_g);
  const int b = blockIdx.y, u0 = blockIdx.x * W, tid = threadIdx.x;
  const float2* src = rowbuf + (size_t)b * N * crop + u0;
  for (int i = tid; i < N * W; i += blockDim.x) {
    const int y = i / W, w = i % W;
    buf[w * LD + pad16(y)] = src[(size_t)y * crop + w];
  }
  __syncthreads();
  fft_smem<N, -1>(buf + (tid / NT) * LD, tw, tid % NT);
  const float scale = 1.0f / (float(N) * float(N));
  float2* dst = mhat + (size_t)b * crop * crop + u0;
  const int half = crop / 2;
  for (int i = tid; i < crop * W; i += blockDim.x) {
    const int cv = i / W, w = i % W;
    const int idx = (cv - half + N) % N;
    float2 v = buf[w * LD + pad16(idx)];
    v = make_float2(v.x * scale, v.y * scale);
    if (gain) {
      const float g = __ldg(gain + cv) * __ldg(gain + u0 + w);
      v = gain_real ? make_float2(g * v.x, g * v.y)  // the blurred plane's spectrum
                    : make_float2(fmaf(-g, v.y, v.x), fmaf(g, v.x, v.y));  // the plane + i its blur
    }
    dst[(size_t)cv * crop + w] = v;
  }
}

// Transfer function of the periodic separable blur on an n-point grid:
// gain[i] = sum_a g[a] cos(2 pi f a / n) for the crop frequency f = i - crop/2
// (the taps are even, so the transform is real).  The angle is reduced
// exactly in integers before cospi.
__global__ void k_blur_gain(ResistTaps taps, int n, int crop, float* __restrict__ gain) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= crop) return;
  const int f = i - crop / 2, r = taps.radius;
  float acc = taps.g[r];
  for (int a = 1; a <= r; ++a) {
    const long long e = ((long long)f * a % n + n) % n;  // f a mod n, in [0, n)
    acc = fmaf(2.0f * taps.g[r + a], cospif(2.0f * float(e) / float(n)), acc);
  }
  gain[i] = acc;
}

// ---- stage 1: band multiply + inverse transform over v (stage1.cuh), FP32 output ------------------
struct OutC64 {
  static constexpr bool kRowWise = false;
  float2* t1;
  int n, crop;
  __device__ __forceinline__ float2* column(int j, int c) const { return t1 + (size_t)j * n * crop + c; }
  template <int W>
  __device__ void store_row(int, int, int, const float2 (&)[W]) const {}
};

// ---- stage 2 (FP32 path): one image row per CTA, all kernels of the plane ------------------------
template <int N, bool BANDED>
__global__ void __launch_bounds__(Plan<N>::NT, 512 / Plan<N>::NT) k_stage2(const float2* __restrict__ t1, const float* __restrict__ lam,
                                                        int nk, int crop, float dose,
                                                        const float2* __restrict__ tw_g, float* __restrict__ img,
                                                        long long t1_plane, long long img_plane, int lam_period) {
  using PL = Plan<N>;
  constexpr int NT = PL::NT;
  constexpr int RL = PL::R[PL::P - 1];
  constexpr int PERL = PassShape<N, NT, RL>::PER;
  __shared__ float2 buf[PadLen<N>::value];
  __shared__ float2 tw[N];
  load_twiddles<N>(tw, tw_g);
  __syncthreads();
  const int y = blockIdx.x, plane = blockIdx.y, t = threadIdx.x, half = crop / 2;
  const float2* base = t1 + plane * t1_plane + (size_t)y * crop;
  const float* lp = lam + (plane % lam_period) * nk;  // planes repeat every lam_period (clips of a batch)
  float acc[PERL][RL];
#pragma unroll
  for (int p = 0; p < PERL; ++p)
#pragma unroll
    for (int q = 0; q < RL; ++q) acc[p][q] = 0.f;
  // middle-pass twiddles in registers: measured faster for 2048-point rows,
  // slower for 1024 (where the registers they take cost more than the
  // shared-memory reads they save)
  constexpr bool kMid = MidTwiddles<N, +1>::kUsable && N >= 2048;
  MidTwiddles<N, +1> mid;
  if constexpr (kMid) mid.load(tw, t);
  for (int j = 0; j < nk; ++j) {
    const float l = __ldg(lp + j);
    if (l == 0.f) continue;  // uniform across the block
    const float2* row = base + (size_t)j * N * crop;
    auto load = [&](int, int r, int idx) {
      const int c = (r < PL::R[0] / 2 ? idx : idx - N) + half;  // first pass: idx < N/2 exactly when r < R/2
      return (c >= 0 && c < crop) ? __ldg(row + c) : make_float2(0.f, 0.f);
    };
    auto use = [&](int p, int q, int, float2 v) { acc[p][q] = fmaf(l, fmaf(v.x, v.x, v.y * v.y), acc[p][q]); };
    if constexpr (kMid)
      fft_load_use_mid<N, +1, decltype(load), decltype(use), BANDED>(buf, tw, t, load, use, mid);
    else
      fft_load_use<N, +1, decltype(load), decltype(use), BANDED>(buf, tw, t, load, use);
  }
  float* out = img + plane * img_plane + (size_t)y * N;
#pragma unroll
  for (int p = 0; p < PERL; ++p) {
    const int jj = t + p * NT;
    if (jj < N / RL) {
#pragma unroll
      for (int q = 0; q < RL; ++q) out[jj + q * (N / RL)] = dose * acc[p][q];
    }
  }
}

// ---- band rows to real image rows: out[p][y][x] = scale Re(sum_c q[p][y][c] e^{2 pi i u_c x/N}) ----------
// Second half of the exact Fourier interpolation from the coarse grid.
template <int N, bool BANDED>
__global__ void __launch_bounds__(Plan<N>::NT) k_band_rows_real(const float2* __restrict__ q, int crop, float scale,
                                                                const float2* __restrict__ tw_g,
                                                                float* __restrict__ out, int rows_per_cta) {
  __shared__ float2 buf[PadLen<N>::value];
  __shared__ float2 tw[N];
  load_twiddles<N>(tw, tw_g);
  __syncthreads();
  const int p = blockIdx.y, half = crop / 2;
  for (int y = blockIdx.x * rows_per_cta; y < min(N, (blockIdx.x + 1) * rows_per_cta); ++y) {
    const float2* row = q + ((size_t)p * N + y) * crop;
    auto load = [&](int, int r, int idx) {
      const int c = (r < Plan<N>::R[0] / 2 ? idx : idx - N) + half;  // first pass: idx < N/2 exactly when r < R/2
      return (c >= 0 && c < crop) ? __ldg(row + c) : make_float2(0.f, 0.f);
    };
    float* o = out + ((size_t)p * N + y) * N;
    auto use = [&](int, int, int x, float2 v) { o[x] = scale * v.x; };
    fft_load_use<N, +1, decltype(load), decltype(use), BANDED>(buf, tw, threadIdx.x, load, use);
  }
}

// Same transform for band rows carrying S (1 + i gain (x) gain) (see
// k_mask_cols): the real part is the image, the imaginary part its blur, and
// printed = [blur >= threshold].  `img` may be NULL (not written).
template <int N, bool BANDED>
__global__ void __launch_bounds__(Plan<N>::NT) k_band_rows_resist(const float2* __restrict__ q, int crop,
                                                                  const float2* __restrict__ tw_g, float thr,
                                                                  float* __restrict__ img, float* __restrict__ iblur,
                                                                  uint8_t* __restrict__ printed, int rows_per_cta) {
  __shared__ float2 buf[PadLen<N>::value];
  __shared__ float2 tw[N];
  load_twiddles<N>(tw, tw_g);
  __syncthreads();
  const int p = blockIdx.y, half = crop / 2;
  for (int y = blockIdx.x * rows_per_cta; y < min(N, (blockIdx.x + 1) * rows_per_cta); ++y) {
    const float2* row = q + ((size_t)p * N + y) * crop;
    auto load = [&](int, int r, int idx) {
      const int c = (r < Plan<N>::R[0] / 2 ? idx : idx - N) + half;  // first pass: idx < N/2 exactly when r < R/2
      return (c >= 0 && c < crop) ? __ldg(row + c) : make_float2(0.f, 0.f);
    };
    const size_t o = ((size_t)p * N + y) * N;
    auto use = [&](int, int, int x, float2 v) {
      if (img) img[o + x] = v.x;
      iblur[o + x] = v.y;
      if (printed) printed[o + x] = v.y >= thr ? 1 : 0;
    };
    fft_load_use<N, +1, decltype(load), decltype(use), BANDED>(buf, tw, threadIdx.x, load, use);
  }
}

// ILT forward end on the coarse grid, for a pair of rows (y0, y0 + 1) of a
// full-grid plane whose band rows R_y carry S (1 + i gain (x) gain), so that
// the imaginary part of IDFT(R_y) is the blurred row.  The blurred row's
// spectrum is (R_y(u) - conj R_y(-u)) / 2i, so one inverse transform of
// Bl_y0 + i Bl_y1 gives both blurred rows as its real and imaginary parts.
// The sigmoid resist z = 1 / (1 + e^{-beta (blur - thr)}) (a smooth Eq. (5)),
// the residual d = z - target of the squared-residual ILT loss and
// dL/dI = 2 d beta z (1 - z) follow on the spot; the two dL/dI rows go forward as one complex row
// q[y0] + i q[y1] and leave as their two band spectra, as k_mask_rows writes
// them.  The pair's sum of d^2 goes to partial[plane][pair] in FP64: one
// partial per row pair, whatever the launch shape, so the loss does not
// depend on how clips are grouped.  Plane p belongs to clip
// p / planes_per_clip of `target`.
template <int N>
struct GradRowsShape {
  using PL = Plan<N>;
  static constexpr int NT = PL::NT, R0 = PL::R[0], RL = PL::R[PL::P - 1];
  static constexpr int PERL = (N / RL + NT - 1) / NT;
  // the inverse transform's last pass hands thread t the elements t + NT r,
  // r = p + PERL q, which are the forward first pass's inputs of thread t
  static constexpr bool kRegs = N / R0 == NT && N / RL == PERL * NT && R0 == PERL * RL;
};

template <int N, bool BANDED>
__global__ void __launch_bounds__(Plan<N>::NT, N >= 512 ? 640 / Plan<N>::NT : 1) k_resist_grad_rows(const float2* __restrict__ band, int crop,
                                                                   const float2* __restrict__ tw_g,
                                                                   const float* __restrict__ target,
                                                                   int planes_per_clip, float beta, float thr,
                                                                   float2* __restrict__ rowbuf,
                                                                   double* __restrict__ partial, int pairs_per_cta) {
  using SH = GradRowsShape<N>;
  constexpr int NT = SH::NT, NW = (NT + 31) / 32, PERL = SH::PERL;
  extern __shared__ float2 smem[];
  float2* tw = smem;
  float2* buf = smem + N;
  // Z(u) on the crop, index u + C/2 (crop + 1 entries); without kRegs, first
  // the pair's dL/dI rows (N entries: x row y0, y row y0 + 1)
  float2* zq = smem + N + PadLen<N>::value;
  __shared__ double wsum[NW];
  load_twiddles<N>(tw, tw_g);
  __syncthreads();
  const int p = blockIdx.y, t = threadIdx.x, half = crop / 2;
  const float* tg = target + (size_t)(p / planes_per_clip) * N * N;
  for (int pr = blockIdx.x * pairs_per_cta; pr < min(N / 2, (blockIdx.x + 1) * pairs_per_cta); ++pr) {
    const int y0 = 2 * pr;
    const float2* r0 = band + ((size_t)p * N + y0) * crop;
    const float2* r1 = r0 + crop;
    const float* t0 = tg + (size_t)y0 * N;
    const float* t1 = t0 + N;
    auto load = [&](int, int r, int idx) {
      const int u = r < Plan<N>::R[0] / 2 ? idx : idx - N;  // first pass: idx < N/2 exactly when r < R/2
      const int c = u + half, cm = half - u;
      const bool in = c >= 0 && c < crop, inm = cm >= 0 && cm < crop;
      const float2 a = in ? __ldg(r0 + c) : make_float2(0.f, 0.f), b = inm ? __ldg(r0 + cm) : make_float2(0.f, 0.f);
      const float2 e = in ? __ldg(r1 + c) : make_float2(0.f, 0.f), f = inm ? __ldg(r1 + cm) : make_float2(0.f, 0.f);
      // Bl0 + i Bl1 = ((R1(u) - conj R1(-u)) - i (R0(u) - conj R0(-u))) / 2
      return make_float2(0.5f * (e.x - f.x + a.y + b.y), 0.5f * (e.y + f.y + b.x - a.x));
    };
    float racc = 0.f;  // this thread's residuals of the pair, summed in FP32 before the FP64 sum
    float2 qreg[SH::kRegs ? SH::R0 : 1];
    auto use = [&](int pp, int qq, int x, float2 v) {
      const float z0 = 1.0f / (1.0f + expf(-beta * (v.x - thr)));
      const float z1 = 1.0f / (1.0f + expf(-beta * (v.y - thr)));
      const float d0 = z0 - __ldg(t0 + x), d1 = z1 - __ldg(t1 + x);
      racc = fmaf(d0, d0, fmaf(d1, d1, racc));
      const float2 q = make_float2(2.0f * d0 * beta * z0 * (1.0f - z0), 2.0f * d1 * beta * z1 * (1.0f - z1));
      if constexpr (SH::kRegs)
        qreg[pp + PERL * qq] = q;
      else
        zq[x] = q;
    };
    fft_load_use<N, +1, decltype(load), decltype(use), BANDED>(buf, tw, t, load, use);
    double acc = double(racc);
    auto usez = [&](int, int, int idx, float2 v) {
      const int u = freq_of(idx, N);
      if (u >= -half && u <= half) zq[u + half] = v;
      if (u == -N / 2 && half == N / 2) zq[crop] = v;  // crop == N: Z(N/2) is Z(-N/2)
    };
    if constexpr (SH::kRegs) {
      auto loadq = [&](int, int r, int) { return qreg[r]; };
      fft_load_use<N, -1, decltype(loadq), decltype(usez), false>(buf, tw, t, loadq, usez);
    } else {
      __syncthreads();  // both dL/dI rows in zq
      auto loadz = [&](int, int, int idx) { return zq[idx]; };
      fft_load_use<N, -1, decltype(loadz), decltype(usez), false>(buf, tw, t, loadz, usez);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (t % 32 == 0) wsum[t / 32] = acc;
    __syncthreads();  // Z on the crop and the warps' sums
    if (t == 0) {
      double sum = 0.0;
      for (int w = 0; w < NW; ++w) sum += wsum[w];
      partial[(size_t)p * (N / 2) + pr] = sum;
    }
    float2* o0 = rowbuf + ((size_t)p * N + y0) * crop;
    float2* o1 = o0 + crop;
    for (int c = t; c < crop; c += NT) {
      const float2 zp = zq[c], zm = zq[crop - c];
      o0[c] = make_float2(0.5f * (zp.x + zm.x), 0.5f * (zp.y - zm.y));
      o1[c] = make_float2(0.5f * (zp.y + zm.y), -0.5f * (zp.x - zm.x));
    }
  }
}

// Rows per CTA for the one-row-per-transform kernels: enough CTAs for about
// eight waves of `per_sm` CTAs per SM, each CTA reusing its twiddle table
// for its rows.
inline int rows_per_cta(int rows, int planes, int per_sm) {
  static int sms = 0;  // the same GPU model throughout a process
  if (!sms) {
    int dev = 0, v = 0;
    sms = cudaGetDevice(&dev) == cudaSuccess &&
                  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0
              ? v
              : 152;
  }
  const long long want = 8LL * sms * per_sm;
  const long long r = std::max<long long>(1, ((long long)rows * planes) / want);
  return int(std::min<long long>(r, rows));
}

template <int N>
cudaError_t band_rows_resist_n(const float2* q, int planes, int crop, const float2* tw, float thr, float* img,
                               float* iblur, uint8_t* printed, cudaStream_t st) {
  const int rpc = rows_per_cta(N, planes, 2048 / Plan<N>::NT), grid = (N + rpc - 1) / rpc;
  if (2 * crop <= N)
    k_band_rows_resist<N, true><<<dim3(grid, planes), Plan<N>::NT, 0, st>>>(q, crop, tw, thr, img, iblur, printed,
                                                                           rpc);
  else
    k_band_rows_resist<N, false><<<dim3(grid, planes), Plan<N>::NT, 0, st>>>(q, crop, tw, thr, img, iblur, printed,
                                                                            rpc);
  return cudaGetLastError();
}

template <int N>
cudaError_t resist_grad_rows_n(const float2* band, int planes, int crop, const float2* tw, const float* target,
                               int planes_per_clip, float beta, float thr, float2* rowbuf, double* partial,
                               cudaStream_t st) {
  static_assert(Plan<N>::NT % 32 == 0, "whole warps");
  const size_t sm = sizeof(float2) * (N + PadLen<N>::value + (GradRowsShape<N>::kRegs ? crop + 1 : N + 1));
  const int ppc = rows_per_cta(N / 2, planes, 2048 / Plan<N>::NT), grid = (N / 2 + ppc - 1) / ppc;
  cudaError_t e;
  if (2 * crop <= N) {
    if ((e = smem_attrs(k_resist_grad_rows<N, true>, sm)) != cudaSuccess) return e;
    k_resist_grad_rows<N, true><<<dim3(grid, planes), Plan<N>::NT, sm, st>>>(band, crop, tw, target, planes_per_clip,
                                                                            beta, thr, rowbuf, partial, ppc);
  } else {
    if ((e = smem_attrs(k_resist_grad_rows<N, false>, sm)) != cudaSuccess) return e;
    k_resist_grad_rows<N, false><<<dim3(grid, planes), Plan<N>::NT, sm, st>>>(band, crop, tw, target,
                                                                             planes_per_clip, beta, thr, rowbuf,
                                                                             partial, ppc);
  }
  return cudaGetLastError();
}

template <int N>
cudaError_t band_rows_real_n(const float2* q, int planes, int crop, float scale, const float2* tw, float* out,
                             cudaStream_t st) {
  const int rpc = rows_per_cta(N, planes, 2048 / Plan<N>::NT), grid = (N + rpc - 1) / rpc;
  if (2 * crop <= N)
    k_band_rows_real<N, true><<<dim3(grid, planes), Plan<N>::NT, 0, st>>>(q, crop, scale, tw, out, rpc);
  else
    k_band_rows_real<N, false><<<dim3(grid, planes), Plan<N>::NT, 0, st>>>(q, crop, scale, tw, out, rpc);
  return cudaGetLastError();
}

template <int N>
size_t col_smem_bytes() {
  return sizeof(float2) * (N + ColW<N>::W * ColLD<N>::value);
}

template <int N>
cudaError_t mask_cols_n(const float2* rowbuf, int b, int crop, const float2* tw, float2* mhat, const float* gain,
                        bool gain_real, cudaStream_t st) {
  const size_t sm = col_smem_bytes<N>();
  cudaError_t e = smem_attrs(k_mask_cols<N>, sm);
  if (e != cudaSuccess) return e;
  k_mask_cols<N><<<dim3(crop / ColW<N>::W, b), Plan<N>::NT * ColW<N>::W, sm, st>>>(rowbuf, crop, tw, gain, mhat,
                                                                                   gain_real ? 1 : 0);
  return cudaGetLastError();
}

template <int N>
cudaError_t mask_rows_n(const float* m, int b, int crop, const float2* tw, float2* rowbuf, cudaStream_t st) {
  const size_t smr = sizeof(float2) * (2 * N + PadLen<N>::value + 1);
  cudaError_t e = smem_attrs(k_mask_rows<N>, smr);
  if (e != cudaSuccess) return e;
  const int ppc = rows_per_cta(N / 2, b, 2048 / Plan<N>::NT);
  k_mask_rows<N><<<dim3((N / 2 + ppc - 1) / ppc, b), Plan<N>::NT, smr, st>>>(m, crop, tw, rowbuf, ppc);
  return cudaGetLastError();
}

template <int N>
cudaError_t mask_spectrum_n(const float* m, int b, int crop, const float2* tw, float2* rowbuf, float2* mhat,
                            const float* gain, bool gain_real, cudaStream_t st) {
  const size_t smr = sizeof(float2) * (2 * N + PadLen<N>::value + 1);
  cudaError_t e = smem_attrs(k_mask_rows<N>, smr);
  if (e != cudaSuccess) return e;
  const int ppc = rows_per_cta(N / 2, b, 2048 / Plan<N>::NT);
  k_mask_rows<N><<<dim3((N / 2 + ppc - 1) / ppc, b), Plan<N>::NT, smr, st>>>(m, crop, tw, rowbuf, ppc);
  const size_t sm = col_smem_bytes<N>();
  e = smem_attrs(k_mask_cols<N>, sm);
  if (e != cudaSuccess) return e;
  k_mask_cols<N><<<dim3(crop / ColW<N>::W, b), Plan<N>::NT * ColW<N>::W, sm, st>>>(rowbuf, crop, tw, gain, mhat,
                                                                                   gain_real ? 1 : 0);
  return cudaGetLastError();
}

template <int N>
cudaError_t stage1_n(const float2* mhat, const float2* phi, int nk, int crop, const float2* tw, float2* t1,
                     cudaStream_t st, int clips) {
  return launch_stage1_cols<N, Stage1W<N>::W>(mhat, phi, nk, crop, tw, OutC64{t1, N, crop}, st, clips);
}

template <int N>
cudaError_t stage2_n(const float2* t1, const float* lam, int nk, int crop, float dose, const float2* tw, float* img,
                     int planes, long long t1_plane, long long img_plane, int lam_period, cudaStream_t st) {
  if (2 * crop <= N)
    k_stage2<N, true><<<dim3(N, planes), Plan<N>::NT, 0, st>>>(t1, lam, nk, crop, dose, tw, img, t1_plane,
                                                               img_plane, lam_period);
  else
    k_stage2<N, false><<<dim3(N, planes), Plan<N>::NT, 0, st>>>(t1, lam, nk, crop, dose, tw, img, t1_plane,
                                                                img_plane, lam_period);
  return cudaGetLastError();
}

// Transform sizes of the full grid (powers of two) ...
#define LITHO_DISPATCH_N(n, CALL)          \
  switch (n) {                             \
    case 32: return CALL(32);              \
    case 64: return CALL(64);              \
    case 128: return CALL(128);            \
    case 256: return CALL(256);            \
    case 512: return CALL(512);            \
    case 1024: return CALL(1024);          \
    case 2048: return CALL(2048);          \
    default: return cudaErrorInvalidValue; \
  }

// ... and of the forward transforms on a coarse grid (also 896, tensor-core path)
#define LITHO_DISPATCH_NC(n, CALL)          \
  switch (n) {                             \
    case 32: return CALL(32);              \
    case 64: return CALL(64);              \
    case 128: return CALL(128);            \
    case 256: return CALL(256);            \
    case 512: return CALL(512);            \
    case 1024: return CALL(1024);          \
    case 2048: return CALL(2048);          \
    case 896: return CALL(896);            \
    default: return cudaErrorInvalidValue; \
  }

}  // namespace

bool fft_twiddle_table(int n, float2* out) {
  switch (n) {
    case 32: fill_twiddle_table<32>(out); return true;
    case 64: fill_twiddle_table<64>(out); return true;
    case 128: fill_twiddle_table<128>(out); return true;
    case 256: fill_twiddle_table<256>(out); return true;
    case 512: fill_twiddle_table<512>(out); return true;
    case 1024: fill_twiddle_table<1024>(out); return true;
    case 2048: fill_twiddle_table<2048>(out); return true;
    case 896: fill_twiddle_table<896>(out); return true;
    default: return false;
  }
}

cudaError_t launch_mask_spectrum(const float* m, int b, int n, int crop, const float2* tw, float2* rowbuf,
                                 float2* mhat, cudaStream_t st, const float* gain, bool gain_real) {
#define CALL(N) mask_spectrum_n<N>(m, b, crop, tw, rowbuf, mhat, gain, gain_real, st)
  LITHO_DISPATCH_NC(n, CALL)
#undef CALL
}

cudaError_t launch_band_rows_real(const float2* q, int planes, int n, int crop, float scale, const float2* tw,
                                  float* out, cudaStream_t st) {
#define CALL(N) band_rows_real_n<N>(q, planes, crop, scale, tw, out, st)
  LITHO_DISPATCH_N(n, CALL)
#undef CALL
}

cudaError_t launch_mask_rows(const float* m, int b, int n, int crop, const float2* tw, float2* rowbuf,
                             cudaStream_t st) {
#define CALL(N) mask_rows_n<N>(m, b, crop, tw, rowbuf, st)
  LITHO_DISPATCH_NC(n, CALL)
#undef CALL
}

cudaError_t launch_blur_gain(const ResistTaps& taps, int n, int crop, float* gain, cudaStream_t st) {
  if (n < 1 || crop < 1) return cudaErrorInvalidValue;
  k_blur_gain<<<(crop + 127) / 128, 128, 0, st>>>(taps, n, crop, gain);
  return cudaGetLastError();
}

cudaError_t launch_resist_grad_rows(const float2* band, int planes, int n, int crop, const float2* tw,
                                    const float* target, int planes_per_clip, float beta, float thr, float2* rowbuf,
                                    double* partial, cudaStream_t st) {
#define CALL(N) resist_grad_rows_n<N>(band, planes, crop, tw, target, planes_per_clip, beta, thr, rowbuf, partial, st)
  LITHO_DISPATCH_N(n, CALL)
#undef CALL
}
cudaError_t launch_mask_cols(const float2* rowbuf, int b, int n, int crop, const float2* tw, float2* mhat,
                             const float* gain, bool gain_real, cudaStream_t st) {
#define CALL(N) mask_cols_n<N>(rowbuf, b, crop, tw, mhat, gain, gain_real, st)
  LITHO_DISPATCH_NC(n, CALL)
#undef CALL
}
cudaError_t launch_band_rows_resist(const float2* q, int planes, int n, int crop, const float2* tw, float threshold,
                                    float* img, float* iblur, uint8_t* printed, cudaStream_t st) {
#define CALL(N) band_rows_resist_n<N>(q, planes, crop, tw, threshold, img, iblur, printed, st)
  LITHO_DISPATCH_N(n, CALL)
#undef CALL
}

cudaError_t launch_stage1_fft(const float2* mhat, const float2* phi, int nk, int n, int crop, const float2* tw,
                              float2* t1, cudaStream_t st, int clips) {
#define CALL(N) stage1_n<N>(mhat, phi, nk, crop, tw, t1, st, clips)
  LITHO_DISPATCH_N(n, CALL)
#undef CALL
}

cudaError_t launch_stage2_fft(const float2* t1, const float* lam, int nk, int n, int crop, float dose,
                              const float2* tw, float* img, int planes, long long t1_plane_stride,
                              long long img_plane_stride, cudaStream_t st, int lam_period, const float2* tw32,
                              const float2* tw512, bool folded, float2* spec, int spec_crop) {
  if (lam_period <= 0) lam_period = planes;
  if (tw32 && stage2_w32_supported(n, crop))
    return launch_stage2_w32(t1, lam, nk, n, crop, dose, tw32, img, planes, t1_plane_stride, img_plane_stride,
                             lam_period, st, folded, spec, spec_crop);
  // only the warp-per-row kernel sums unweighted or writes row spectra
  if (folded || spec) return cudaErrorInvalidValue;
  if (tw512 && stage2_w512_supported(n, crop))
    return launch_stage2_w512(t1, lam, nk, n, crop, dose, tw512, img, planes, t1_plane_stride, img_plane_stride,
                              lam_period, st);
#define CALL(N) stage2_n<N>(t1, lam, nk, crop, dose, tw, img, planes, t1_plane_stride, img_plane_stride, lam_period, st)
  LITHO_DISPATCH_N(n, CALL)
#undef CALL
}

}  // namespace litho
