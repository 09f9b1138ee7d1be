// ILT loss and its adjoint (mask gradient) on the FP32 FFT path.
//
// Objective (pixel-based ILT, the paper's Section I prior art; dI/dM is the
// input channel of its Eq. (9)):
//   m = sigmoid(a theta),  I_f = D sum_k lam_fk |E_fk|^2 (Eq. (4)),
//   Ib_f = g (x) I_f (Eq. (5) blur),  Z_f = sigmoid(b (Ib_f - t)),
//   L = sum_f sum_x (Z_f - target)^2.
// Adjoint by the chain rule (g symmetric, so the blur is its own adjoint):
//   q_f = 2 (Z_f - target) b Z_f (1 - Z_f),  G_f = g (x) q_f          (= dL/dI_f)
//   H_fk(u) = sum_x G_f(x) E_fk(x) e^{-2 pi i u.x/N}    on the crop
//   S(u) = sum_f sum_k lam_fk conj(Phi_fk(u)) H_fk(u)
//   dL/dm(x) = 2 D N^-2 Re sum_u S(u) e^{+2 pi i u.x/N},  dL/dtheta = dL/dm a m (1 - m).
//
// Kernels (per clip, for a group of P focus planes at a time):
//   k_sigmoid        m from theta
//   (mask spectrum, stage 1, stage 2, resist blur: shared with the forward path)
//   k_resist_grad    Z, q and per-block FP64 partial sums of (Z - target)^2
//                    (coarse grid: k_resist_grad_rows, per row pair, with the
//                    forward row spectra of q)
//   k_reduce_loss    fixed-order FP64 sum of the partials (deterministic)
//   k_adj_rows       per image row: E_fk from the stage-1 field (inverse FFT),
//                    times G_f, forward FFT, crop columns -> U_fk[y][c]
//   k_adj_cols       per crop column block and run of a clip's fields: forward
//                    FFT over y, crop rows, times lam conj(Phi), summed over
//                    the run in registers -> one partial S per run
//   k_sum_planes     S = sum of a clip's runs in fixed order
//   k_grad_rows      band-to-full inverse of S along x (after stage 1 along y),
//                    real part, chain factor -> dL/dtheta
// The fields E are never stored: each backward row recomputes E_fk from the
// stage-1 field T_fk (C values per row) that the forward pass kept.
#include <algorithm>
#include <cmath>

#include "fft_common.cuh"
#include "litho_internal.h"

namespace litho {

namespace {

constexpr int kPartials = 1024;  // blocks of k_resist_grad, fixed for a deterministic reduction

__device__ __forceinline__ int freq_of_idx(int idx, int n) { return idx < n / 2 ? idx : idx - n; }

// m = sigmoid(alpha theta), four values per thread and step (count a multiple of 4, 16-byte aligned)
__global__ void k_sigmoid(const float4* __restrict__ theta, float alpha, float4* __restrict__ m, size_t count4) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 t = theta[i];
    m[i] = make_float4(1.0f / (1.0f + expf(-alpha * t.x)), 1.0f / (1.0f + expf(-alpha * t.y)),
                       1.0f / (1.0f + expf(-alpha * t.z)), 1.0f / (1.0f + expf(-alpha * t.w)));
  }
}

// Clip blockIdx.y: its `planes` planes of ib and q, its target, its
// kPartials partial sums (the same partition for every group size).
__global__ void __launch_bounds__(256) k_resist_grad(const float* __restrict__ ib, const float* __restrict__ target,
                                                     size_t nn, int planes, float beta, float thr,
                                                     float* __restrict__ q, double* __restrict__ partial) {
  const size_t clip = blockIdx.y;
  ib += clip * planes * nn;
  q += clip * planes * nn;
  target += clip * nn;
  partial += clip * gridDim.x;
  double acc = 0.0;
  const size_t total = nn * planes, stride = (size_t)gridDim.x * blockDim.x;
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t pix = i % nn;  // i mod nn, carried along instead of recomputed
  for (; i < total; i += stride) {
    const float z = 1.0f / (1.0f + expf(-beta * (ib[i] - thr)));
    const float d = z - target[pix];
    acc += double(d) * double(d);
    q[i] = 2.0f * d * beta * z * (1.0f - z);
    pix += stride;
    while (pix >= nn) pix -= nn;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double ws[8];
  if (threadIdx.x % 32 == 0) ws[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += ws[w];
    partial[blockIdx.x] = s;
  }
}

// Clip blockIdx.x: out[clip] (+)= the fixed-order sum of its `count` partials.
__global__ void __launch_bounds__(1024) k_reduce_loss(const double* __restrict__ partial, int count,
                                                      double* __restrict__ out, int accumulate) {
  __shared__ double s[1024];
  partial += (size_t)blockIdx.x * count;
  out += blockIdx.x;
  double a = 0.0;
  for (int i = threadIdx.x; i < count; i += 1024) a += partial[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (accumulate ? *out : 0.0) + s[0];
}

// Backward rows: for every kernel of the plane, E = inverse FFT of the band row
// T[y][:], P = G[y][:] E, U[y][c] = forward FFT of P on the crop columns.
// Plane p takes lam[(p mod lam_period) nk ...] (clips of a group repeat the focus planes).
// BANDED (2 crop <= N): the band row's zero half is skipped in the first pass.
template <int N, bool BANDED>
__global__ void __launch_bounds__(Plan<N>::NT) k_adj_rows(const float2* __restrict__ t1, const float* __restrict__ lam,
                                                          int nk, int crop, const float* __restrict__ g,
                                                          const float2* __restrict__ tw_g, float2* __restrict__ u,
                                                          int lam_period) {
  using PL = Plan<N>;
  constexpr int NT = PL::NT, RL = PL::R[PL::P - 1];
  constexpr int PERL = PassShape<N, NT, RL>::PER;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* bufa = sm + N;
  float2* bufb = sm + N + PadLen<N>::value;
  load_twiddles<N>(tw, tw_g);
  const int y = blockIdx.x, plane = blockIdx.y, t = threadIdx.x, half = crop / 2;
  float gv[PERL][RL];
  const float* grow = g + ((size_t)plane * N + y) * N;
#pragma unroll
  for (int p = 0; p < PERL; ++p)
#pragma unroll
    for (int q = 0; q < RL; ++q) {
      const int jj = t + p * NT;
      gv[p][q] = jj < N / RL ? grow[jj + q * (N / RL)] : 0.f;
    }
  __syncthreads();
  for (int k = 0; k < nk; ++k) {
    if (lam[(plane % lam_period) * nk + k] == 0.f) continue;
    const size_t rowoff = (((size_t)plane * nk + k) * N + y) * crop;
    const float2* row = t1 + rowoff;
    auto load_band = [&](int, int r, int idx) {
      const int c = (r < PL::R[0] / 2 ? idx : idx - N) + half;  // first pass: idx < N/2 exactly when r < R/2
      return (c >= 0 && c < crop) ? __ldg(row + c) : make_float2(0.f, 0.f);
    };
    auto times_g = [&](int p, int q, int idx, float2 v) {
      bufb[pad16(idx)] = make_float2(v.x * gv[p][q], v.y * gv[p][q]);
    };
    fft_load_use<N, +1, decltype(load_band), decltype(times_g), BANDED>(bufa, tw, t, load_band, times_g);
    __syncthreads();
    auto load_prod = [&](int idx) { return bufb[pad16(idx)]; };
    float2* urow = u + rowoff;
    auto store_crop = [&](int, int, int idx, float2 v) {
      const int c = freq_of_idx(idx, N) + half;
      if (c >= 0 && c < crop) urow[c] = v;
    };
    fft_load_use<N, -1>(bufa, tw, t, load_prod, store_crop);
  }
}

// Backward rows for 512-point rows, two rows per warp (same result as
// k_adj_rows<512>): per kernel, E = inverse transform of the band row, P = G E,
// U = forward transform of P on the crop columns.  512 = 16 x 32 in Stockham
// order:
//   inverse pass 1 (radix 16): lane l takes x[l + 32 r] of both rows -> 16 l + q;
//   inverse pass 2 (radix 32): lanes 0-15 take row A, lanes 16-31 row B; lane j
//     takes position j + 16 r, applies w^(r j) (w = e^{+2 pi i/512}) and forms a
//     32-point DFT whose output q is E(x) at x = j + 16 q;
//   forward pass 1 (radix 32): the forward transform's first butterfly j needs
//     P(j + 16 r), r < 32 -- exactly what lane j holds, so P = G E and this
//     pass stay in registers (output q at 32 j + q);
//   forward pass 2 (radix 16): lane l takes position l + 32 r of both rows,
//     applies conj(w)^(r l) and forms a 16-point DFT whose output q is U(u) at
//     u = l + 32 q; the crop columns are stored.
// Two shared-memory exchanges per row and kernel (padded i + i/16 and
// i + i/32, conflict-free), no block barrier inside the kernel loop; the next
// kernel's band rows are staged with cp.async while the current ones are
// transformed.  BANDED: crop / 2 <= 128, so inputs r in [4, 12) of the first
// pass are zero.
constexpr int kAdjWarps = 8;
constexpr int kAdjTw1 = 31 * 16, kAdjTw2 = 15 * 32;  // w^(r j), r < 32, j < 16; conj(w)^(r l), r < 16, l < 32
constexpr int kAdjBuf = 512 + 32;                     // one row, either padding

__device__ __forceinline__ void adj_cp16(void* smem_dst, const void* gmem_src) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem_src) : "memory");
}

template <bool BANDED>
__global__ void __launch_bounds__(32 * kAdjWarps, 2)
    k_adj_rows_w512(const float2* __restrict__ t1, const float* __restrict__ lam, int nk, int crop,
                    const float* __restrict__ g, const float2* __restrict__ tw_g, float2* __restrict__ u,
                    int lam_period) {
  constexpr int N = 512;
  extern __shared__ float4 smem_raw[];
  float2* tw1 = reinterpret_cast<float2*>(smem_raw);  // inverse pass 2: (r - 1) 16 + j
  float2* tw2 = tw1 + kAdjTw1;                        // forward pass 2: (r - 1) 32 + l
  float2* bufs = tw2 + kAdjTw2;                       // [warp][2 rows][kAdjBuf]
  float2* stage0 = bufs + kAdjWarps * 2 * kAdjBuf;    // [warp][2 rows][crop]
  for (int i = threadIdx.x; i < kAdjTw1 + kAdjTw2; i += blockDim.x) tw1[i] = tw_g[i];
  __syncthreads();
  const int lane = threadIdx.x % 32, wp = threadIdx.x / 32, half = crop / 2;
  const int y0 = (blockIdx.x * kAdjWarps + wp) * 2, plane = blockIdx.y;
  if (y0 >= N) return;  // no block barrier below
  float2* buf = bufs + wp * 2 * kAdjBuf;
  float2* stage = stage0 + (size_t)wp * 2 * crop;
  const float* lp = lam + (plane % lam_period) * nk;
  const size_t field = (size_t)N * crop;
  const float2* t1p = t1 + (size_t)plane * nk * field;
  float2* up = u + (size_t)plane * nk * field;
  // this lane's row in passes 2 and 3 (inverse pass 2, forward pass 1) and its butterfly
  const int rsel = lane / 16, jj = lane % 16;
  float gv[32];  // G(y, jj + 16 q) of the lane's row
  {
    const float* grow = g + ((size_t)plane * N + y0 + rsel) * N;
#pragma unroll
    for (int q = 0; q < 32; ++q) gv[q] = __ldg(grow + jj + 16 * q);
  }
  auto fetch = [&](int k) {  // band rows y0, y0 + 1 of kernel k: 2 x crop/2 pieces of 16 bytes
    const float2* src = t1p + (size_t)k * field + (size_t)y0 * crop;
    for (int i = lane; i < crop; i += 32) adj_cp16(stage + 2 * i, src + 2 * i);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  fetch(0);
  for (int k = 0; k < nk; ++k) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    // inverse pass 1 for both rows (lane l: x[l + 32 r])
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
    __syncwarp();  // both band rows are in registers: the staging buffer takes kernel k + 1
    if (k + 1 < nk) fetch(k + 1);
    if (lp[k] == 0.f) continue;  // a zero kernel: U is not written (the column pass skips it)
#pragma unroll
    for (int row = 0; row < 2; ++row) {
      dft_reg<16, +1, BANDED>(a[row]);
#pragma unroll
      for (int q = 0; q < 16; ++q) buf[row * kAdjBuf + pad16(16 * lane + q)] = a[row][q];
    }
    __syncwarp();
    // inverse pass 2: lane j = jj of row rsel, positions j + 16 r
    float2 v[32];
    const float2* rb = buf + rsel * kAdjBuf;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      v[r] = rb[pad16(jj + 16 * r)];
      if (r > 0) v[r] = cmul(v[r], tw1[(r - 1) * 16 + jj]);
    }
    __syncwarp();  // the row buffers are read; the forward pass writes them next
    dft32<+1, false>(v);  // v[q] = E(jj + 16 q)
    // P = G E, then forward pass 1 over the same 32 values
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = make_float2(v[q].x * gv[q], v[q].y * gv[q]);
    dft32<-1, false>(v);  // output q at 32 jj + q
    float2* wb = buf + rsel * kAdjBuf;
#pragma unroll
    for (int q = 0; q < 32; ++q) wb[32 * jj + q + jj] = v[q];  // padded i + i/32 (i = 32 jj + q)
    __syncwarp();
    // forward pass 2 for both rows: lane l, positions l + 32 r
#pragma unroll
    for (int row = 0; row < 2; ++row) {
      const float2* fb = buf + row * kAdjBuf;
      float2 b[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int i = lane + 32 * r;
        b[r] = fb[i + i / 32];
        if (r > 0) b[r] = cmul(b[r], tw2[(r - 1) * 32 + lane]);
      }
      dft_reg<16, -1, false>(b);  // b[q] = U(lane + 32 q)
      float2* urow = up + (size_t)k * field + (size_t)(y0 + row) * crop;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int idx = lane + 32 * q;
        const int c = (q < 8 ? idx : idx - N) + half;
        if (c >= 0 && c < crop) urow[c] = b[q];
      }
    }
    __syncwarp();  // the row buffers are free for the next kernel
  }
}

// Backward columns: forward FFT over y of U_j[:, c], crop rows, times lam_j conj(Phi_j);
// field j uses kernel j mod period.  W columns per CTA with the lanes of a
// warp interleaved over them (as in stage 1): the first pass reads U straight
// from global memory (W adjacent columns of 32/W rows per warp load: whole
// sectors), the last pass hands each thread the same output positions for
// every field, and a CTA runs a run of fields in turn so that its twiddle
// table is loaded once.
template <int N> struct AdjW { static constexpr int W = Plan<N>::NT <= 64 ? 8 : 4; };

// Where the adjoint columns keep their sums: in registers they cost the
// 512-point kernel its second CTA per SM (or spills), in shared memory they
// cost the 1024-point one (twice the slots); so shared memory up to 512.
template <int N> struct AdjAccInSmem { static constexpr bool value = N <= 512; };

// Runs of fields per clip in the adjoint columns: the largest divisor of the
// clip's field count that is at most 8 (a function of that count alone, so a
// clip's sums do not depend on how many clips a launch holds).
int adj_col_splits(int period) {
  for (int d = 8; d > 1; --d)
    if (period % d == 0) return d;
  return 1;
}

// Per crop column block and run of fields j in [j0, j1) of one clip (the
// clip's `period` fields split into `splits` runs of period / splits): the
// forward transform over y of each field's column, the crop, lam conj(Phi)
// times it, summed over the run (in registers, or up to 512 points in shared
// memory, one slot per thread and output position) and written once, to
// part[clip splits + split][cv][c].  k_sum_planes then adds a clip's runs in
// order, so the sum's order depends on the clip's own field count only.
template <int N>
__global__ void __launch_bounds__(Plan<N>::NT * AdjW<N>::W, AdjAccInSmem<N>::value ? 2 : 1) k_adj_cols(const float2* __restrict__ u,
                                                                        const float2* __restrict__ phi,
                                                                        const float* __restrict__ lam, int crop,
                                                                        const float2* __restrict__ tw_g,
                                                                        float2* __restrict__ part, int period,
                                                                        int splits) {
  constexpr int W = AdjW<N>::W, NT = Plan<N>::NT, LD = (PadLen<N>::value + 15) / 16 * 16 + 16 / W;
  constexpr int RL = Plan<N>::R[Plan<N>::P - 1], PERL = PassShape<N, NT, RL>::PER;
  constexpr int T = NT * W;
  constexpr bool kSmem = AdjAccInSmem<N>::value;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  constexpr int R0 = Plan<N>::R[0], NB0 = N / R0;
  static_assert(PassShape<N, NT, R0>::PER == 1, "one first-pass butterfly per thread");
  const int tid = threadIdx.x, g = tid % W, t = tid / W, c0 = blockIdx.x * W, half = crop / 2;
  const int clip = blockIdx.y / splits, split = blockIdx.y % splits, jb = period / splits;
  float2* acc_s = buf + W * LD;  // kSmem: this thread's PERL x RL sums at (pp RL + q) T + tid
  float2 acc_r[kSmem ? 1 : PERL * RL];
  auto acc = [&](int i) -> float2& {
    if constexpr (kSmem)
      return acc_s[i * T + tid];  // read and written by tid alone
    else
      return acc_r[i];
  };
  const int j0 = clip * period + split * jb, j1 = j0 + jb;
  load_twiddles<N>(tw, tw_g);
  // this thread's first-pass inputs (rows t + r N/R0) of a field, loaded one field ahead
  float2 nxt[R0];
  auto prefetch = [&](int j) {
    const float2* src = u + (size_t)j * N * crop + c0 + g;  // row y at src[y crop]
#pragma unroll
    for (int r = 0; r < R0; ++r) nxt[r] = t < NB0 ? __ldg(src + (size_t)(t + r * NB0) * crop) : make_float2(0.f, 0.f);
  };
  prefetch(j0);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PERL * RL; ++i) acc(i) = make_float2(0.f, 0.f);
  for (int j = j0; j < j1; ++j) {
    const int jk = j % period;
    const float l = lam[jk];
    if (l == 0.f) {  // uniform across the block: nothing to add
      if (j + 1 < j1) prefetch(j + 1);
      continue;
    }
    const float2* ph = phi + (size_t)jk * crop * crop + c0 + g;
    float2 cur[R0];
#pragma unroll
    for (int r = 0; r < R0; ++r) cur[r] = nxt[r];
    auto load = [&](int, int r, int) { return cur[r]; };
    // once the first pass has consumed this field's inputs, the next field's loads go out
    auto after_first = [&]() {
      if (j + 1 < j1) prefetch(j + 1);
    };
    auto use = [&](int pp, int q, int idx, float2 h) {
      const int cv = freq_of_idx(idx, N) + half;
      if (cv >= 0 && cv < crop) {
        const float2 p = __ldg(ph + (size_t)cv * crop);
        // += lam conj(p) h
        float2& a = acc(pp * RL + q);
        a = make_float2(fmaf(l, p.x * h.x + p.y * h.y, a.x), fmaf(l, p.x * h.y - p.y * h.x, a.y));
      }
    };
    fft_load_use<N, -1, decltype(load), decltype(use), false>(buf + g * LD, tw, t, load, use, after_first);
  }
  // the last pass's output positions of this thread: idx = jj + q N/RL, jj = t + pp NT
  float2* dst = part + (size_t)blockIdx.y * crop * crop + c0 + g;  // crop row cv at dst[cv crop]
#pragma unroll
  for (int pp = 0; pp < PERL; ++pp) {
    const int jj = t + pp * NT;
    if (jj < N / RL) {
#pragma unroll
      for (int q = 0; q < RL; ++q) {
        const int cv = freq_of_idx(jj + q * (N / RL), N) + half;
        if (cv >= 0 && cv < crop) dst[(size_t)cv * crop] = acc(pp * RL + q);
      }
    }
  }
}

// x[i][ch] = img[i] for the planes i of a group (x: [.][3][nn]).
__global__ void k_to_channel(const float* __restrict__ img, float* __restrict__ x, int planes, size_t nn, int ch) {
  const size_t total = size_t(planes) * nn;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    x[(i / nn) * 3 * nn + size_t(ch) * nn + i % nn] = img[i];
}

// The adjoint for dL/dI = 1 on every pixel (the AI input's gradient channel,
// Eq. (9), and the intensity VJP without an upstream).  By Parseval,
// sum_x |E_k(x)|^2 = N^2 sum_v |mhat(v) Phi_k(v)|^2, so the sum the adjoint
// rows and columns form for G = 1 collapses to
//   S(v,u) = N^2 sum_k lam_k |Phi_k(v,u)|^2 mhat(v,u),
// exactly (on the coarse grid too: there G is the constant (N/nc)^2 and the
// transforms are on nc).  No field is transformed.  Clip blockIdx.y; the nk
// kernels of phi and lam (all planes of the call) are summed in order.
__global__ void k_ones_adjoint(const float2* __restrict__ mhat, const float2* __restrict__ phi,
                               const float* __restrict__ lam, int nk, size_t cc, float n2, float2* __restrict__ s,
                               int accumulate) {
  mhat += (size_t)blockIdx.y * cc;
  s += (size_t)blockIdx.y * cc;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cc; i += (size_t)gridDim.x * blockDim.x) {
    float d = 0.f;
    for (int k = 0; k < nk; ++k) {
      const float2 p = __ldg(phi + (size_t)k * cc + i);
      d = fmaf(__ldg(lam + k), fmaf(p.x, p.x, p.y * p.y), d);
    }
    const float2 m = mhat[i];
    float2 a = accumulate ? s[i] : make_float2(0.f, 0.f);
    a.x = fmaf(n2 * d, m.x, a.x);
    a.y = fmaf(n2 * d, m.y, a.y);
    s[i] = a;
  }
}

// s[clip] (+)= sum over the clip's `planes` planes of sk, in order (clip = blockIdx.y).
__global__ void k_sum_planes(const float2* __restrict__ sk, int planes, size_t cc, float2* __restrict__ s,
                             int accumulate) {
  sk += (size_t)blockIdx.y * planes * cc;
  s += (size_t)blockIdx.y * cc;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cc; i += (size_t)gridDim.x * blockDim.x) {
    float2 a = accumulate ? s[i] : make_float2(0.f, 0.f);
    for (int j = 0; j < planes; ++j) {
      const float2 v = sk[(size_t)j * cc + i];
      a.x += v.x;
      a.y += v.y;
    }
    s[i] = a;
  }
}

// Final rows: grad[y][x] = scale Re(sum_c Q[y][c] e^{2 pi i u_c x/N}) a m (1 - m).
template <int N>
__global__ void __launch_bounds__(Plan<N>::NT) k_grad_rows(const float2* __restrict__ qf, int crop, float scale,
                                                           const float* __restrict__ m, float alpha,
                                                           const float2* __restrict__ tw_g, float* __restrict__ grad,
                                                           long long grad_stride) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  load_twiddles<N>(tw, tw_g);
  __syncthreads();
  const int y = blockIdx.x, t = threadIdx.x, half = crop / 2;
  const size_t clip = blockIdx.y;  // clip of the group: its band rows, mask and gradient
  qf += clip * N * crop;
  if (m) m += clip * N * N;
  grad += clip * grad_stride;
  const float2* row = qf + (size_t)y * crop;
  auto load = [&](int idx) {
    const int c = freq_of_idx(idx, N) + half;
    return (c >= 0 && c < crop) ? __ldg(row + c) : make_float2(0.f, 0.f);
  };
  const float* mr = m ? m + (size_t)y * N : nullptr;
  float* gr = grad + (size_t)y * N;
  auto use = [&](int, int, int x, float2 v) {
    if (m) {
      const float mm = mr[x];
      gr[x] = scale * v.x * alpha * mm * (1.0f - mm);
    } else {
      gr[x] = scale * v.x;  // no chain factor: the gradient with respect to m itself
    }
  };
  fft_load_use<N, +1>(buf, tw, t, load, use);
}

template <int N>
cudaError_t adj_rows_n(const float2* t1, const float* lam, int nk, int crop, const float* g, const float2* tw,
                       float2* u, int planes, int lam_period, cudaStream_t st, const float2* tw512) {
  if (N == 512 && tw512 && crop % 2 == 0 && crop / 2 <= 128) {  // two rows per warp
    const size_t sm = sizeof(float2) * (kAdjTw1 + kAdjTw2 + kAdjWarps * 2 * (size_t(kAdjBuf) + crop));
    cudaError_t e = smem_attrs(k_adj_rows_w512<true>, sm);
    if (e != cudaSuccess) return e;
    k_adj_rows_w512<true><<<dim3(N / (2 * kAdjWarps), planes), 32 * kAdjWarps, sm, st>>>(t1, lam, nk, crop, g,
                                                                                          tw512, u, lam_period);
    return cudaGetLastError();
  }
  const size_t sm = sizeof(float2) * (N + 2 * PadLen<N>::value);
  auto kern = 2 * crop <= N ? k_adj_rows<N, true> : k_adj_rows<N, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<dim3(N, planes), Plan<N>::NT, sm, st>>>(t1, lam, nk, crop, g, tw, u, lam_period);
  return cudaGetLastError();
}

template <int N>
cudaError_t adj_cols_n(const float2* u, const float2* phi, const float* lam, int crop, const float2* tw, float2* part,
                       int fields, int period, cudaStream_t st) {
  constexpr int W = AdjW<N>::W;
  if (crop % W != 0 || period < 1 || fields % period != 0) return cudaErrorInvalidValue;
  constexpr int LD = (PadLen<N>::value + 15) / 16 * 16 + 16 / W;
  constexpr int RL = Plan<N>::R[Plan<N>::P - 1], PERL = PassShape<N, Plan<N>::NT, RL>::PER;
  const size_t sm = sizeof(float2) * (N + W * LD + (AdjAccInSmem<N>::value ? size_t(PERL) * RL * Plan<N>::NT * W : 0));
  cudaError_t e = smem_attrs(k_adj_cols<N>, sm);
  if (e != cudaSuccess) return e;
  const int splits = adj_col_splits(period);
  k_adj_cols<N><<<dim3(crop / W, (fields / period) * splits), Plan<N>::NT * W, sm, st>>>(u, phi, lam, crop, tw, part,
                                                                                          period, splits);
  return cudaGetLastError();
}

template <int N>
cudaError_t grad_rows_n(const float2* qf, int crop, float scale, const float* m, float alpha, const float2* tw,
                        float* grad, int clips, long long grad_stride, cudaStream_t st) {
  const size_t sm = sizeof(float2) * (N + PadLen<N>::value);
  cudaError_t e = cudaFuncSetAttribute(k_grad_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_grad_rows<N><<<dim3(N, clips), Plan<N>::NT, sm, st>>>(qf, crop, scale, m, alpha, tw, grad, grad_stride);
  return cudaGetLastError();
}

#define ILT_DISPATCH(n, CALL)              \
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

cudaError_t launch_adj_rows(int n, const float2* t1, const float* lam, int nk, int crop, const float* g,
                            const float2* tw, float2* u, int planes, int lam_period, cudaStream_t st,
                            const float2* tw512) {
#define CALL(N) adj_rows_n<N>(t1, lam, nk, crop, g, tw, u, planes, lam_period, st, tw512)
  ILT_DISPATCH(n, CALL)
#undef CALL
}
// fields = clips x period; part receives clips x adj_col_splits(period) crop x crop sums.
cudaError_t launch_adj_cols(int n, const float2* u, const float2* phi, const float* lam, int crop, const float2* tw,
                            float2* part, int fields, int period, cudaStream_t st) {
#define CALL(N) adj_cols_n<N>(u, phi, lam, crop, tw, part, fields, period, st)
  ILT_DISPATCH(n, CALL)
#undef CALL
}
// Clip i of `clips` writes grad + i grad_stride.
cudaError_t launch_grad_rows(int n, const float2* qf, int crop, float scale, const float* m, float alpha,
                             const float2* tw, float* grad, int clips, long long grad_stride, cudaStream_t st) {
#define CALL(N) grad_rows_n<N>(qf, crop, scale, m, alpha, tw, grad, clips, grad_stride, st)
  ILT_DISPATCH(n, CALL)
#undef CALL
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

struct IltLayout {
  float* m;
  float2 *rowbuf, *mhat, *t1, *u, *sk, *s, *qf;
  float *img, *blur;
  double *partial, *loss;
  // coarse grid (nc x nc, band 2C of the image): coarse images and the coarse
  // samples of the low-passed dL/dI (ic), row spectra on nc (mid), band rows
  // on N (big), image spectra (spec)
  float* ic;
  float2 *mid, *big, *spec;
  float* gain;  // the resist blur's transfer function on the 2C band
  size_t bytes;
};

// Clips per group: the group's stage-1 fields at the full grid within 2 GiB,
// and groups of equal size.
int ilt_group(const litho_kernels* h, int b) {
  const size_t per_clip = size_t(h->n_focus) * h->k * h->n * h->crop * sizeof(float2);
  const size_t cap = std::max<size_t>(1, std::min<size_t>(size_t(b), (size_t(2) << 30) / per_clip));
  const size_t groups = (size_t(b) + cap - 1) / cap;
  return int((size_t(b) + groups - 1) / groups);
}

// Carves the workspace for groups of G clips and P focus planes at a time
// (P = all planes with G = ilt_group, or P = 1 with G = 1).  The b FP64
// losses come first, so their address does not depend on P or G.
IltLayout ilt_layout(const litho_kernels* h, int b, int P, int G, void* base) {
  const size_t N = h->n, C = h->crop, K = h->k, g = size_t(G), PG = size_t(P) * G;
  IltLayout L{};
  size_t off = 0;
  char* p = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> char* {
    char* r = p ? p + off : nullptr;
    off += up256(bytes);
    return r;
  };
  L.loss = reinterpret_cast<double*>(take(size_t(b) * 8));
  L.m = reinterpret_cast<float*>(take(g * N * N * 4));
  L.rowbuf = reinterpret_cast<float2*>(take(g * N * C * 8));
  L.mhat = reinterpret_cast<float2*>(take(g * C * C * 8));
  L.t1 = reinterpret_cast<float2*>(take(PG * K * N * C * 8));
  L.u = reinterpret_cast<float2*>(take(PG * K * N * C * 8));
  L.sk = reinterpret_cast<float2*>(take(PG * K * C * C * 8));
  L.s = reinterpret_cast<float2*>(take(g * C * C * 8));
  L.qf = reinterpret_cast<float2*>(take(g * N * C * 8));
  L.img = reinterpret_cast<float*>(take(PG * N * N * 4));
  L.blur = reinterpret_cast<float*>(take(PG * N * N * 4));
  // k_resist_grad: kPartials per clip; the coarse grid's fused rows: one per row pair of each plane
  L.partial = reinterpret_cast<double*>(take(g * std::max<size_t>(kPartials, size_t(P) * N / 2) * 8));
  const size_t NC = h->nc, C2 = 2 * C;
  if (NC > 0) {
    L.ic = reinterpret_cast<float*>(take(PG * NC * NC * 4));
    L.mid = reinterpret_cast<float2*>(take(PG * NC * C2 * 8));
    L.big = reinterpret_cast<float2*>(take(PG * N * C2 * 8));
    L.spec = reinterpret_cast<float2*>(take(PG * C2 * C2 * 8));
    L.gain = reinterpret_cast<float*>(take(C2 * 4));
  }
  L.bytes = off;
  return L;
}

// Planes and clips per pass for a workspace of `bytes` (false: below the minimum).
bool ilt_plan(const litho_kernels* h, int b, int planes, size_t bytes, int* P, int* G) {
  const int g = ilt_group(h, b);
  if (bytes >= ilt_layout(h, b, planes, g, nullptr).bytes) {
    *P = planes;
    *G = g;
    return true;
  }
  *P = 1;  // one focus plane of one clip at a time: its stage-1 fields are rebuilt per plane
  *G = 1;
  return bytes >= ilt_layout(h, b, 1, 1, nullptr).bytes;
}

}  // namespace

void adj512_table(float2* out) {
  const double two_pi = 2.0 * 3.14159265358979323846;
  for (int r = 1; r < 32; ++r)
    for (int j = 0; j < 16; ++j) {
      const double a = two_pi * double(r * j) / 512.0;
      out[(r - 1) * 16 + j] = make_float2(float(std::cos(a)), float(std::sin(a)));
    }
  for (int r = 1; r < 16; ++r)
    for (int l = 0; l < 32; ++l) {
      const double a = two_pi * double(r * l) / 512.0;
      out[kAdjTw1 + (r - 1) * 32 + l] = make_float2(float(std::cos(a)), float(-std::sin(a)));
    }
}

double* ilt_loss_device(const litho_kernels* h, int b, void* workspace, size_t workspace_bytes) {
  (void)h;
  (void)b;
  (void)workspace_bytes;
  return static_cast<double*>(workspace);  // the losses lead every layout
}

size_t ai_channels_bytes(const litho_kernels* h, int b) { return ilt_layout(h, b, 1, ilt_group(h, b), nullptr).bytes; }

litho_status ai_channels(const litho_kernels* h, const float* target, int b, double dose, int focus, bool coarse,
                         float* x, void* workspace, cudaStream_t st) {
  const int G = ilt_group(h, b), K = h->k, N = h->n, C = h->crop;
  IltLayout L = ilt_layout(h, b, 1, G, workspace);
  const size_t nn = size_t(N) * N;
  coarse = coarse && h->nc > 0 && interp_cols_supported(h->nc, N);
  const int NE = coarse ? h->nc : N, C2 = 2 * C;
  const float2* twe = coarse ? h->d_twc : h->d_tw;
  const float2* phi = h->d_phi + size_t(focus) * K * C * C;
  const float* lam = h->d_lambda + size_t(focus) * K;
  const float scale = float(2.0 * dose / (double(N) * double(N)));
  // a 1024-point coarse grid: the warp-per-row stage 2 writes the coarse image's row spectra itself
  const bool rows2 = coarse && h->d_tw32 && stage2_w32_supported(NE, C);
  for (int c0 = 0; c0 < b; c0 += G) {
    const int g = std::min(G, b - c0);
    {  // channel 1: the aerial image of the targets (interpolated from the coarse grid)
      ProfScope ps(kStageIltForward, st, coarse ? (rows2 ? 6 : 7) : 4);
      LITHO_TRY_CUDA(launch_mask_spectrum(target + c0 * nn, g, N, C, h->d_tw, L.rowbuf, L.mhat, st));
      LITHO_TRY_CUDA(launch_stage1_fft(L.mhat, phi, K, NE, C, twe, L.t1, st, g));
      LITHO_TRY_CUDA(launch_stage2_fft(L.t1, lam, K, NE, C, float(dose), twe, coarse ? L.ic : L.img, g,
                                       (long long)K * NE * C, (long long)NE * NE, st, 1, h->d_tw32, h->d_tw512, false,
                                       rows2 ? L.mid : nullptr, C2));
      if (coarse) {
        if (!rows2) LITHO_TRY_CUDA(launch_mask_rows(L.ic, g, NE, C2, twe, L.mid, st));
        LITHO_TRY_CUDA(launch_interp_cols(L.mid, g, NE, N, C2, twe, h->d_tw, nullptr, L.big, st));
        LITHO_TRY_CUDA(launch_band_rows_real(L.big, g, N, C2, 1.0f, h->d_tw, L.img, st));
      }
      k_to_channel<<<512, 256, 0, st>>>(L.img, x + size_t(c0) * 3 * nn, g, nn, 1);
      LITHO_TRY_CUDA(cudaGetLastError());
    }
    {  // channel 2: the adjoint applied to dL/dI = 1, in closed form (k_ones_adjoint)
      ProfScope ps(kStageIltBackward, st, 3);
      k_ones_adjoint<<<dim3(128, g), 256, 0, st>>>(L.mhat, phi, lam, K, size_t(C) * C,
                                                   float(double(N) * double(N)), L.s, 0);
      LITHO_TRY_CUDA(cudaGetLastError());
      LITHO_TRY_CUDA(launch_stage1_fft(L.s, nullptr, g, N, C, h->d_tw, L.qf, st));
      LITHO_TRY_CUDA(launch_grad_rows(N, L.qf, C, scale, nullptr, 0.f, h->d_tw, x + (size_t(c0) * 3 + 2) * nn, g,
                                      (long long)3 * nn, st));
    }
  }
  return LITHO_OK;
}

}  // namespace litho

using namespace litho;

extern "C" {

litho_status litho_ilt_workspace_size(const litho_kernels* h, int b, size_t* full_bytes, size_t* min_bytes) {
  if (!h || b < 1) {
    set_error("null handle or b < 1");
    return LITHO_EINVAL;
  }
  if (full_bytes) *full_bytes = ilt_layout(h, b, h->n_focus, ilt_group(h, b), nullptr).bytes;
  if (min_bytes) *min_bytes = ilt_layout(h, b, 1, 1, nullptr).bytes;
  return LITHO_OK;
}

litho_status litho_ilt_grad(const litho_kernels* h, const float* theta_dev, const float* target_dev, int b,
                            double dose, double mask_steep, double resist_steep, double threshold, double sigma_nm,
                            litho_precision prec, float* grad_dev, double* loss_host, void* workspace_dev,
                            size_t workspace_bytes, void* stream) {
  if (!h || !theta_dev || !target_dev || !grad_dev || !workspace_dev || b < 1) {
    set_error("null argument or b < 1");
    return LITHO_EINVAL;
  }
  if ((int(prec) & ~LITHO_GRID_COARSE) != LITHO_PREC_FFT32) {
    set_error("litho_ilt_grad implements the FP32 FFT path only (LITHO_PREC_FFT32, optionally | LITHO_GRID_COARSE)");
    return LITHO_EUNSUPPORTED;
  }
  if (!std::isfinite(dose) || !std::isfinite(mask_steep) || !std::isfinite(resist_steep) ||
      !std::isfinite(threshold)) {
    set_error("non-finite parameter");
    return LITHO_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(workspace_dev) & 255) != 0) {
    set_error("workspace must be 256-byte aligned");
    return LITHO_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(theta_dev) & 15) != 0) {
    set_error("theta must be 16-byte aligned");
    return LITHO_EINVAL;
  }
  ResistTaps taps;
  std::string why;
  if (!resist_taps(sigma_nm, h->pixel_nm, &taps, &why)) {
    set_error("%s", why.c_str());
    return LITHO_EINVAL;
  }
  if (2 * taps.radius >= h->n) {
    set_error("blur radius must be below n/2");
    return LITHO_EINVAL;
  }
  const int F = h->n_focus, K = h->k, N = h->n, C = h->crop;
  int P, G;
  if (!ilt_plan(h, b, F, workspace_bytes, &P, &G)) {
    set_error("workspace too small: %zu bytes given, at least %zu needed", workspace_bytes,
              ilt_layout(h, b, 1, 1, nullptr).bytes);
    return LITHO_ENOMEM;
  }
  IltLayout L = ilt_layout(h, b, P, G, workspace_dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nn = size_t(N) * N;
  const float scale = float(2.0 * dose / (double(N) * double(N)));
  // Coarse grid: the fields, the image and the adjoint transforms run on
  // nc >= 2C.  The image is interpolated exactly to N for the resist and the
  // loss; dL/dI enters the adjoint only through its frequencies below C in
  // magnitude (the products with the fields are cropped to the field band),
  // so it is low-passed to the 2C band and sampled on nc, times (N/nc)^2 for
  // the sums over nc^2 instead of N^2 points.  No product frequency aliases
  // into the field band on nc >= 2C, so the result is the full-grid one.
  const bool coarse = (int(prec) & LITHO_GRID_COARSE) && h->nc > 0 && interp_cols_supported(h->nc, N);
  const int NE = coarse ? h->nc : N, C2 = 2 * C;
  const float2* twe = coarse ? h->d_twc : h->d_tw;
  const float lp_scale = float((double(N) / NE) * (double(N) / NE));
  if (coarse) LITHO_TRY_CUDA(launch_blur_gain(taps, N, C2, L.gain, st));
  // a 1024-point coarse grid: the warp-per-row stage 2 writes the coarse image's row spectra itself
  const bool rows2 = coarse && h->d_tw32 && stage2_w32_supported(NE, C);
  // coarse grid: the row spectra of dL/dI on the 2C band, gp x N x 2C, in the image buffer (gp x N x N floats)
  // (the coarse grid is a power of two nc <= N/2 with 2C <= nc, so 2 x 2C floats fit in a row of N)
  if (coarse && 2 * C2 > N) {
    set_error("coarse grid band 2C = %d wider than half the grid (%d)", C2, N);
    return LITHO_EINVAL;
  }
  float2* qrows = reinterpret_cast<float2*>(L.img);
  // Groups of g clips: every launch covers the group's g x P planes (plane
  // i P + p is focus plane f0 + p of clip c0 + i; its fields follow the
  // plane's K kernels).
  for (int c0 = 0; c0 < b; c0 += G) {
    const int g = std::min(G, b - c0), gp = g * P;
    {
      ProfScope ps(kStageIltForward, st, 3);
      {
        const size_t c4 = size_t(g) * nn / 4;  // nn = N^2 with N >= 32: a multiple of 4
        const int blocks = int(std::min<size_t>((c4 + 255) / 256, 4096));
        k_sigmoid<<<blocks, 256, 0, st>>>(reinterpret_cast<const float4*>(theta_dev + c0 * nn), float(mask_steep),
                                          reinterpret_cast<float4*>(L.m), c4);
      }
      LITHO_TRY_CUDA(cudaGetLastError());
      LITHO_TRY_CUDA(launch_mask_spectrum(L.m, g, N, C, h->d_tw, L.rowbuf, L.mhat, st));
    }
    for (int f0 = 0; f0 < F; f0 += P) {
      const float2* phi = h->d_phi + size_t(f0) * K * C * C;
      const float* lam = h->d_lambda + size_t(f0) * K;
      {
        ProfScope ps(kStageIltForward, st, coarse ? (rows2 ? 5 : 6) : 5);
        LITHO_TRY_CUDA(launch_stage1_fft(L.mhat, phi, P * K, NE, C, twe, L.t1, st, g));
        LITHO_TRY_CUDA(launch_stage2_fft(L.t1, lam, K, NE, C, float(dose), twe, coarse ? L.ic : L.img, gp,
                                         (long long)K * NE * C, (long long)NE * NE, st, P, h->d_tw32, h->d_tw512,
                                         false, rows2 ? L.mid : nullptr, C2));
        if (coarse) {  // the blurred image straight from the interpolation (blur applied to the spectrum)
          if (!rows2) LITHO_TRY_CUDA(launch_mask_rows(L.ic, gp, NE, C2, twe, L.mid, st));
          LITHO_TRY_CUDA(launch_interp_cols(L.mid, gp, NE, N, C2, twe, h->d_tw, L.gain, L.big, st));
          // blurred rows, resist, dL/dI and its row spectra on the 2C band (into the free image
          // buffer), partial losses per row pair
          LITHO_TRY_CUDA(launch_resist_grad_rows(L.big, gp, N, C2, h->d_tw, target_dev + c0 * nn, P,
                                                 float(resist_steep), float(threshold), qrows, L.partial, st));
          k_reduce_loss<<<g, 1024, 0, st>>>(L.partial, P * N / 2, L.loss + c0, f0 > 0 ? 1 : 0);
        } else {
          LITHO_TRY_CUDA(launch_resist(L.img, gp, N, taps, float(threshold), L.blur, nullptr, st));
          k_resist_grad<<<dim3(kPartials, g), 256, 0, st>>>(L.blur, target_dev + c0 * nn, nn, P,
                                                           float(resist_steep), float(threshold), L.img, L.partial);
          LITHO_TRY_CUDA(cudaGetLastError());
          k_reduce_loss<<<g, 1024, 0, st>>>(L.partial, kPartials, L.loss + c0, f0 > 0 ? 1 : 0);
        }
        LITHO_TRY_CUDA(cudaGetLastError());
      }
      {
        ProfScope ps(kStageIltBackward, st, coarse ? 6 : 4);
        const float* gsrc = L.blur;
        if (coarse) {  // low-pass of g (x) q: the spectrum of q on the 2C band times the blur's transfer function
          LITHO_TRY_CUDA(launch_mask_cols(qrows, gp, N, C2, h->d_tw, L.spec, L.gain, true, st));
          LITHO_TRY_CUDA(launch_stage1_fft(L.spec, nullptr, gp, NE, C2, twe, L.mid, st));
          LITHO_TRY_CUDA(launch_band_rows_real(L.mid, gp, NE, C2, lp_scale, twe, L.ic, st));
          gsrc = L.ic;
        } else {
          LITHO_TRY_CUDA(launch_resist(L.img, gp, N, taps, float(threshold), L.blur, nullptr, st));
        }
        LITHO_TRY_CUDA(launch_adj_rows(NE, L.t1, lam, K, C, gsrc, twe, L.u, gp, P, st, h->d_tw512));
        LITHO_TRY_CUDA(launch_adj_cols(NE, L.u, phi, lam, C, twe, L.sk, gp * K, P * K, st));
        k_sum_planes<<<dim3(256, g), 256, 0, st>>>(L.sk, adj_col_splits(P * K), size_t(C) * C, L.s, f0 > 0 ? 1 : 0);
        LITHO_TRY_CUDA(cudaGetLastError());
      }
    }
    ProfScope ps(kStageIltBackward, st, 2);
    LITHO_TRY_CUDA(launch_stage1_fft(L.s, nullptr, g, N, C, h->d_tw, L.qf, st));
    LITHO_TRY_CUDA(launch_grad_rows(N, L.qf, C, scale, L.m, float(mask_steep), h->d_tw, grad_dev + c0 * nn, g,
                                    (long long)nn, st));
  }
  if (loss_host) {
    LITHO_TRY_CUDA(cudaMemcpyAsync(loss_host, L.loss, size_t(b) * sizeof(double), cudaMemcpyDeviceToHost, st));
    LITHO_TRY_CUDA(cudaStreamSynchronize(st));
  }
  return LITHO_OK;
}

litho_status litho_intensity_vjp_workspace_size(const litho_kernels* h, int b, size_t* full_bytes, size_t* min_bytes) {
  return litho_ilt_workspace_size(h, b, full_bytes, min_bytes);
}

litho_status litho_intensity_vjp(const litho_kernels* h, const float* mask_dev, int b, double dose,
                                 litho_precision prec, int f_first, int f_count, const float* upstream_dev,
                                 float* dm_dev, void* workspace_dev, size_t workspace_bytes, void* stream) {
  if (!h || !mask_dev || !dm_dev || !workspace_dev || b < 1) {
    set_error("null argument or b < 1");
    return LITHO_EINVAL;
  }
  if (f_first < 0 || f_count < 1 || f_first + f_count > h->n_focus || !std::isfinite(dose)) {
    set_error("focus planes [f_first, f_first + f_count) must lie in [0, n_focus); dose finite");
    return LITHO_EINVAL;
  }
  if ((int(prec) & ~LITHO_GRID_COARSE) != LITHO_PREC_FFT32) {
    set_error("litho_intensity_vjp implements the FP32 FFT path only (LITHO_PREC_FFT32, optionally | "
              "LITHO_GRID_COARSE)");
    return LITHO_EUNSUPPORTED;
  }
  if ((reinterpret_cast<uintptr_t>(workspace_dev) & 255) != 0) {
    set_error("workspace must be 256-byte aligned");
    return LITHO_EINVAL;
  }
  const int F = h->n_focus, K = h->k, N = h->n, C = h->crop;
  int P, G;
  if (!ilt_plan(h, b, f_count, workspace_bytes, &P, &G)) {
    set_error("workspace too small: %zu bytes given, at least %zu needed", workspace_bytes,
              ilt_layout(h, b, 1, 1, nullptr).bytes);
    return LITHO_ENOMEM;
  }
  // clips are grouped when their upstream planes follow one another: all
  // focus planes of each clip, or no upstream (ones)
  if (upstream_dev && !(P == F && f_first == 0)) G = 1;
  IltLayout L = ilt_layout(h, b, P, G, workspace_dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nn = size_t(N) * N;
  const float scale = float(2.0 * dose / (double(N) * double(N)));
  // coarse grid as in litho_ilt_grad: the upstream low-passed to the 2C band
  // and sampled on nc (no upstream: the closed form, on no grid)
  const bool coarse = (int(prec) & LITHO_GRID_COARSE) && h->nc > 0 && interp_cols_supported(h->nc, N);
  const int NE = coarse ? h->nc : N, C2 = 2 * C;
  const float2* twe = coarse ? h->d_twc : h->d_tw;
  const float lp_scale = float((double(N) / NE) * (double(N) / NE));
  ProfScope ps(kStageIltBackward, st, 1);
  for (int c0 = 0; c0 < b; c0 += G) {
    const int g = std::min(G, b - c0);
    LITHO_TRY_CUDA(launch_mask_spectrum(mask_dev + c0 * nn, g, N, C, h->d_tw, L.rowbuf, L.mhat, st));
    if (!upstream_dev) {  // dL/dI = 1 on every pixel of the selected planes: the closed form
      k_ones_adjoint<<<dim3(128, g), 256, 0, st>>>(L.mhat, h->d_phi + size_t(f_first) * K * C * C,
                                                   h->d_lambda + size_t(f_first) * K, f_count * K, size_t(C) * C,
                                                   float(double(N) * double(N)), L.s, 0);
      LITHO_TRY_CUDA(cudaGetLastError());
    }
    for (int f0 = f_first; upstream_dev && f0 < f_first + f_count; f0 += P) {
      const int p = std::min(P, f_first + f_count - f0);
      const float* up = upstream_dev + (size_t(c0) * F + f0) * nn;
      if (coarse) {
        LITHO_TRY_CUDA(launch_mask_spectrum(up, g * p, N, C2, h->d_tw, L.big, L.spec, st));
        LITHO_TRY_CUDA(launch_stage1_fft(L.spec, nullptr, g * p, NE, C2, twe, L.mid, st));
        LITHO_TRY_CUDA(launch_band_rows_real(L.mid, g * p, NE, C2, lp_scale, twe, L.ic, st));
        up = L.ic;
      }
      LITHO_TRY_CUDA(launch_stage1_fft(L.mhat, h->d_phi + size_t(f0) * K * C * C, p * K, NE, C, twe, L.t1, st, g));
      LITHO_TRY_CUDA(
          launch_adj_rows(NE, L.t1, h->d_lambda + size_t(f0) * K, K, C, up, twe, L.u, g * p, p, st, h->d_tw512));
      LITHO_TRY_CUDA(launch_adj_cols(NE, L.u, h->d_phi + size_t(f0) * K * C * C, h->d_lambda + size_t(f0) * K, C,
                                     twe, L.sk, g * p * K, p * K, st));
      k_sum_planes<<<dim3(256, g), 256, 0, st>>>(L.sk, adj_col_splits(p * K), size_t(C) * C, L.s,
                                                 f0 > f_first ? 1 : 0);
      LITHO_TRY_CUDA(cudaGetLastError());
    }
    LITHO_TRY_CUDA(launch_stage1_fft(L.s, nullptr, g, N, C, h->d_tw, L.qf, st));
    LITHO_TRY_CUDA(launch_grad_rows(N, L.qf, C, scale, nullptr, 0.f, h->d_tw, dm_dev + c0 * nn, g, (long long)nn,
                                    st));
  }
  return LITHO_OK;
}

}  // extern "C"
