// Column pass of the exact Fourier interpolation from a coarse grid (paper
// Eq. (4) evaluated on nc x nc, then resampled to N x N): for each crop
// column u of the row spectra R[p][y][u] of coarse images (y in [0, NC)),
//
//   S[v][u]  = NC^-2 sum_y R[y][u] e^{-2 pi i v y/NC},   v in [-C2/2, C2/2)
//   S'[v][u] = S[v][u] (1 + i gain[v] gain[u])          (with gain: blur channel)
//   Q[y][u]  = sum_v S'[v][u] e^{+2 pi i v y/N},        y in [0, N)
//
// in one kernel: the forward transform on NC, the crop, the scale and the
// blur channel, and the inverse transform on N, with the column staying in
// shared memory in between (one pass over the data instead of a forward
// column kernel writing the crop spectrum and an inverse column kernel
// reading it back).  Same arithmetic, in the same order, as those two
// kernels.  Thread layout as in stage 1: column w = tid mod W, transform
// thread t = tid / W, so the loads of R and the stores of Q cover W adjacent
// columns of 32/W rows per warp.
#include "fft_common.cuh"
#include "litho_internal.h"

namespace litho {

namespace {

template <int N, int W>
struct InterpShape {
  static constexpr int LD = (PadLen<N>::value + 15) / 16 * 16 + 16 / W;
};

template <int NC, int N, int W>
__global__ void __launch_bounds__(Plan<N>::NT * W)
    k_interp_cols(const float2* __restrict__ rspec, int c2, const float2* __restrict__ tw_nc_g,
                  const float2* __restrict__ tw_n_g, const float* __restrict__ gain, float2* __restrict__ q) {
  constexpr int NT = Plan<N>::NT, NTC = Plan<NC>::NT, T = NT * W, LD = InterpShape<N, W>::LD;
  constexpr bool BANDED = 2 * NC <= N;  // |v| < C2/2 <= NC/2 <= N/4
  static_assert(NTC <= NT, "the coarse transform runs on a subset of the threads");
  extern __shared__ float4 smem_raw[];
  float2* smem = reinterpret_cast<float2*>(smem_raw);
  float2* tw_n = smem;
  float2* tw_c = smem + N;
  float2* buf = smem + N + NC;
  const int tid = threadIdx.x, g = tid % W, t = tid / W;
  const int u0 = blockIdx.x * W, p = blockIdx.y, half = c2 / 2;
  for (int i = tid; i < N; i += T) tw_n[i] = tw_n_g[i];
  for (int i = tid; i < NC; i += T) tw_c[i] = tw_nc_g[i];
  __syncthreads();
  float2* col = buf + g * LD;
  // forward transform over y on NC, shared by all NT threads of the column
  // (a pass with fewer butterflies than threads leaves the rest idle)
  const float2* src = rspec + (size_t)p * NC * c2 + u0 + g;
  auto load_c = [&](int y) { return __ldg(src + (size_t)y * c2); };
  fft_load_smem<NC, -1, decltype(load_c), false, NT>(col, tw_c, t, load_c);
  // crop, scale, blur channel, and the inverse transform over v on N
  const float scale = 1.0f / (float(NC) * float(NC));
  const float gu = gain ? __ldg(gain + u0 + g) : 0.f;
  auto load_f = [&](int, int r, int idx) {
    const int v = r < Plan<N>::R[0] / 2 ? idx : idx - N;  // first pass: idx < N/2 exactly when r < R/2
    if (v < -half || v >= half) return make_float2(0.f, 0.f);
    float2 s = col[pad16(v < 0 ? v + NC : v)];
    s = make_float2(s.x * scale, s.y * scale);
    if (gain) {
      const float gg = __ldg(gain + v + half) * gu;
      s = make_float2(fmaf(-gg, s.y, s.x), fmaf(gg, s.x, s.y));
    }
    return s;
  };
  float2* dst = q + (size_t)p * N * c2 + u0 + g;
  auto use = [&](int, int, int y, float2 v) { dst[(size_t)y * c2] = v; };
  fft_load_use<N, +1, decltype(load_f), decltype(use), BANDED>(col, tw_n, t, load_f, use);
}

template <int NC, int N>
cudaError_t interp_cols_n(const float2* rspec, int planes, int c2, const float2* tw_nc, const float2* tw_n,
                          const float* gain, float2* q, cudaStream_t st) {
  constexpr int W = 8;
  if (c2 % W != 0 || c2 > NC) return cudaErrorInvalidValue;
  const size_t sm = sizeof(float2) * (size_t(N) + NC + size_t(W) * InterpShape<N, W>::LD);
  cudaError_t e = smem_attrs(k_interp_cols<NC, N, W>, sm);
  if (e != cudaSuccess) return e;
  k_interp_cols<NC, N, W><<<dim3(c2 / W, planes), Plan<N>::NT * W, sm, st>>>(rspec, c2, tw_nc, tw_n, gain, q);
  return cudaGetLastError();
}

}  // namespace

bool interp_cols_supported(int nc, int n) {
  if (nc == 896) return n == 1024 || n == 2048;
  return nc >= 32 && (nc == n / 2 || nc == n / 4 || nc == n / 8) && n >= 64 && n <= 2048;
}

cudaError_t launch_interp_cols(const float2* rspec, int planes, int nc, int n, int c2, const float2* tw_nc,
                               const float2* tw_n, const float* gain, float2* q, cudaStream_t st) {
#define IC(NC, N) \
  if (nc == NC && n == N) return interp_cols_n<NC, N>(rspec, planes, c2, tw_nc, tw_n, gain, q, st);
  IC(1024, 2048) IC(512, 2048) IC(256, 2048) IC(896, 2048)
  IC(512, 1024) IC(256, 1024) IC(128, 1024) IC(896, 1024)
  IC(256, 512) IC(128, 512) IC(64, 512)
  IC(128, 256) IC(64, 256) IC(32, 256)
  IC(64, 128) IC(32, 128)
  IC(32, 64)
#undef IC
  return cudaErrorInvalidValue;
}

}  // namespace litho
