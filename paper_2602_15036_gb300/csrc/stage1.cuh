// Stage 1 of the SOCS evaluation (paper Eq. (4)): band multiply and inverse
// transform over the y frequency, T_j[y][c] = sum_v mhat[v][c] Phi_j[v][c] e^{+2 pi i v y/N},
// for a block of W crop columns c and a run of kernels j.
//
// A CTA keeps the twiddle table in shared memory and loops over a run of kernels;
// the next kernel's Phi block is copied in with cp.async while the current
// block's W column transforms run.  The FP32 output takes one block buffer,
// refilled as soon as the first pass (the only one that reads the block) is
// done, so that two CTAs fit an SM's shared memory; the split 16-bit output
// keeps two buffers.  The band multiply happens in
// the first pass's load: the mask-spectrum values a thread multiplies are
// the same for every kernel, so they are loaded once into registers.
// Without kernels (phi == NULL) each j transforms its own spectrum mhat[j].
//
// Thread layout: column w = tid mod W, transform thread t = tid / W, so a
// warp holds 32/W consecutive t of all W columns.  In the last pass a warp's
// outputs for one element are then 32/W rows x W adjacent columns: whole
// 32-byte sectors for W = 4, stored straight from registers (FP32 output).
// The split 16-bit output for the tensor-core path packs a row's W columns
// in one thread and goes through shared memory.
//
// With kernels, one launch can image several clips (grid x = clip, the
// fastest-varying block index): the CTAs of all clips that need the same Phi
// block run side by side, so each block comes from DRAM once and from L2
// for the other clips.  Clip i writes j + i nk.  The row-wise (split 16-bit)
// output swaps the two: its W columns fill only part of each 32-byte sector
// of an operand row, so the column blocks that share those sectors are made
// the fastest index and run side by side, and their pieces meet in L2.
#pragma once

#include <algorithm>

#include "fft_common.cuh"

namespace litho {

__device__ __forceinline__ void cp_async16_cg(void* smem_dst, const void* gmem_src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Shared memory of a CTA: the twiddle table, W column transforms at stride LD
// (the padded length rounded up to 16 complex values plus 16/W, so that a
// half-warp of 16/W transform threads x W columns touches 16 different bank
// pairs) and two operand blocks [crop][W] in the operand's own row-major
// order (a row's W values are one or more whole 16-byte copies; a half-warp
// reading rows c..c+16/W-1 of all W columns again hits 16 bank pairs).
// Columns per CTA: as many as fit one CTA of at most 512 threads, since a
// warp's final-pass stores then cover longer pieces of each output row (W = 8:
// 64-byte pieces; measured faster than W = 4 at 2 CTAs per SM for N = 1024).
template <int N>
struct Stage1W {
  static constexpr int W = Plan<N>::NT <= 64 ? 8 : 4;
};

template <int N, int W>
struct Stage1Shape {
  static_assert(W % 2 == 0, "W even: rows of whole 16-byte pieces");
  static constexpr int LD = (PadLen<N>::value + 15) / 16 * 16 + 16 / W;
  static size_t smem_elems(int crop, int buffers) {
    return size_t(N) + size_t(W) * LD + size_t(buffers) * W * crop;
  }
};

// Block buffers and CTAs per SM the launch bounds ask for: the FP32 output
// single-buffers its Phi block and runs two CTAs per SM.
template <class Out>
struct Stage1Pipe {
  static constexpr int kBuffers = Out::kRowWise ? 2 : 1;
  static constexpr int kMinBlocks = Out::kRowWise ? 1 : 2;
};

template <int N, int W, class Out, bool BANDED>
__global__ void __launch_bounds__(Plan<N>::NT * W, Stage1Pipe<Out>::kMinBlocks)
    k_stage1_cols(const float2* __restrict__ mhat, const float2* __restrict__ phi, int crop, int nk, int jb,
                  const float2* __restrict__ tw_g, Out out) {
  constexpr int NT = Plan<N>::NT, LD = Stage1Shape<N, W>::LD, T = W * NT;
  constexpr int R0 = Plan<N>::R[0], NB0 = N / R0;  // first pass: radix and butterflies
  static_assert(PassShape<N, NT, R0>::PER == 1, "one first-pass butterfly per thread");
  extern __shared__ float4 smem_raw[];
  float2* smem = reinterpret_cast<float2*>(smem_raw);
  float2* tw = smem;
  float2* buf = smem + N;
  float2* const blk0 = buf + W * LD;  // Phi (or spectrum) blocks [crop][W], double-buffered
  auto blk = [&](int s) { return blk0 + s * W * crop; };
  const int clip = Out::kRowWise ? blockIdx.y : blockIdx.x, cblk = Out::kRowWise ? blockIdx.x : blockIdx.y;
  const int tid = threadIdx.x, u0 = cblk * W, half = crop / 2;
  const int j0 = blockIdx.z * jb, j1 = min(nk, j0 + jb), jofs = clip * nk;
  if (j0 >= j1) return;
  mhat += (size_t)clip * crop * crop;
  load_twiddles<N>(tw, tw_g);
  const float2* src_base = phi ? phi : mhat;  // the per-j operand
  auto issue = [&](int j, float2* dst) {  // W/2 16-byte pieces per row
    const float2* src = src_base + (size_t)j * crop * crop + u0;
    for (int i = tid; i < crop * (W / 2); i += T) {
      const int cv = i / (W / 2), part = i % (W / 2);
      cp_async16_cg(dst + 2 * i, src + (size_t)cv * crop + 2 * part);
    }
    cp_async_commit();
  };
  issue(j0, blk(0));
  const int g = tid % W, t = tid / W;
  auto band_row = [&](int idx) { return (idx < N / 2 ? idx : idx - N) + half; };  // crop row of index idx
  float2 mreg[R0];  // mask spectrum at this thread's first-pass inputs (column u0 + g)
#pragma unroll
  for (int r = 0; r < R0; ++r) {
    const int c = band_row(t + r * NB0);
    const bool zero = !phi || t >= NB0 || c < 0 || c >= crop || (BANDED && r >= R0 / 4 && r < 3 * R0 / 4);
    mreg[r] = zero ? make_float2(0.f, 0.f) : __ldg(mhat + (size_t)c * crop + u0 + g);
  }
  constexpr bool kSingle = Stage1Pipe<Out>::kBuffers == 1;
  for (int j = j0; j < j1; ++j) {
    const int s = kSingle ? 0 : (j - j0) & 1;
    if (!kSingle && j + 1 < j1) {
      issue(j + 1, blk(s ^ 1));
      cp_async_wait_one();
    } else {
      cp_async_wait_all();
    }
    // Block j (and, first time round, tw) visible to all threads; every thread
    // has finished transform j - 1, so buf and the other Phi buffer are free.
    __syncthreads();
    const float2* b = blk(s) + g;
    // single buffer: the first pass has read block j in every thread, so block j + 1 may land
    auto refill = [&]() {
      if (kSingle && j + 1 < j1) issue(j + 1, blk(0));
    };
    auto load = [&](int, int r, int idx) {
      const int c = (r < R0 / 2 ? idx : idx - N) + half;  // idx < N/2 exactly when r < R0/2
      if (c < 0 || c >= crop) return make_float2(0.f, 0.f);
      return phi ? cmul(mreg[r], b[c * W]) : b[c * W];
    };
    if constexpr (Out::kRowWise) {
      fft_load_smem<N, +1, decltype(load), BANDED>(buf + g * LD, tw, t, load);
      // one thread per output row writes the block's W consecutive columns
      for (int y = tid; y < N; y += T) {
        float2 v[W];
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = buf[w * LD + pad16(y)];
        out.template store_row<W>(jofs + j, y, u0, v);
      }
    } else {
      float2* const col = out.column(jofs + j, u0 + g);  // element y at col[y crop]
      auto use = [&](int, int, int y, float2 v) { col[y * crop] = v; };
      fft_load_use<N, +1, decltype(load), decltype(use), BANDED>(buf + g * LD, tw, t, load, use, refill);
    }
  }
}

template <int N, int W, class Out, bool BANDED>
cudaError_t launch_stage1_cols_t(const float2* mhat, const float2* phi, int nk, int crop, const float2* tw, Out out,
                                 cudaStream_t st, int clips) {
  // Kernels per CTA: runs of kernels as long as possible (each CTA loads its
  // twiddles and mask values once and starts its copy pipeline once), split
  // so that the CTAs fill whole waves: the fewest waves x (kernels per CTA
  // + half a kernel of set-up).
  // (One run per CTA block leaves, e.g., 448 CTAs on 304 slots: a second wave
  // half empty for a whole CTA's time.)
  static int sms = 0;  // the same GPU model throughout a process; a racing first call stores the same value
  if (!sms) {
    int dev = 0, v = 0;
    sms = cudaGetDevice(&dev) == cudaSuccess &&
                  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0
              ? v
              : 152;
  }
  const long long ctas = (long long)clips * (crop / W), slots = (long long)Stage1Pipe<Out>::kMinBlocks * sms;
  int jblocks = 1;
  long long best = -1;
  for (int jb = 1; jb <= std::min(nk, 32); ++jb) {
    const long long per = (nk + jb - 1) / jb;
    const long long waves = (ctas * ((nk + per - 1) / per) + slots - 1) / slots;
    const long long cost = waves * (2 * per + 1);  // half a kernel's time per CTA for its set-up
    if (best < 0 || cost < best) {
      best = cost;
      jblocks = jb;
    }
  }
  const int JB = (nk + jblocks - 1) / jblocks;
  const size_t sm = sizeof(float2) * Stage1Shape<N, W>::smem_elems(crop, Stage1Pipe<Out>::kBuffers);
  cudaError_t e = smem_attrs(k_stage1_cols<N, W, Out, BANDED>, sm);
  if (e != cudaSuccess) return e;
  const dim3 grid = Out::kRowWise ? dim3(crop / W, clips, (nk + JB - 1) / JB) : dim3(clips, crop / W, (nk + JB - 1) / JB);
  k_stage1_cols<N, W, Out, BANDED><<<grid, Plan<N>::NT * W, sm, st>>>(mhat, phi, crop, nk, JB, tw, out);
  return cudaGetLastError();
}

// W columns per CTA (a divisor of 32; crop is a multiple of 32).  `clips`
// spectra mhat[clips][C][C] share the kernels (clips must be 1 without them).
// A crop of at most N/2 takes the banded first pass.
template <int N, int W, class Out>
cudaError_t launch_stage1_cols(const float2* mhat, const float2* phi, int nk, int crop, const float2* tw, Out out,
                               cudaStream_t st, int clips = 1) {
  if (clips < 1 || (!phi && clips != 1)) return cudaErrorInvalidValue;
  if (2 * crop <= N) return launch_stage1_cols_t<N, W, Out, true>(mhat, phi, nk, crop, tw, out, st, clips);
  return launch_stage1_cols_t<N, W, Out, false>(mhat, phi, nk, crop, tw, out, st, clips);
}

}  // namespace litho
