// Stage 1 of the SOCS evaluation (paper Eq. (4)): band multiply and inverse
// transform over the y frequency, T_j[y][c] = sum_v mhat[v][c] Phi_j[v][c] e^{+2 pi i v y/N},
// for a block of W crop columns c and a run of kernels j.
//
// A CTA keeps its column block of the mask spectrum and the twiddle table in
// shared memory and loops over JB kernels; the next kernel's Phi block is
// copied in with cp.async (two buffers) while the current block's W column
// transforms run, and the band multiply happens inside the first pass's load.
// Without kernels (phi == NULL) each j transforms its own spectrum mhat[j].
// The output policy `Out` stores element (j, y, c): FP32 complex for the FFT
// path, split 16-bit hi/lo rows for the tensor-core path.
//
// With kernels, one launch can image several clips (grid x = clip, the
// fastest-varying block index): the CTAs of all clips that need the same Phi
// block run side by side, so each block comes from DRAM once and from L2
// for the other clips.  Clip i writes j + i nk.
#pragma once

#include "fft_common.cuh"

namespace litho {

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Strides for a block of W columns: each column's padded transform, rounded
// up to 16 complex values plus 16/W, and the compact band buffers crop + 16/W,
// so that the cooperative copies (w fastest) hit 16 different bank pairs.
template <int N, int W>
struct Stage1Shape {
  static constexpr int LD = (PadLen<N>::value + 15) / 16 * 16 + 16 / W;
  static int bld(int crop) { return crop + 16 / W; }
  static size_t smem_elems(int crop) { return size_t(N) + size_t(W) * LD + 3 * size_t(W) * bld(crop); }
};

template <int N, int W, class Out, bool BANDED>
__global__ void __launch_bounds__(Plan<N>::NT * W)
    k_stage1_cols(const float2* __restrict__ mhat, const float2* __restrict__ phi, int crop, int nk, int jb,
                  const float2* __restrict__ tw_g, Out out) {
  constexpr int NT = Plan<N>::NT, LD = Stage1Shape<N, W>::LD, T = W * NT;
  extern __shared__ float2 smem[];
  const int bld = crop + 16 / W;
  float2* tw = smem;
  float2* buf = smem + N;
  float2* const blk0 = buf + W * LD;  // Phi (or spectrum) blocks, double-buffered: blk0 + s W bld
  auto blk = [&](int s) { return blk0 + s * W * bld; };
  float2* msk = buf + W * LD + 2 * W * bld;                 // mask-spectrum block (with kernels)
  const int tid = threadIdx.x, u0 = blockIdx.y * W, half = crop / 2;
  const int j0 = blockIdx.z * jb, j1 = min(nk, j0 + jb), jofs = blockIdx.x * nk;
  if (j0 >= j1) return;
  mhat += (size_t)blockIdx.x * crop * crop;
  load_twiddles<N>(tw, tw_g);
  const float2* src_base = phi ? phi : mhat;  // the per-j operand
  auto issue = [&](int j, float2* dst) {
    const float2* src = src_base + (size_t)j * crop * crop + u0;
    for (int i = tid; i < crop * W; i += T) {
      const int cv = i / W, w = i % W;
      cp_async8(dst + w * bld + cv, src + (size_t)cv * crop + w);
    }
    cp_async_commit();
  };
  if (phi) {
    for (int i = tid; i < crop * W; i += T) {
      const int cv = i / W, w = i % W;
      msk[w * bld + cv] = __ldg(mhat + (size_t)cv * crop + u0 + w);
    }
  }
  issue(j0, blk(0));
  const int g = tid / NT, t = tid % NT;
  for (int j = j0; j < j1; ++j) {
    const int s = (j - j0) & 1;
    if (j + 1 < j1) {
      issue(j + 1, blk(s ^ 1));
      cp_async_wait_one();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();  // block j (and, first time round, msk and tw) visible to all threads
    const float2* b = blk(s) + g * bld;
    const float2* m = msk + g * bld;
    auto load = [&](int idx) {
      const int c = (idx < N / 2 ? idx : idx - N) + half;
      if (c < 0 || c >= crop) return make_float2(0.f, 0.f);
      return phi ? cmul(m[c], b[c]) : b[c];
    };
    fft_load_smem<N, +1, decltype(load), BANDED>(buf + g * LD, tw, t, load);
    if constexpr (Out::kRowWise) {
      // one thread per output row writes the block's W consecutive columns
      for (int y = tid; y < N; y += T) {
        float2 v[W];
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = buf[w * LD + pad16(y)];
        out.template store_row<W>(jofs + j, y, u0, v);
      }
    } else {
      // consecutive threads write consecutive columns of a row (full sectors per warp)
      for (int i = tid; i < N * W; i += T) {
        const int y = i / W, w = i % W;
        out.store(jofs + j, y, u0 + w, buf[w * LD + pad16(y)]);
      }
    }
    __syncthreads();  // copy-out done before the next transform overwrites buf
  }
}

template <int N, int W, class Out, bool BANDED>
cudaError_t launch_stage1_cols_t(const float2* mhat, const float2* phi, int nk, int crop, const float2* tw, Out out,
                                 cudaStream_t st, int clips) {
  constexpr int JB = 8;
  const size_t sm = sizeof(float2) * Stage1Shape<N, W>::smem_elems(crop);
  cudaError_t e = smem_attrs(k_stage1_cols<N, W, Out, BANDED>, sm);
  if (e != cudaSuccess) return e;
  k_stage1_cols<N, W, Out, BANDED><<<dim3(clips, crop / W, (nk + JB - 1) / JB), Plan<N>::NT * W, sm, st>>>(
      mhat, phi, crop, nk, JB, tw, out);
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
