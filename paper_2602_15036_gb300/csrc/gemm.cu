// Tensor-core (tcgen05) DFT-GEMM path for the SOCS image, paper Eq. (4).
//
// For one focus plane, E_k(y, x) = sum_c T_k(y, c) W(c, x) with the stage-1
// field T_k (rows y, crop columns c) and the inverse-DFT matrix
// W(c, x) = exp(+2 pi i u_c x / N), u_c = c - C/2.  Written over real
// operands with Ar = Re T, Ai = Im T, Wr = cos, Wi = sin.
//
// Split modes use Gauss's three-multiplication complex product: with the sums
// As = Ar + Ai and Ws = Wr + Wi,
//   D1 = Ar Wr^T,  D2 = Ai Wi^T,  D3 = As Ws^T,
//   Re E = D1 - D2,  Im E = D3 - D1 - D2,
// three real products per complex multiply-add instead of four (9 MMAs per
// K step with the hi/lo split instead of 12).  The plain 16-bit modes keep
// the four-product form, D3 = Ar Wi^T + Ai Wr^T and Im E = D3: their operands
// carry 8 to 11 significand bits, and the cancellation in D3 - D1 - D2 would
// enlarge their error.  Either way I(y, x) += lam_k (Re E^2 + Im E^2); the
// three accumulators live in TMEM (3 x 128 fp32 columns).  The k loop runs
// inside the CTA: the epilogue warps fold each kernel's |E|^2 into
// registers, so I is written once per tile.
//
// Operand layout in global memory (16-bit elements, K-major): the contraction
// index c is cut into chunks of 32 complex values stored as one 64-element
// (128-byte) row segment [Re 32 | Im 32].  A (hi and lo): [plane * K + k][y][2C],
// B (hi and lo): [x][2C] (same chunking, cos | sin).  The sums are stored the
// same way with hi and lo side by side: AS = [As_hi 32 | As_lo 32] per chunk,
// BS = [Ws_hi 32 | Ws_lo 32].  TMA loads 128-row x 64-element boxes with
// 128-byte swizzling, which is the canonical K-major SWIZZLE_128B layout that
// tcgen05.mma reads through shared-memory descriptors; the four 16-element K
// steps of a chunk sit at byte offsets 0, 32 (first half: Re, or the hi sums)
// and 64, 96 (second half: Im, or the lo sums).
//
// Precision modes: BF16 / FP16 (one product), BF16X3 and FP16X3
// (operands split into hi + lo, three products hi.hi + hi.lo + lo.hi; FP16
// stage-1 fields are scaled per kernel by a power of two so that hi and lo
// stay in the normal range; plain FP16 is scaled the same way).  FP32
// accumulation throughout.
//
// Kernel structure: persistent, one CTA per SM (192 KB shared memory ring:
// two stages of six tiles in the split modes, six stages of two tiles in the
// plain ones; all 512 TMEM columns), warp 0 = TMA producer, warp 1 = MMA
// issuer (one thread), warps 2..9 = epilogue.  Every mbarrier wait is bounded: past ~2 s it records
// an error code in a device flag, the CTA drains its own copies and MMAs with
// bounded waits, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "fft_common.cuh"
#include "gemm.h"
#include "stage1.cuh"

namespace litho {

namespace {

constexpr int BM = 128;               // rows (y) per tile = UMMA M
constexpr int XT = 128;               // x per tile = UMMA N
constexpr int CH = 32;                // complex values per chunk
constexpr int KE = 2 * CH;            // 16-bit elements per chunk row (128 bytes)
constexpr int TILE_BYTES = BM * KE * 2;  // 16 KB (A and B boxes are both 128 x 64)
constexpr int RING_BYTES = 12 * TILE_BYTES;  // 192 KB of pipeline stages
constexpr int MAX_STAGES = 6;
// Tiles of a stage: split modes A_hi, A_lo, AS, B_hi, B_lo, BS (2 stages);
// plain modes A_hi, B_hi (6 stages).
constexpr int TILES_SPLIT = 6, TILES_PLAIN = 2;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;
constexpr int SMEM_BYTES = RING_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr int GROUP_CLIPS = 4;        // clips per GEMM launch
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

enum Mode { kBF16 = 0, kBF16X3 = 1, kFP16X3 = 2, kFP16 = 3, kModes = 4 };

int mode_of(litho_precision p) {
  return p == LITHO_PREC_BF16 ? kBF16 : p == LITHO_PREC_BF16X3 ? kBF16X3 : p == LITHO_PREC_FP16 ? kFP16 : kFP16X3;
}
__host__ __device__ constexpr bool is_split(int m) { return m == kBF16X3 || m == kFP16X3; }
__host__ __device__ constexpr bool is_fp16(int m) { return m == kFP16X3 || m == kFP16; }

// ---- PTX helpers ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// K-major, 128-byte-swizzled shared-memory matrix descriptor (tcgen05): start
// address >> 4, leading-dimension offset (unused for this layout) 16 B, stride
// between 8-row groups 1024 B, descriptor version 1, swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, A/B format (0 fp16,
// 1 bf16), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int fmt, int m, int n) {
  return (1u << 4) | (uint32_t(fmt) << 7) | (uint32_t(fmt) << 10) | (uint32_t(n >> 3) << 17) |
         (uint32_t(m >> 4) << 24);
}

struct GemmParams {
  int n, nk, n_focus, planes, tiles_y, tiles_x, chunks, split, fmt;
  const float* lamp;  // [F][K] lambda / scale^2
  float dose;
  float* img;         // [planes][n][n]
  int* err;
};

// Bounded wait: true when the phase completed; false after the limit or
// when another role already gave up (abort flag in shared memory).
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err,
                                         int code, long long limit = kWaitCycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      atomicExch(err, code);
      return false;
    }
  }
  return true;
}

// Self-test of the bounded wait: one barrier that nothing ever arrives on.
// The wait must give up after `limit` cycles, record `code` and return.
__global__ void k_wait_selftest(int* err, long long limit, int code) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) wait_bar(smem_u32(&bar), 0, &abort_flag, err, code, limit);
}

__global__ void __launch_bounds__(THREADS, 1)
    k_dft_gemm(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
               const __grid_constant__ CUtensorMap ta_s, const __grid_constant__ CUtensorMap tb_hi,
               const __grid_constant__ CUtensorMap tb_lo, const __grid_constant__ CUtensorMap tb_s, GemmParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RING_BYTES);
  // bars: full[MAX_STAGES], empty[MAX_STAGES], acc_full, acc_empty, drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * MAX_STAGES + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + MAX_STAGES);
  const uint32_t acc_full = smem_u32(bars + 2 * MAX_STAGES), acc_empty = smem_u32(bars + 2 * MAX_STAGES + 1);
  const uint32_t drain = smem_u32(bars + 2 * MAX_STAGES + 2);
  // stage geometry of this mode (uniform across the grid)
  const int tiles = p.split ? TILES_SPLIT : TILES_PLAIN;
  const int STAGES = RING_BYTES / (tiles * TILE_BYTES);
  const int STAGE_BYTES = tiles * TILE_BYTES;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, EPI_WARPS);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int tiles_per_plane = p.tiles_y * p.tiles_x;
  const int total = p.planes * tiles_per_plane;
  const uint32_t tx_bytes = STAGE_BYTES;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
        const int plane = t / tiles_per_plane, rem = t % tiles_per_plane;
        const int yt = rem / p.tiles_x, xt = rem % p.tiles_x;
        const float* lam = p.lamp + (plane % p.n_focus) * p.nk;
        for (int k = 0; k < p.nk && ok; ++k) {
          if (lam[k] == 0.f) continue;
          const int arow = (plane * p.nk + k) * p.n + yt * BM;
          for (int ch = 0; ch < p.chunks; ++ch, ++it) {
            const int s = it % STAGES;
            const uint32_t use = it / STAGES;
            if (!wait_bar(empty0 + 8 * s, (use & 1) ^ 1, abort_flag, p.err, 1)) {
              ok = false;
              break;
            }
            const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
            mbar_expect_tx(full0 + 8 * s, tx_bytes);
            if (p.split) {
              tma_load_2d(base, &ta_hi, full0 + 8 * s, ch * KE, arow);
              tma_load_2d(base + TILE_BYTES, &ta_lo, full0 + 8 * s, ch * KE, arow);
              tma_load_2d(base + 2 * TILE_BYTES, &ta_s, full0 + 8 * s, ch * KE, arow);
              tma_load_2d(base + 3 * TILE_BYTES, &tb_hi, full0 + 8 * s, ch * KE, xt * XT);
              tma_load_2d(base + 4 * TILE_BYTES, &tb_lo, full0 + 8 * s, ch * KE, xt * XT);
              tma_load_2d(base + 5 * TILE_BYTES, &tb_s, full0 + 8 * s, ch * KE, xt * XT);
            } else {
              tma_load_2d(base, &ta_hi, full0 + 8 * s, ch * KE, arow);
              tma_load_2d(base + TILE_BYTES, &tb_hi, full0 + 8 * s, ch * KE, xt * XT);
            }
          }
        }
      }
      // drain: the last use of every stage must have landed before the CTA exits
      for (int d = 0; d < STAGES && it > 0; ++d) {
        const uint32_t j = it - 1 - d;
        if ((int)j < 0 || j >= it) break;
        const int s = j % STAGES;
        const long long t0 = clock64();
        while (!mbar_try_wait(full0 + 8 * s, (j / STAGES) & 1) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(p.fmt, BM, XT);
      const uint32_t d1 = tmem, d2 = tmem + 128, d3 = tmem + 256;
      uint32_t it = 0, acc_it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
        const int plane = t / tiles_per_plane;
        const float* lam = p.lamp + (plane % p.n_focus) * p.nk;
        for (int k = 0; k < p.nk && ok; ++k) {
          if (lam[k] == 0.f) continue;
          if (!wait_bar(acc_empty, (acc_it & 1) ^ 1, abort_flag, p.err, 2)) {
            ok = false;
            break;
          }
          tc_fence_after();
          for (int ch = 0; ch < p.chunks; ++ch, ++it) {
            const int s = it % STAGES;
            if (!wait_bar(full0 + 8 * s, (it / STAGES) & 1, abort_flag, p.err, 3)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
            if (p.split) {
              const uint64_t ahi = sdesc_sw128(base), alo = sdesc_sw128(base + TILE_BYTES);
              const uint64_t as = sdesc_sw128(base + 2 * TILE_BYTES), bhi = sdesc_sw128(base + 3 * TILE_BYTES);
              const uint64_t blo = sdesc_sw128(base + 4 * TILE_BYTES), bs = sdesc_sw128(base + 5 * TILE_BYTES);
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                // byte offsets >> 4: first half (Re, or the hi sums), second half (Im, or the lo sums)
                const uint64_t h1 = uint64_t(2 * ks), h2 = uint64_t(4 + 2 * ks);
                const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
                // Gauss: D1 += Ar Wr ; D2 += Ai Wi ; D3 += As Ws, each as hi.hi + hi.lo + lo.hi
                umma_f16(d1, ahi + h1, bhi + h1, idesc, first);
                umma_f16(d1, ahi + h1, blo + h1, idesc, 1u);
                umma_f16(d1, alo + h1, bhi + h1, idesc, 1u);
                umma_f16(d2, ahi + h2, bhi + h2, idesc, first);
                umma_f16(d2, ahi + h2, blo + h2, idesc, 1u);
                umma_f16(d2, alo + h2, bhi + h2, idesc, 1u);
                umma_f16(d3, as + h1, bs + h1, idesc, first);
                umma_f16(d3, as + h1, bs + h2, idesc, 1u);
                umma_f16(d3, as + h2, bs + h1, idesc, 1u);
              }
            } else {
              const uint64_t ahi = sdesc_sw128(base), bhi = sdesc_sw128(base + TILE_BYTES);
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                const uint64_t re = uint64_t(2 * ks), im = uint64_t(4 + 2 * ks);
                const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
                // D1 += Ar Wr ; D2 += Ai Wi ; D3 += Ar Wi + Ai Wr
                umma_f16(d1, ahi + re, bhi + re, idesc, first);
                umma_f16(d2, ahi + im, bhi + im, idesc, first);
                umma_f16(d3, ahi + re, bhi + im, idesc, first);
                umma_f16(d3, ahi + im, bhi + re, idesc, 1u);
              }
            }
            umma_commit(empty0 + 8 * s);  // frees the stage once these MMAs complete
          }
          if (!ok) break;
          umma_commit(acc_full);  // accumulator of kernel k complete
          ++acc_it;
        }
      }
      // drain outstanding MMAs before the CTA can release TMEM
      umma_commit(drain);
      const long long t0 = clock64();
      while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else {
    // ---------------- epilogue ----------------
    const int e = warp - 2, q = warp % 4, half = e / 4;
    const uint32_t lane_base = tmem + (uint32_t(q * 32) << 16);
    uint32_t acc_it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
      const int plane = t / tiles_per_plane, rem = t % tiles_per_plane;
      const int yt = rem / p.tiles_x, xt = rem % p.tiles_x;
      const float* lam = p.lamp + (plane % p.n_focus) * p.nk;
      float acc[64];
#pragma unroll
      for (int i = 0; i < 64; ++i) acc[i] = 0.f;
      for (int k = 0; k < p.nk; ++k) {
        const float l = lam[k];
        if (l == 0.f) continue;
        if (!wait_bar(acc_full, acc_it & 1, abort_flag, p.err, 4)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const uint32_t col = half * 64 + cc * 16;
          float a[16], b[16], c[16];
          tmem_ld16(lane_base + col, a);
          tmem_ld16(lane_base + 128 + col, b);
          tmem_ld16(lane_base + 256 + col, c);
          tmem_wait_ld();
          if (p.split) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float re = a[i] - b[i], im = c[i] - (a[i] + b[i]);
              acc[cc * 16 + i] = fmaf(l, fmaf(re, re, im * im), acc[cc * 16 + i]);
            }
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float re = a[i] - b[i];
              acc[cc * 16 + i] = fmaf(l, fmaf(re, re, c[i] * c[i]), acc[cc * 16 + i]);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);
        ++acc_it;
      }
      if (!ok) break;
      const int row = yt * BM + q * 32 + lane;
      float4* out = reinterpret_cast<float4*>(p.img + ((size_t)plane * p.n + row) * p.n + xt * XT + half * 64);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        out[i] = make_float4(p.dose * acc[4 * i], p.dose * acc[4 * i + 1], p.dose * acc[4 * i + 2],
                             p.dose * acc[4 * i + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---- stage 1 for the GEMM path: band multiply + inverse transform over v, written as split 16-bit A ---
// 16-bit bit patterns of the hi part and the rounded remainder (lo; 0 for the
// one-product modes).  fp16 values are scaled by the kernel's power of two.
template <int MODE>
__device__ __forceinline__ void split16(float x, float scale, uint32_t& h, uint32_t& l) {
  if (MODE == kFP16X3 || MODE == kFP16) {
    const float xs = x * scale;
    const __half hh = __float2half_rn(xs);
    h = __half_as_ushort(hh);
    l = MODE == kFP16X3 ? __half_as_ushort(__float2half_rn(xs - __half2float(hh))) : 0u;
  } else {
    const __nv_bfloat16 hh = __float2bfloat16_rn(x);
    h = __bfloat16_as_ushort(hh);
    l = MODE == kBF16X3 ? __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(hh))) : 0u;
  }
}

// Split 16-bit output of stage 1: row (j, y) of the A operand, chunked
// [Re 32 | Im 32], and in the split modes the sums As = Re + Im for the
// Gauss product, chunked [As_hi 32 | As_lo 32] (the sum is formed in FP32,
// scaled like the parts, then split).  W consecutive columns (W a multiple
// of 4 dividing 32) are packed into 8-byte stores per part.
template <int MODE>
struct OutSplit {
  static constexpr bool kRowWise = true;
  __device__ float2* column(int, int) const { return nullptr; }
  void* hi;
  void* lo;
  void* sum;
  const float* scales;
  int n, crop, nk;  // row j of the operand belongs to kernel j mod nk
  template <int W>
  __device__ __forceinline__ void store_row(int j, int y, int c0, const float2 (&v)[W]) const {
    static_assert(W % 4 == 0 && CH % W == 0, "column block");
    const size_t o = ((size_t)j * n + y) * (size_t)(2 * crop) + (size_t)(c0 / CH) * KE + (c0 % CH);
    const float s = scales[j % nk];
    uint32_t rh[W], rl[W], ih[W], il[W], sh[W], sl[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      split16<MODE>(v[w].x, s, rh[w], rl[w]);
      split16<MODE>(v[w].y, s, ih[w], il[w]);
      split16<MODE>(v[w].x + v[w].y, s, sh[w], sl[w]);
    }
    // one store per part and row: W 16-bit values, 16 bytes for W = 8 (fewer L2 write transactions)
    auto put = [&](void* base, size_t off, const uint32_t (&x)[W]) {
      uint16_t* d = static_cast<uint16_t*>(base) + off;
      if constexpr (W == 8) {
        *reinterpret_cast<uint4*>(d) = make_uint4(x[0] | (x[1] << 16), x[2] | (x[3] << 16), x[4] | (x[5] << 16),
                                                  x[6] | (x[7] << 16));
      } else {
#pragma unroll
        for (int q = 0; q < W / 4; ++q)
          reinterpret_cast<uint2*>(d)[q] = make_uint2(x[4 * q] | (x[4 * q + 1] << 16), x[4 * q + 2] | (x[4 * q + 3] << 16));
      }
    };
    put(hi, o, rh);
    put(hi, o + CH, ih);
    if (MODE == kFP16X3 || MODE == kBF16X3) {
      put(lo, o, rl);
      put(lo, o + CH, il);
      put(sum, o, sh);
      put(sum, o + CH, sl);
    }
  }
};

// `clips` spectra in one launch; clip i writes the operand rows of kernels j + i nk.
template <int N, int MODE>
cudaError_t stage1_split_n(const float2* mhat, const float2* phi, int nk, int crop, const float2* tw,
                           const float* scales, void* a_hi, void* a_lo, void* a_s, int clips, cudaStream_t st) {
  return launch_stage1_cols<N, Stage1W<N>::W>(mhat, phi, nk, crop, tw,
                                           OutSplit<MODE>{a_hi, a_lo, a_s, scales, N, crop, nk}, st, clips);
}

template <int MODE>
cudaError_t stage1_split_mode(int n, const float2* mhat, const float2* phi, int nk, int crop, const float2* tw,
                              const float* scales, void* a_hi, void* a_lo, void* a_s, int clips, cudaStream_t st) {
  switch (n) {
    case 128: return stage1_split_n<128, MODE>(mhat, phi, nk, crop, tw, scales, a_hi, a_lo, a_s, clips, st);
    case 256: return stage1_split_n<256, MODE>(mhat, phi, nk, crop, tw, scales, a_hi, a_lo, a_s, clips, st);
    case 512: return stage1_split_n<512, MODE>(mhat, phi, nk, crop, tw, scales, a_hi, a_lo, a_s, clips, st);
    case 896: return stage1_split_n<896, MODE>(mhat, phi, nk, crop, tw, scales, a_hi, a_lo, a_s, clips, st);
    case 1024: return stage1_split_n<1024, MODE>(mhat, phi, nk, crop, tw, scales, a_hi, a_lo, a_s, clips, st);
    case 2048: return stage1_split_n<2048, MODE>(mhat, phi, nk, crop, tw, scales, a_hi, a_lo, a_s, clips, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---- host side ---------------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// 2-D tensor map over rows x (2C) 16-bit elements, 128 x 64 boxes, 128-byte swizzle.
bool make_map(CUtensorMap* m, void* base, int fmt, unsigned long long rows, unsigned long long cols) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {KE, BM};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Constant operands per precision mode and grid (0 = full N, 1 = coarse nc).
struct GemmOperands {
  std::mutex mu;
  bool built[kModes][2] = {};
  void* b_hi[kModes][2] = {};
  void* b_lo[kModes][2] = {};
  void* b_s[kModes][2] = {};  // [Ws_hi 32 | Ws_lo 32] chunks, split modes
  CUtensorMap map_hi[kModes][2], map_lo[kModes][2], map_s[kModes][2];
  float* d_lamp[kModes] = {};   // lambda / scale^2 per (f, k)
  float* d_scale[kModes] = {};  // stage-1 scale per (f, k)
  int* d_err = nullptr;
  int sm_count = 0;
};

namespace {

int eval_n(const litho_kernels* h, bool coarse) { return coarse ? h->nc_tc : h->n; }

// Bytes of one 16-bit operand array (A hi, A lo or AS) for one clip.
size_t per_clip_array_bytes(const litho_kernels* h, bool coarse) {
  const size_t rows = size_t(h->n_focus) * h->k * eval_n(h, coarse), cols = size_t(2) * h->crop;
  return rows * cols * 2;
}
int arrays_of(int mode) { return is_split(mode) ? 3 : 1; }  // A_hi (+ A_lo, AS when split)

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Builds the twiddle operand B (cos | sin chunks, split) and the per-kernel
// scales for one precision mode.  Host FP64, then rounded.
litho_status build_operands(const litho_kernels* hc, int mode, bool coarse) {
  litho_kernels* h = const_cast<litho_kernels*>(hc);
  static std::mutex create_mu;
  {
    std::lock_guard<std::mutex> lk0(create_mu);
    if (!h->gemm) h->gemm = new GemmOperands();
  }
  GemmOperands* g = h->gemm;
  std::lock_guard<std::mutex> lk(g->mu);
  const int gi = coarse ? 1 : 0;
  if (g->built[mode][gi]) return LITHO_OK;
  const int N = eval_n(h, coarse), C = h->crop, F = h->n_focus, K = h->k;
  const size_t cols = size_t(2) * C, count = size_t(N) * cols;
  std::vector<uint16_t> hi(count), lo(count), sum(count);
  auto split = [&](double w, uint16_t& h16, uint16_t& l16) {
    if (is_fp16(mode)) {
      const __half hh = __float2half_rn(float(w));
      h16 = __half_as_ushort(hh);
      l16 = __half_as_ushort(__float2half_rn(float(w - double(__half2float(hh)))));
    } else {
      const __nv_bfloat16 hh = __float2bfloat16_rn(float(w));
      h16 = __bfloat16_as_ushort(hh);
      l16 = __bfloat16_as_ushort(__float2bfloat16_rn(float(w - double(__bfloat162float(hh)))));
    }
  };
  for (int x = 0; x < N; ++x) {
    for (size_t kk = 0; kk < cols; ++kk) {
      const int chunk = int(kk / KE), within = int(kk % KE), part = within / CH;
      const int c = chunk * CH + within % CH;
      const long long e = ((long long)(c - C / 2) * x % N + N) % N;
      const double a = 2.0 * M_PI * double(e) / double(N);
      split(part ? std::sin(a) : std::cos(a), hi[size_t(x) * cols + kk], lo[size_t(x) * cols + kk]);
      // the sum cos + sin of the Gauss product: hi in the first half of the chunk, lo in the second
      uint16_t sh = 0, sl = 0;
      split(std::cos(a) + std::sin(a), sh, sl);
      sum[size_t(x) * cols + kk] = part ? sl : sh;
    }
  }
  // per-kernel scales: |T_k| <= max_u sum_v |Phi_k(v, u)| for masks with |m| <= 1
  std::vector<float> scale(size_t(F) * K, 1.f), lamp(size_t(F) * K, 0.f);
  for (int f = 0; f < F; ++f)
    for (int k = 0; k < K; ++k) {
      const size_t fk = size_t(f) * K + k;
      double s = 1.0;
      if (is_fp16(mode)) {
        double bound = 0.0;
        const double* ph = &h->phi_host[fk * size_t(C) * C * 2];
        for (int u = 0; u < C; ++u) {
          double col = 0.0;
          for (int v = 0; v < C; ++v) col += std::hypot(ph[(size_t(v) * C + u) * 2], ph[(size_t(v) * C + u) * 2 + 1]);
          bound = std::max(bound, col);
        }
        if (bound > 0.0) s = std::ldexp(1.0, int(std::floor(std::log2(8192.0 / bound))));
      }
      scale[fk] = float(s);
      lamp[fk] = float(h->lambda[fk] / (s * s));
    }
  LITHO_TRY_CUDA(cudaMalloc(&g->b_hi[mode][gi], count * 2));
  LITHO_TRY_CUDA(cudaMemcpy(g->b_hi[mode][gi], hi.data(), count * 2, cudaMemcpyHostToDevice));
  if (is_split(mode)) {
    LITHO_TRY_CUDA(cudaMalloc(&g->b_lo[mode][gi], count * 2));
    LITHO_TRY_CUDA(cudaMemcpy(g->b_lo[mode][gi], lo.data(), count * 2, cudaMemcpyHostToDevice));
    LITHO_TRY_CUDA(cudaMalloc(&g->b_s[mode][gi], count * 2));
    LITHO_TRY_CUDA(cudaMemcpy(g->b_s[mode][gi], sum.data(), count * 2, cudaMemcpyHostToDevice));
  }
  if (!g->d_scale[mode]) {
    LITHO_TRY_CUDA(cudaMalloc(&g->d_scale[mode], scale.size() * sizeof(float)));
    LITHO_TRY_CUDA(cudaMemcpy(g->d_scale[mode], scale.data(), scale.size() * sizeof(float), cudaMemcpyHostToDevice));
    LITHO_TRY_CUDA(cudaMalloc(&g->d_lamp[mode], lamp.size() * sizeof(float)));
    LITHO_TRY_CUDA(cudaMemcpy(g->d_lamp[mode], lamp.data(), lamp.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  if (!g->d_err) {
    LITHO_TRY_CUDA(cudaMalloc(&g->d_err, sizeof(int)));
    LITHO_TRY_CUDA(cudaMemset(g->d_err, 0, sizeof(int)));
  }
  const int fmt = is_fp16(mode) ? 0 : 1;
  if (!make_map(&g->map_hi[mode][gi], g->b_hi[mode][gi], fmt, N, cols) ||
      !make_map(&g->map_lo[mode][gi], is_split(mode) ? g->b_lo[mode][gi] : g->b_hi[mode][gi], fmt, N, cols) ||
      !make_map(&g->map_s[mode][gi], is_split(mode) ? g->b_s[mode][gi] : g->b_hi[mode][gi], fmt, N, cols)) {
    set_error("cuTensorMapEncodeTiled failed for the twiddle operand");
    return LITHO_ECUDA;
  }
  int dev = 0;
  LITHO_TRY_CUDA(cudaGetDevice(&dev));
  LITHO_TRY_CUDA(cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, dev));
  g->built[mode][gi] = true;
  return LITHO_OK;
}

}  // namespace

size_t gemm_workspace_bytes(const litho_kernels* h, litho_precision prec, int b, bool coarse) {
  const int mode = mode_of(prec);
  const int g = std::min(b, GROUP_CLIPS);
  return arrays_of(mode) * up256(size_t(g) * per_clip_array_bytes(h, coarse));
}

litho_status gemm_supported(const litho_kernels* h, litho_precision prec, bool coarse) {
  const int n = eval_n(h, coarse);
  if (n < 128 || n % 128 != 0 || h->crop % CH != 0) {
    set_error("tensor-core path needs an evaluation grid that is a multiple of 128 (got %d, crop = %d)", n, h->crop);
    return LITHO_EUNSUPPORTED;
  }
  int dev = 0, major = 0, minor = 0;
  LITHO_TRY_CUDA(cudaGetDevice(&dev));
  LITHO_TRY_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  LITHO_TRY_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
  if (major != 10 || minor != 3) {
    set_error("tensor-core path is built for sm_103a (this device is sm_%d%d)", major, minor);
    return LITHO_EUNSUPPORTED;
  }
  if (!encode_fn()) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return LITHO_EUNSUPPORTED;
  }
  return build_operands(h, mode_of(prec), coarse);
}

litho_status gemm_aerial_group(const litho_kernels* h, const float2* mhat, int clips, float dose,
                               litho_precision prec, bool coarse, float* img, void* ws, cudaStream_t st) {
  const int mode = mode_of(prec), gi = coarse ? 1 : 0;
  GemmOperands* g = h->gemm;
  const int N = eval_n(h, coarse), C = h->crop, F = h->n_focus, K = h->k;
  const float2* tw = coarse ? h->d_twc_tc : h->d_tw;
  const size_t arr = up256(size_t(std::min(clips, GROUP_CLIPS)) * per_clip_array_bytes(h, coarse));
  char* a_hi = static_cast<char*>(ws);
  char* a_lo = is_split(mode) ? a_hi + arr : a_hi;
  char* a_s = is_split(mode) ? a_hi + 2 * arr : a_hi;
  {
    ProfScope ps(kStageGemmOperands, st, 1);  // one launch for the group
    cudaError_t e;
    if (mode == kBF16)
      e = stage1_split_mode<kBF16>(N, mhat, h->d_phi, F * K, C, tw, g->d_scale[mode], a_hi, nullptr, nullptr, clips,
                                   st);
    else if (mode == kFP16)
      e = stage1_split_mode<kFP16>(N, mhat, h->d_phi, F * K, C, tw, g->d_scale[mode], a_hi, nullptr, nullptr, clips,
                                   st);
    else if (mode == kBF16X3)
      e = stage1_split_mode<kBF16X3>(N, mhat, h->d_phi, F * K, C, tw, g->d_scale[mode], a_hi, a_lo, a_s, clips, st);
    else
      e = stage1_split_mode<kFP16X3>(N, mhat, h->d_phi, F * K, C, tw, g->d_scale[mode], a_hi, a_lo, a_s, clips, st);
    LITHO_TRY_CUDA(e);
  }
  const int fmt = is_fp16(mode) ? 0 : 1;
  const unsigned long long rows = (unsigned long long)clips * F * K * N;
  CUtensorMap ta_hi, ta_lo, ta_s;
  if (!make_map(&ta_hi, a_hi, fmt, rows, 2ull * C) || !make_map(&ta_lo, a_lo, fmt, rows, 2ull * C) ||
      !make_map(&ta_s, a_s, fmt, rows, 2ull * C)) {
    set_error("cuTensorMapEncodeTiled failed for the stage-1 operand");
    return LITHO_ECUDA;
  }
  GemmParams p;
  p.n = N;
  p.nk = K;
  p.n_focus = F;
  p.planes = clips * F;
  p.tiles_y = N / BM;
  p.tiles_x = N / XT;
  p.chunks = C / CH;
  p.split = is_split(mode) ? 1 : 0;
  p.fmt = fmt;
  p.lamp = g->d_lamp[mode];
  p.dose = dose;
  p.img = img;
  p.err = g->d_err;
  const int total = p.planes * p.tiles_y * p.tiles_x;
  const int grid = std::min(total, g->sm_count);
  LITHO_TRY_CUDA(cudaFuncSetAttribute(k_dft_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  ProfScope ps(kStageStage2Gemm, st, 1);
  k_dft_gemm<<<grid, THREADS, SMEM_BYTES, st>>>(ta_hi, ta_lo, ta_s, g->map_hi[mode][gi], g->map_lo[mode][gi],
                                                g->map_s[mode][gi], p);
  LITHO_TRY_CUDA(cudaGetLastError());
  return LITHO_OK;
}

int gemm_group_clips() { return GROUP_CLIPS; }

litho_status gemm_wait_selftest(const litho_kernels* hc, double limit_ms, cudaStream_t st) {
  litho_kernels* h = const_cast<litho_kernels*>(hc);
  {
    static std::mutex create_mu;
    std::lock_guard<std::mutex> lk0(create_mu);
    if (!h->gemm) h->gemm = new GemmOperands();
  }
  {
    std::lock_guard<std::mutex> lk(h->gemm->mu);
    if (!h->gemm->d_err) {
      LITHO_TRY_CUDA(cudaMalloc(&h->gemm->d_err, sizeof(int)));
      LITHO_TRY_CUDA(cudaMemset(h->gemm->d_err, 0, sizeof(int)));
    }
  }
  int dev = 0, khz = 0;
  LITHO_TRY_CUDA(cudaGetDevice(&dev));
  LITHO_TRY_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
  const long long limit = (long long)(limit_ms * double(khz > 0 ? khz : 2000000));
  k_wait_selftest<<<1, 32, 0, st>>>(h->gemm->d_err, limit, 9);
  LITHO_TRY_CUDA(cudaGetLastError());
  return gemm_check_device(h, st);
}

litho_status gemm_check_device(const litho_kernels* h, cudaStream_t st) {
  if (!h->gemm || !h->gemm->d_err) return LITHO_OK;
  int flag = 0;
  LITHO_TRY_CUDA(cudaMemcpyAsync(&flag, h->gemm->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LITHO_TRY_CUDA(cudaStreamSynchronize(st));
  if (flag) {
    LITHO_TRY_CUDA(cudaMemsetAsync(h->gemm->d_err, 0, sizeof(int), st));
    set_error("a tensor-core kernel gave up waiting on a pipeline barrier (code %d)", flag);
    return LITHO_ETIMEOUT;
  }
  return LITHO_OK;
}

void gemm_free_operands(litho_kernels* h) {
  if (!h->gemm) return;
  for (int m = 0; m < kModes; ++m) {
    for (int gi = 0; gi < 2; ++gi) {
      cudaFree(h->gemm->b_hi[m][gi]);
      cudaFree(h->gemm->b_lo[m][gi]);
      cudaFree(h->gemm->b_s[m][gi]);
    }
    cudaFree(h->gemm->d_lamp[m]);
    cudaFree(h->gemm->d_scale[m]);
  }
  cudaFree(h->gemm->d_err);
  delete h->gemm;
  h->gemm = nullptr;
}

}  // namespace litho
