// Shared-memory Stockham FFT building blocks for sm_103a.
//
// A length-N transform (N a power of two, 32..2048, or 896) is a sequence of
// radix-R passes (R in {4, 7, 8, 16}); before pass p, `NS` is the product of the earlier
// radices.  Butterfly j in [0, N/R) of a pass reads x[j + r N/R] (r < R),
// multiplies element r by w^(r (j mod NS) N/(NS R)) (w = e^{-2 pi i/N}, or its
// conjugate for the inverse), takes an R-point DFT in registers and writes
// element q to y[(j div NS) NS R + (j mod NS) + q NS].  This is Stockham's
// self-sorting formulation: the output comes out in natural order with no bit
// reversal, and each pass reads with unit stride across threads.
//
// Shared-memory layout: element i of a transform sits at pad16(i) = i + i/16,
// one spare slot per 16 complex values.  The first pass writes with stride R
// across threads; without the spare slots a half-warp of 8-byte stores would
// land in the same two banks.  With them every pass is conflict-free for
// R = 16 and at most two-way for R = 8 at NS = 8.
//
// Twiddles come from a per-pass table built on the host in FP64 and staged in
// shared memory: for each pass after the first, entries (r-1) NS + k hold
// w^(r k N/(NS R)) for r in [1, R), k in [0, NS), so consecutive butterflies
// read consecutive entries.  The R-point DFTs are radix-2
// decimation-in-frequency networks in registers (R = 7: symmetric pairs).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

namespace litho {

// Complex arithmetic on the packed two-lane FP32 instructions of sm_100+
// (one instruction for both components, each rounded as the scalar form).
// cmul: (a.x b.x - a.y b.y, a.x b.y + a.y b.x) = fma(a.x, b, (-a.y b.y, a.y b.x)).
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return __ffma2_rn(make_float2(a.x, a.x), b, __fmul2_rn(make_float2(a.y, a.y), make_float2(-b.y, b.x)));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as fma(b, -1, a): exact product, one rounding, as the scalar subtraction
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__host__ __device__ __forceinline__ constexpr int pad16(int i) { return i + (i >> 4); }
template <int N>
struct PadLen {
  static constexpr int value = N + N / 16;
};

// cos and sin of 2 pi t / 16 (exact mathematical constants rounded to float)
__device__ __forceinline__ constexpr float cos16(int t) {
  return t == 0 ? 1.0f : t == 1 ? 0.92387953251128674f : t == 2 ? 0.70710678118654752f
       : t == 3 ? 0.38268343236508977f : t == 4 ? 0.0f : t == 5 ? -0.38268343236508977f
       : t == 6 ? -0.70710678118654752f : t == 7 ? -0.92387953251128674f : -1.0f;
}
__device__ __forceinline__ constexpr float sin16(int t) {
  return t == 0 ? 0.0f : t == 1 ? 0.38268343236508977f : t == 2 ? 0.70710678118654752f
       : t == 3 ? 0.92387953251128674f : t == 4 ? 1.0f : t == 5 ? 0.92387953251128674f
       : t == 6 ? 0.70710678118654752f : t == 7 ? 0.38268343236508977f : 0.0f;
}

// cos and sin of 2 pi t / 7, t = 1, 2, 3 (exact mathematical constants rounded to float)
__device__ __forceinline__ constexpr float cos7(int t) {
  return t == 1 ? 0.62348980185873353f : t == 2 ? -0.22252093395631440f : -0.90096886790241913f;
}
__device__ __forceinline__ constexpr float sin7(int t) {
  return t == 1 ? 0.78183148246802981f : t == 2 ? 0.97492791218182361f : 0.43388373911755812f;
}

// 7-point DFT, v'[q] = sum_r v[r] e^{SIGN 2 pi i r q / 7}, from the symmetric
// pairs a_m = v[m] + v[7-m] and b_m = v[m] - v[7-m] (m = 1..3):
// v'[q] = v[0] + sum_m a_m cos(2 pi m q/7) + SIGN i sum_m b_m sin(2 pi m q/7),
// and v'[7-q] the same with the sine term negated.
template <int SIGN>
__device__ __forceinline__ void dft7(float2 (&v)[7]) {
  float2 a[4], b[4];
#pragma unroll
  for (int m = 1; m <= 3; ++m) {
    a[m] = cadd(v[m], v[7 - m]);
    b[m] = csub(v[m], v[7 - m]);
  }
  const float2 x0 = v[0];
  v[0] = make_float2(x0.x + a[1].x + a[2].x + a[3].x, x0.y + a[1].y + a[2].y + a[3].y);
#pragma unroll
  for (int q = 1; q <= 3; ++q) {
    float2 p = x0, s = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
      const int k = (m * q) % 7;  // angle 2 pi k / 7; k > 3 is the mirror 7 - k with the sine negated
      const float c = k <= 3 ? cos7(k) : cos7(7 - k);
      const float sn = k <= 3 ? sin7(k) : -sin7(7 - k);
      p = make_float2(fmaf(a[m].x, c, p.x), fmaf(a[m].y, c, p.y));
      s = make_float2(fmaf(b[m].x, sn, s.x), fmaf(b[m].y, sn, s.y));
    }
    // SIGN i s = (-SIGN s.y, SIGN s.x)
    v[q] = make_float2(p.x - SIGN * s.y, p.y + SIGN * s.x);
    v[7 - q] = make_float2(p.x + SIGN * s.y, p.y - SIGN * s.x);
  }
}

__host__ __device__ __forceinline__ constexpr int ilog2(int x) {
  int r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
}
__host__ __device__ __forceinline__ constexpr int bitrev(int q, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r = (r << 1) | ((q >> i) & 1);
  return r;
}

// In-register R-point DFT, v'[q] = sum_r v[r] e^{SIGN 2 pi i r q / R}.
// BANDED: only v[r] with r < R/4 or r >= 3R/4 may be nonzero and the others
// are not read, so the first radix-2 layer reduces to copies, negations and
// twiddles.  A first pass (stride N/R) over a spectrum whose nonzero entries
// lie in the lowest and highest quarter of the indices has this form.
template <int R, int SIGN, bool BANDED = false>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
  static_assert(R == 2 || R == 4 || R == 7 || R == 8 || R == 16, "radix");
  static_assert(!BANDED || (R >= 4 && R != 7), "banded input needs a power-of-two R >= 4");
  if constexpr (R == 7) {
    dft7<SIGN>(v);
    return;
  } else {
#pragma unroll
  for (int span = R / 2; span >= 1; span /= 2) {
#pragma unroll
    for (int b = 0; b < R; b += 2 * span) {
#pragma unroll
      for (int i = 0; i < span; ++i) {
        float2 d;
        if (BANDED && span == R / 2) {
          if (i < R / 4) {
            d = v[i];  // v[i + span] is zero
          } else {     // v[i] is zero
            v[i] = v[i + span];
            d = make_float2(-v[i].x, -v[i].y);
          }
        } else {
          const float2 a = v[b + i], c = v[b + i + span];
          v[b + i] = cadd(a, c);
          d = csub(a, c);
        }
        const int t = i * (16 / (2 * span));  // e^{SIGN 2 pi i i/(2 span)} = e^{SIGN 2 pi i t/16}
        if (t != 0) {
          const float wr = cos16(t), wi = SIGN * sin16(t);
          if (t == 4) {
            d = make_float2(-wi * d.y, wi * d.x);  // multiply by +-i
          } else {
            d = cmul(d, make_float2(wr, wi));
          }
        }
        v[b + i + span] = d;
      }
    }
  }
  constexpr int LB = ilog2(R);
  float2 o[R];
#pragma unroll
  for (int q = 0; q < R; ++q) o[q] = v[bitrev(q, LB)];
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = o[q];
  }
}

// cos and sin of 2 pi t / 32 for t in [0, 32) (exact mathematical constants rounded to float)
__device__ __forceinline__ constexpr float cos32(int t) {
  t &= 31;
  if (t > 16) t = 32 - t;  // cos is even
  const float c[17] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
                       0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
                       0.19509032201612826785f, 0.0f, -0.19509032201612826785f, -0.38268343236508977173f,
                       -0.55557023301960222474f, -0.70710678118654752440f, -0.83146961230254523708f,
                       -0.92387953251128675613f, -0.98078528040323044913f, -1.0f};
  return c[t];
}
__device__ __forceinline__ constexpr float sin32(int t) { return cos32(8 - t); }

// x times e^{SIGN 2 pi i t / 32} for a compile-time t (the multiples of 8 are a
// quarter turn, a sign or nothing).
template <int SIGN, int T>
__device__ __forceinline__ float2 twiddle32(float2 x) {
  constexpr int t = T % 32;
  if constexpr (t == 0) {
    return x;
  } else if constexpr (t == 8) {
    return make_float2(-SIGN * x.y, SIGN * x.x);
  } else if constexpr (t == 16) {
    return make_float2(-x.x, -x.y);
  } else if constexpr (t == 24) {
    return make_float2(SIGN * x.y, -SIGN * x.x);
  } else {
    return cmul(x, make_float2(cos32(t), SIGN * sin32(t)));
  }
}

// 4-point DFT in place, y[k] = sum_m x[m] e^{SIGN 2 pi i m k / 4}, on v[i0 + s m].
// X1_X2_ZERO: v[i0 + s] and v[i0 + 2 s] are known to be zero and are not read.
template <int SIGN, bool X1_X2_ZERO>
__device__ __forceinline__ void dft4_at(float2 (&v)[32], int i0, int s) {
  const float2 x0 = v[i0], x3 = v[i0 + 3 * s];
  float2 a, b, c, d;
  if constexpr (X1_X2_ZERO) {
    a = x0;
    b = x0;
    c = x3;
    d = make_float2(-SIGN * x3.y, SIGN * x3.x);  // (x1 - x3) SIGN i with x1 = 0 ...
    d = make_float2(-d.x, -d.y);                 // ... = -x3 SIGN i
  } else {
    const float2 x1 = v[i0 + s], x2 = v[i0 + 2 * s];
    a = cadd(x0, x2);
    b = csub(x0, x2);
    c = cadd(x1, x3);
    const float2 e = csub(x1, x3);
    d = make_float2(-SIGN * e.y, SIGN * e.x);  // e SIGN i
  }
  v[i0] = cadd(a, c);
  v[i0 + s] = cadd(b, d);
  v[i0 + 2 * s] = csub(a, c);
  v[i0 + 3 * s] = csub(b, d);
}

// 32-point DFT in registers, v'[q] = sum_r v[r] e^{SIGN 2 pi i r q / 32}, output in
// natural order.  Decimation in frequency with radices 4, 4, 2: a radix-4 stage over
// stride 8 with twiddles w^(i k1), a radix-4 stage over stride 2 within each block of
// 8 with twiddles w^(4 j k2), a radix-2 stage on pairs; position 8 k1 + 2 k2 + k3 then
// holds output k1 + 4 k2 + 16 k3.  28 non-trivial twiddle products against 34 for a
// radix-2 network, the same additions.  BANDED: v[r] for r in [8, 24) is zero and
// not read (the first stage's middle inputs).
template <int SIGN, bool BANDED>
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) dft4_at<SIGN, BANDED>(v, i, 8);
#pragma unroll
  for (int i = 1; i < 8; ++i) {
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) {
      const int t = i * k1;
      float2& x = v[i + 8 * k1];
      if (t == 8) {
        x = twiddle32<SIGN, 8>(x);
      } else if (t % 32 != 0) {
        x = cmul(x, make_float2(cos32(t), SIGN * sin32(t)));
      }
    }
  }
#pragma unroll
  for (int blk = 0; blk < 4; ++blk) {
#pragma unroll
    for (int j = 0; j < 2; ++j) dft4_at<SIGN, false>(v, 8 * blk + j, 2);
    // j = 1: twiddles w^(4 k2), k2 = 1, 2, 3 (w^8 is a quarter turn)
    v[8 * blk + 3] = cmul(v[8 * blk + 3], make_float2(cos32(4), SIGN * sin32(4)));
    v[8 * blk + 5] = twiddle32<SIGN, 8>(v[8 * blk + 5]);
    v[8 * blk + 7] = cmul(v[8 * blk + 7], make_float2(cos32(12), SIGN * sin32(12)));
  }
#pragma unroll
  for (int p = 0; p < 32; p += 2) {
    const float2 a = v[p], b = v[p + 1];
    v[p] = cadd(a, b);
    v[p + 1] = csub(a, b);
  }
  float2 o[32];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2)
#pragma unroll
      for (int k3 = 0; k3 < 2; ++k3) o[k1 + 4 * k2 + 16 * k3] = v[8 * k1 + 2 * k2 + k3];
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = o[q];
}

// Radix plans: passes in order, product N.  NT = threads per transform.
// Besides the powers of two, 896 = 16 x 8 x 7: the smallest grid that holds
// the 2C - 1 frequencies of an image whose field band has C = 448 columns.
template <int N> struct Plan;
template <> struct Plan<32>   { static constexpr int NT = 32;  static constexpr int R[2] = {8, 4}; static constexpr int P = 2; };
template <> struct Plan<64>   { static constexpr int NT = 32;  static constexpr int R[2] = {8, 8}; static constexpr int P = 2; };
template <> struct Plan<128>  { static constexpr int NT = 32;  static constexpr int R[2] = {16, 8}; static constexpr int P = 2; };
template <> struct Plan<256>  { static constexpr int NT = 32;  static constexpr int R[2] = {16, 16}; static constexpr int P = 2; };
template <> struct Plan<512>  { static constexpr int NT = 64;  static constexpr int R[3] = {8, 8, 8}; static constexpr int P = 3; };
template <> struct Plan<1024> { static constexpr int NT = 64;  static constexpr int R[3] = {16, 8, 8}; static constexpr int P = 3; };
template <> struct Plan<2048> { static constexpr int NT = 128; static constexpr int R[3] = {16, 16, 8}; static constexpr int P = 3; };
template <> struct Plan<896>  { static constexpr int NT = 64;  static constexpr int R[3] = {16, 8, 7}; static constexpr int P = 3; };

template <int N, int NT, int R>
struct PassShape {
  static constexpr int NB = N / R;                  // butterflies
  static constexpr int PER = (NB + NT - 1) / NT;    // butterflies per thread
};

// Padded offset of element i + step from that of i when step is a multiple
// of 16: pad16(i + step) = pad16(i) + step + step/16, a compile-time
// distance.  Otherwise (small transforms) the full index is formed.
template <int STEP>
__device__ __forceinline__ int pad16_step(int i, int r) {
  if constexpr (STEP % 16 == 0) {
    return pad16(i) + r * (STEP + STEP / 16);
  } else {
    return pad16(i + r * STEP);
  }
}

// Offsets of the passes' twiddle blocks: pass 1 at 0, pass 2 after it.
template <int N>
struct TwOff {
  static constexpr int p1 = 0;
  static constexpr int p2 = (Plan<N>::P == 3) ? (Plan<N>::R[1] - 1) * Plan<N>::R[0] : 0;
};

// Twiddle + DFT of one butterfly's R values.
// The pass's table holds w^(r k), r = 1..R-1, for its root w.  For R = 4, 8
// and 16 only the powers r = 1, 2, 4, 8 are read and the others formed as
// products of two or three of them (w^3 = w^1 w^2, w^(r+4) = w^r w^4,
// w^(r+8) = w^r w^8): a few packed multiplies instead of shared-memory loads,
// which bound the column transforms, at one to two roundings more per twiddle.
template <int N, int R, int NS, int SIGN, int OFF, bool BANDED = false>
__device__ __forceinline__ void twiddle_dft(float2 (&v)[R], int j, const float2* __restrict__ tw) {
  if (NS > 1) {
    const int k = j % NS;
    auto ld = [&](int r) {
      float2 w = tw[OFF + (r - 1) * NS + k];
      if (SIGN > 0) w.y = -w.y;
      return w;
    };
    if constexpr (R == 4 || R == 8 || R == 16) {
      float2 w[R];
      w[1] = ld(1);
      w[2] = ld(2);
      w[3] = cmul(w[1], w[2]);
      if constexpr (R >= 8) {
        w[4] = ld(4);
#pragma unroll
        for (int r = 5; r < 8; ++r) w[r] = cmul(w[r - 4], w[4]);
      }
      if constexpr (R == 16) {
        w[8] = ld(8);
#pragma unroll
        for (int r = 9; r < 16; ++r) w[r] = cmul(w[r - 8], w[8]);
      }
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r]);
    } else {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], ld(r));
    }
  }
  dft_reg<R, SIGN, BANDED>(v);
}

// Stockham output of one pass: butterfly j's R values to their places in
// shared memory (no barrier).
template <int N, int NT, int R, int NS>
__device__ __forceinline__ void store_pass(float2* buf, int t, const float2 (&v)[PassShape<N, NT, R>::PER][R]) {
  using S = PassShape<N, NT, R>;
#pragma unroll
  for (int p = 0; p < S::PER; ++p) {
    const int j = t + p * NT;
    if (j < S::NB) {
      const int base = (j / NS) * NS * R + (j % NS);
      if constexpr (NS == 1 && 16 % R == 0) {
        // base is a multiple of R, which divides 16: base + r stays in one run of 16
        float2* wb = buf + pad16(base);
#pragma unroll
        for (int r = 0; r < R; ++r) wb[r] = v[p][r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pad16_step<NS>(base, r)] = v[p][r];
      }
    }
  }
}

// One pass whose inputs come from `load(index)` (or shared memory when
// FROM_SMEM) and whose outputs go to shared memory.  Ends with a barrier.
// A loader that also takes (p, r, index) gets the butterfly slot p and the
// element r (compile-time after unrolling), so it can keep per-element
// operands in registers.  BANDED (first pass only): indices in [N/4, 3N/4)
// are known to be zero and are neither loaded nor added.
template <int N, int NT, int R, int NS, int SIGN, int OFF, bool FROM_SMEM, class Load, bool BANDED = false>
__device__ __forceinline__ void pass_to_smem(float2* buf, const float2* tw, int t, Load& load) {
  using S = PassShape<N, NT, R>;
  static_assert(!BANDED || NS == 1, "banded input applies to the first pass");
  float2 v[S::PER][R];
#pragma unroll
  for (int p = 0; p < S::PER; ++p) {
    const int j = t + p * NT;
    if (j < S::NB) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (BANDED && r >= R / 4 && r < 3 * R / 4) {
          v[p][r] = make_float2(0.f, 0.f);  // never read
        } else {
          if constexpr (FROM_SMEM) {
            v[p][r] = buf[pad16_step<S::NB>(j, r)];
          } else if constexpr (std::is_invocable_v<Load&, int, int, int>) {
            v[p][r] = load(p, r, j + r * S::NB);
          } else {
            v[p][r] = load(j + r * S::NB);
          }
        }
      }
      twiddle_dft<N, R, NS, SIGN, OFF, BANDED>(v[p], j, tw);
    }
  }
  __syncthreads();
  store_pass<N, NT, R, NS>(buf, t, v);
  __syncthreads();
}

// Last pass from shared memory; hands each output element to
// use(p, q, index, value), index = j + q N/R with j = t + p NT (NS R = N, so
// the Stockham output position of element q is j + q NS).  p and q are
// compile-time after unrolling, so `use` can index register arrays with them.
// No barrier at the end.
template <int N, int NT, int R, int NS, int SIGN, int OFF, class Use>
__device__ __forceinline__ void pass_last(const float2* buf, const float2* tw, int t, Use& use) {
  using S = PassShape<N, NT, R>;
  static_assert(NS * R == N, "last pass");
#pragma unroll
  for (int p = 0; p < S::PER; ++p) {
    const int j = t + p * NT;
    if (j < S::NB) {
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = buf[pad16_step<S::NB>(j, r)];
      twiddle_dft<N, R, NS, SIGN, OFF>(v, j, tw);
#pragma unroll
      for (int q = 0; q < R; ++q) use(p, q, j + q * S::NB, v[q]);
    }
  }
}

struct SmemLoadUnused {
  __device__ float2 operator()(int) const { return make_float2(0.f, 0.f); }
};

struct NoHook {
  __device__ void operator()() const {}
};

// Full transform: first pass from `load`, middle passes in shared memory,
// last pass into `use`.  Threads t in [0, NT) of the calling group take part;
// every thread of the block must call it (it contains __syncthreads).
// `after_first` runs in every thread once the first pass has finished in all
// of them (after its closing barrier): whatever `load` read is free again.
template <int N, int SIGN, class Load, class Use, bool BANDED = false, class Hook = NoHook>
__device__ __forceinline__ void fft_load_use(float2* buf, const float2* tw, int t, Load& load, Use& use,
                                             const Hook& after_first = Hook()) {
  using PL = Plan<N>;
  constexpr int NT = PL::NT;
  if constexpr (PL::P == 2) {
    pass_to_smem<N, NT, PL::R[0], 1, SIGN, 0, false, Load, BANDED>(buf, tw, t, load);
    after_first();
    pass_last<N, NT, PL::R[1], PL::R[0], SIGN, TwOff<N>::p1>(buf, tw, t, use);
  } else {
    pass_to_smem<N, NT, PL::R[0], 1, SIGN, 0, false, Load, BANDED>(buf, tw, t, load);
    after_first();
    SmemLoadUnused none;
    pass_to_smem<N, NT, PL::R[1], PL::R[0], SIGN, TwOff<N>::p1, true>(buf, tw, t, none);
    pass_last<N, NT, PL::R[2], PL::R[0] * PL::R[1], SIGN, TwOff<N>::p2>(buf, tw, t, use);
  }
}

// Twiddles of the middle pass of a three-pass plan, held in registers.
// When the plan's thread count is a multiple of that pass's stride, all
// butterflies of a thread use the same R - 1 twiddles, so a thread that runs
// many transforms loads them once.
template <int N, int SIGN>
struct MidTwiddles {
  using PL = Plan<N>;
  static constexpr int R = PL::R[1], NS = PL::R[0];
  static constexpr bool kUsable = PL::P == 3 && PL::NT % NS == 0;
  float2 w[R - 1];
  __device__ __forceinline__ void load(const float2* tw, int t) {
    const int k = t % NS;
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 x = tw[TwOff<N>::p1 + (r - 1) * NS + k];
      if (SIGN > 0) x.y = -x.y;
      w[r - 1] = x;
    }
  }
};

// fft_load_use with the middle pass's twiddles from `mid` (same result).
template <int N, int SIGN, class Load, class Use, bool BANDED = false>
__device__ __forceinline__ void fft_load_use_mid(float2* buf, const float2* tw, int t, Load& load, Use& use,
                                                 const MidTwiddles<N, SIGN>& mid) {
  using PL = Plan<N>;
  using M = MidTwiddles<N, SIGN>;
  static_assert(M::kUsable, "middle-pass twiddles are per thread only when NT is a multiple of the stride");
  constexpr int NT = PL::NT, R = M::R, NS = M::NS;
  using S = PassShape<N, NT, R>;
  pass_to_smem<N, NT, PL::R[0], 1, SIGN, 0, false, Load, BANDED>(buf, tw, t, load);
  float2 v[S::PER][R];
#pragma unroll
  for (int p = 0; p < S::PER; ++p) {
    const int j = t + p * NT;
    if (j < S::NB) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[p][r] = buf[pad16_step<S::NB>(j, r)];
#pragma unroll
      for (int r = 1; r < R; ++r) v[p][r] = cmul(v[p][r], mid.w[r - 1]);
      dft_reg<R, SIGN, false>(v[p]);
    }
  }
  __syncthreads();
  store_pass<N, NT, R, NS>(buf, t, v);
  __syncthreads();
  pass_last<N, NT, PL::R[2], PL::R[0] * PL::R[1], SIGN, TwOff<N>::p2>(buf, tw, t, use);
}

// Full transform in place in shared memory (padded layout on entry and on
// return, natural order).  Ends with a barrier.
template <int N, int SIGN>
__device__ __forceinline__ void fft_smem(float2* buf, const float2* tw, int t) {
  using PL = Plan<N>;
  constexpr int NT = PL::NT;
  SmemLoadUnused none;
  pass_to_smem<N, NT, PL::R[0], 1, SIGN, 0, true>(buf, tw, t, none);
  if constexpr (PL::P == 2) {
    pass_to_smem<N, NT, PL::R[1], PL::R[0], SIGN, TwOff<N>::p1, true>(buf, tw, t, none);
  } else {
    pass_to_smem<N, NT, PL::R[1], PL::R[0], SIGN, TwOff<N>::p1, true>(buf, tw, t, none);
    pass_to_smem<N, NT, PL::R[2], PL::R[0] * PL::R[1], SIGN, TwOff<N>::p2, true>(buf, tw, t, none);
  }
}

// Full transform with the first pass from `load` and every pass's output in
// shared memory (padded layout, natural order on return).  Ends with a barrier.
// NTX: the threads that share the transform (default: the plan's own; more
// threads take the butterflies of a pass in fewer rounds).
template <int N, int SIGN, class Load, bool BANDED = false, int NTX = Plan<N>::NT>
__device__ __forceinline__ void fft_load_smem(float2* buf, const float2* tw, int t, Load& load) {
  using PL = Plan<N>;
  constexpr int NT = NTX;
  SmemLoadUnused none;
  pass_to_smem<N, NT, PL::R[0], 1, SIGN, 0, false, Load, BANDED>(buf, tw, t, load);
  if constexpr (PL::P == 2) {
    pass_to_smem<N, NT, PL::R[1], PL::R[0], SIGN, TwOff<N>::p1, true>(buf, tw, t, none);
  } else {
    pass_to_smem<N, NT, PL::R[1], PL::R[0], SIGN, TwOff<N>::p1, true>(buf, tw, t, none);
    pass_to_smem<N, NT, PL::R[2], PL::R[0] * PL::R[1], SIGN, TwOff<N>::p2, true>(buf, tw, t, none);
  }
}

// Columns per CTA for the column-transform kernels (W transforms of
// Plan<N>::NT threads each): 8, so that a CTA loads its twiddle table for
// many columns, except at 512 points (4 columns, several CTAs per SM).
template <int N> struct ColW { static constexpr int W = N == 512 ? 4 : 8; };
// Column stride in shared memory: the padded length rounded up to 16 complex
// values plus 16/W, so that a half-warp of the cooperative copies (w fastest,
// W columns x 16/W rows) touches 16 different 8-byte bank pairs.
template <int N> struct ColLD {
  static constexpr int value = (PadLen<N>::value + 15) / 16 * 16 + 16 / ColW<N>::W;
};
// Stride of the compact band buffers [W][crop] (crop is a multiple of 32).
template <int N>
__host__ __device__ __forceinline__ int band_ld(int crop) { return crop + 16 / ColW<N>::W; }

// Prefer the largest shared-memory carveout for a kernel that uses a lot of it.
template <class K>
inline cudaError_t smem_attrs(K kernel, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

// Stage the twiddle table (N entries, see above) into shared memory.
template <int N>
__device__ __forceinline__ void load_twiddles(float2* s_tw, const float2* __restrict__ g_tw) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) s_tw[i] = g_tw[i];
}

// Host: fills the N-entry per-pass twiddle table of the plan for N (FP64
// angles, rounded to float).  Unused tail entries are zero.
template <int N>
void fill_twiddle_table(float2* out) {
  using PL = Plan<N>;
  for (int i = 0; i < N; ++i) out[i] = make_float2(0.f, 0.f);
  int off = 0, ns = PL::R[0];
  for (int p = 1; p < PL::P; ++p) {
    const int rp = PL::R[p];
    for (int r = 1; r < rp; ++r)
      for (int k = 0; k < ns; ++k) {
        const long long e = (long long)r * k * (N / (ns * rp));
        const double a = 2.0 * 3.14159265358979323846 * double(e) / double(N);
        out[off + (r - 1) * ns + k] = make_float2(float(std::cos(a)), float(-std::sin(a)));
      }
    off += (rp - 1) * ns;
    ns *= rp;
  }
}

}  // namespace litho
