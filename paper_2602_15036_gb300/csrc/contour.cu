// Contours of the resist image and the edge-placement error (paper section
// II.D and Eqs. (6)-(8)).
//
// Marching squares: cell (i, j) has the corners TL = I[i][j], TR = I[i][j+1],
// BR = I[i+1][j+1], BL = I[i+1][j] (periodic); a corner is inside when
// I >= T.  Edges 0 top (TL-TR), 1 right (TR-BR), 2 bottom (BL-BR), 3 left
// (TL-BL) are crossed where their corners differ, at the point of linear
// interpolation of I - T from the edge's first corner to its second.  Each
// segment is oriented with the corner it cuts off on its left when that
// corner is inside and on its right when outside, and, between opposite
// edges, with the inside pair on its left (left of p0 -> p1: cross(p1 - p0,
// q - p0) > 0).  A saddle (only TL and BR, or only TR and BL, inside) joins
// its inside corners when ((TL + TR) + (BR + BL)) / 4 >= T and separates them
// otherwise.  The segment table below is that rule worked out per case.
//
// Four launches, all deterministic: the number of segments per unit (a row
// of cells, or a 128-cell chunk of one when rows are a multiple of 128), one
// CTA per plane scanning its units' counts, one thread placing the planes
// one after another, and the segments written at those offsets in row-major
// cell order (saddle segments ordered by their start edge).
#include <algorithm>
#include <cstdint>

#include "litho_internal.h"

namespace litho {

namespace {

constexpr int kRowThreads = 256;

// Segment table: for each case (inside bits TL = 1, TR = 2, BR = 4, BL = 8)
// up to two (start edge, end edge) pairs packed as s0 | e0 << 2 | s1 << 4 | e1 << 6,
// with the count in bits 8-9.  Saddles 5 and 10 have a second entry for the
// separated variant (index 16 + case).
__constant__ uint16_t kSegTable[32] = {
    // 0: none
    0,
    // 1 TL in: top -> left
    (1 << 8) | (0 | 3 << 2),
    // 2 TR in: right -> top
    (1 << 8) | (1 | 0 << 2),
    // 3 TL, TR in: right -> left
    (1 << 8) | (1 | 3 << 2),
    // 4 BR in: bottom -> right
    (1 << 8) | (2 | 1 << 2),
    // 5 TL, BR in, joined: top -> right (cuts TR), bottom -> left (cuts BL)
    (2 << 8) | (0 | 1 << 2) | ((2 | 3 << 2) << 4),
    // 6 TR, BR in: bottom -> top
    (1 << 8) | (2 | 0 << 2),
    // 7 BL out: bottom -> left
    (1 << 8) | (2 | 3 << 2),
    // 8 BL in: left -> bottom
    (1 << 8) | (3 | 2 << 2),
    // 9 TL, BL in: top -> bottom
    (1 << 8) | (0 | 2 << 2),
    // 10 TR, BL in, joined: right -> bottom (cuts BR), left -> top (cuts TL)
    (2 << 8) | (1 | 2 << 2) | ((3 | 0 << 2) << 4),
    // 11 BR out: right -> bottom
    (1 << 8) | (1 | 2 << 2),
    // 12 BR, BL in: left -> right
    (1 << 8) | (3 | 1 << 2),
    // 13 TR out: top -> right
    (1 << 8) | (0 | 1 << 2),
    // 14 TL out: left -> top
    (1 << 8) | (3 | 0 << 2),
    // 15: none
    0,
    // 16..31: separated saddles (only 21 and 26 used)
    0, 0, 0, 0, 0,
    // 21 = 16 + 5, TL and BR cut off: top -> left, bottom -> right
    (2 << 8) | (0 | 3 << 2) | ((2 | 1 << 2) << 4),
    0, 0, 0, 0,
    // 26 = 16 + 10, TR and BL cut off: right -> top, left -> bottom
    (2 << 8) | (1 | 0 << 2) | ((3 | 2 << 2) << 4),
    0, 0, 0, 0, 0};

struct Cell {
  float tl, tr, br, bl;
};

__device__ __forceinline__ Cell load_cell(const float* __restrict__ img, int n, int i, int j) {
  const int i1 = i + 1 == n ? 0 : i + 1, j1 = j + 1 == n ? 0 : j + 1;
  return Cell{__ldg(img + (size_t)i * n + j), __ldg(img + (size_t)i * n + j1), __ldg(img + (size_t)i1 * n + j1),
              __ldg(img + (size_t)i1 * n + j)};
}

// Index into the segment table (case, or 16 + case for a separated saddle).
__device__ __forceinline__ int cell_case(const Cell& c, float thr) {
  const int cs = (c.tl >= thr) | (c.tr >= thr) << 1 | (c.br >= thr) << 2 | (c.bl >= thr) << 3;
  if (cs == 5 || cs == 10) {
    const float centre = ((c.tl + c.tr) + (c.br + c.bl)) * 0.25f;
    if (!(centre >= thr)) return 16 + cs;
  }
  return cs;
}

// Segments of a case without a table look-up (lanes of a warp index the
// table at different places, which the constant cache would serialise).
__device__ __forceinline__ int case_segments(int cs) {
  cs &= 15;
  return cs == 0 || cs == 15 ? 0 : cs == 5 || cs == 10 ? 2 : 1;
}

// The table entry from a shared-memory copy (one per CTA).
__device__ __forceinline__ uint16_t cell_entry(const Cell& c, float thr, const uint16_t* tab) {
  return tab[cell_case(c, thr)];
}

// Crossing point of edge e in cell-local coordinates (x, y).
__device__ __forceinline__ float2 edge_point(const Cell& c, int e, float thr) {
  float va, vb;
  float2 a, b;
  switch (e) {
    case 0: va = c.tl; vb = c.tr; a = make_float2(0.f, 0.f); b = make_float2(1.f, 0.f); break;
    case 1: va = c.tr; vb = c.br; a = make_float2(1.f, 0.f); b = make_float2(1.f, 1.f); break;
    case 2: va = c.bl; vb = c.br; a = make_float2(0.f, 1.f); b = make_float2(1.f, 1.f); break;
    default: va = c.tl; vb = c.bl; a = make_float2(0.f, 0.f); b = make_float2(0.f, 1.f); break;
  }
  const float da = va - thr, db = vb - thr;
  const float t = da / (da - db);
  return make_float2(a.x + t * (b.x - a.x), a.y + t * (b.y - a.y));
}

// Exclusive block scan of one int per thread (blockDim.x a multiple of 32, at
// most 1024); returns the thread's offset, *total the sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_sums[lane] = s;  // inclusive
  }
  __syncthreads();
  const int before = (w > 0 ? warp_sums[w - 1] : 0) + x - v;
  *total = warp_sums[nw - 1];
  __syncthreads();  // warp_sums reusable
  return before;
}

__global__ void __launch_bounds__(kRowThreads) k_ms_count(const float* __restrict__ img, int n, float thr,
                                                          int* __restrict__ row_count) {
  const int i = blockIdx.x, p = blockIdx.y;
  const float* plane = img + (size_t)p * n * n;
  int cnt = 0;
  for (int j = threadIdx.x; j < n; j += kRowThreads) cnt += case_segments(cell_case(load_cell(plane, n, i, j), thr));
  int total;
  block_exclusive_scan(cnt, &total);
  if (threadIdx.x == 0) row_count[(size_t)p * n + i] = total;
}

// One CTA per plane: exclusive scan of the plane's row counts into
// row_start (offsets within the plane) and the plane's total.  Chunks of one
// row per thread (contiguous loads and stores), the running total carried.
__global__ void __launch_bounds__(1024) k_ms_scan(const int* __restrict__ row_count, int n,
                                                         long long* __restrict__ row_start,
                                                         long long* __restrict__ plane_total) {
  const size_t base = (size_t)blockIdx.x * n;
  long long run = 0;
  for (int r0 = 0; r0 < n; r0 += blockDim.x) {
    const int r = r0 + threadIdx.x;
    const int c = r < n ? row_count[base + r] : 0;
    int chunk;
    const int before = block_exclusive_scan(c, &chunk);
    if (r < n) row_start[base + r] = run + before;
    run += chunk;
  }
  if (threadIdx.x == 0) plane_total[blockIdx.x] = run;
}

// plane_start[p] = sum of the totals of the planes before p; [planes] = all.
__global__ void k_ms_planes(const long long* __restrict__ plane_total, int planes,
                            long long* __restrict__ plane_start) {
  long long run = 0;
  for (int p = 0; p < planes; ++p) {
    plane_start[p] = run;
    run += plane_total[p];
  }
  plane_start[planes] = run;
}

__global__ void __launch_bounds__(kRowThreads) k_ms_emit(const float* __restrict__ img, int n, float thr,
                                                         const long long* __restrict__ row_start,
                                                         const long long* __restrict__ plane_start,
                                                         long long capacity, float4* __restrict__ seg,
                                                         int* __restrict__ cell_id) {
  __shared__ uint16_t tab[32];
  if (threadIdx.x < 32) tab[threadIdx.x] = kSegTable[threadIdx.x];
  __syncthreads();
  const int i = blockIdx.x, p = blockIdx.y;
  const float* plane = img + (size_t)p * n * n;
  long long base = plane_start[p] + row_start[(size_t)p * n + i];
  for (int j0 = 0; j0 < n; j0 += kRowThreads) {  // uniform trip count: every thread takes part in each scan
    const int j = j0 + threadIdx.x;
    Cell c{0.f, 0.f, 0.f, 0.f};
    uint16_t ent = 0;
    if (j < n) {
      c = load_cell(plane, n, i, j);
      ent = cell_entry(c, thr, tab);
    }
    const int ns = ent >> 8;
    int chunk;
    long long o = base + block_exclusive_scan(ns, &chunk);
    base += chunk;
    for (int k = 0; k < ns; ++k, ++o) {
      if (o >= capacity) continue;
      const int s0 = (ent >> (4 * k)) & 3, e0 = (ent >> (4 * k + 2)) & 3;
      const float2 a = edge_point(c, s0, thr), b = edge_point(c, e0, thr);
      seg[o] = make_float4(j + a.x, i + a.y, j + b.x, i + b.y);
      if (cell_id) cell_id[o] = i * n + j;
    }
  }
}

// Rows whose length is a multiple of 128: a warp walks one row of cells in
// chunks of 128 (lane l: cells 4l .. 4l + 3, one 16-byte load per pixel row;
// the fifth corner comes from the next lane, for lane 31 from the next
// chunk's lane 0, and after the last chunk from the row's first pixel),
// loading the next chunk while it works on the current one.  The count pass
// writes one count per chunk (warp reduction), a per-plane scan turns them
// into offsets, and the emit pass places each lane's segments with a warp
// scan: no block barrier in either pass; grid y = plane, warps over the
// plane's rows in a grid-stride loop.
struct RowWalk {
  const float* ra;  // row i, this lane's first pixel
  const float* rb;  // row i + 1 (periodic)
  float4 a, b;      // current chunk
  float a_first, b_first;  // pixel 0 of the two rows
};

__device__ __forceinline__ RowWalk row_walk_begin(const float* __restrict__ plane, int n, int i, int lane) {
  const int i1 = i + 1 == n ? 0 : i + 1;
  RowWalk w;
  w.ra = plane + (size_t)i * n + 4 * lane;
  w.rb = plane + (size_t)i1 * n + 4 * lane;
  w.a = __ldg(reinterpret_cast<const float4*>(w.ra));
  w.b = __ldg(reinterpret_cast<const float4*>(w.rb));
  w.a_first = __shfl_sync(0xffffffffu, w.a.x, 0);
  w.b_first = __shfl_sync(0xffffffffu, w.b.x, 0);
  return w;
}

// Chunk c + 1 of the row (its loads in flight while chunk c is worked on);
// past the last chunk, values that only supply the wrap-around corner.
struct Chunk2 {
  float4 a, b;
};

__device__ __forceinline__ Chunk2 row_walk_next(const RowWalk& w, int c, int chunks) {
  if (c + 1 < chunks)
    return Chunk2{__ldg(reinterpret_cast<const float4*>(w.ra + 128 * (c + 1))),
                  __ldg(reinterpret_cast<const float4*>(w.rb + 128 * (c + 1)))};
  return Chunk2{make_float4(w.a_first, 0.f, 0.f, 0.f), make_float4(w.b_first, 0.f, 0.f, 0.f)};
}

// The fifth corner of each lane (pixel 4l + 4 of the chunk): from lane l + 1,
// for lane 31 the next chunk's first pixel.
__device__ __forceinline__ void fifth_corner(const float4& a, const float4& b, const float4& na, const float4& nb,
                                             int lane, float* a4, float* b4) {
  *a4 = __shfl_sync(0xffffffffu, lane == 0 ? na.x : a.x, (lane + 1) & 31);
  *b4 = __shfl_sync(0xffffffffu, lane == 0 ? nb.x : b.x, (lane + 1) & 31);
}

// Inside bits of five consecutive pixels (bit k: pixel k >= T).
__device__ __forceinline__ unsigned inside5(const float4& v, float v4, float thr) {
  return unsigned(v.x >= thr) | unsigned(v.y >= thr) << 1 | unsigned(v.z >= thr) << 2 | unsigned(v.w >= thr) << 3 |
         unsigned(v4 >= thr) << 4;
}

// Segments of the lane's four cells from the inside bits of their top and
// bottom pixel rows: a cell's crossed edges number 0, 2 or 4 and it has half
// as many segments, so the four cells have half their total crossings (top
// edges, bottom edges, left edges, right edges).
__device__ __forceinline__ int segments4(unsigned top, unsigned bot) {
  const unsigned v = top ^ bot;
  return (__popc((top ^ (top >> 1)) & 15u) + __popc((bot ^ (bot >> 1)) & 15u) + __popc(v & 15u) + __popc(v & 30u)) >>
         1;
}

__global__ void __launch_bounds__(256, 4) k_ms_count4(const float* __restrict__ img, int n, int planes, float thr,
                                                   int* __restrict__ chunk_count) {
  const int chunks = n / 128, p = blockIdx.y, lane = threadIdx.x & 31;
  const float* plane = img + (size_t)p * n * n;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
    RowWalk w = row_walk_begin(plane, n, i, lane);
    int* out = chunk_count + ((size_t)p * n + i) * chunks;
    for (int c = 0; c < chunks; ++c) {
      const Chunk2 nx = row_walk_next(w, c, chunks);
      const float4 na = nx.a, nb = nx.b;
      float a4, b4;
      fifth_corner(w.a, w.b, na, nb, lane, &a4, &b4);
      int cnt = segments4(inside5(w.a, a4, thr), inside5(w.b, b4, thr));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
      if (lane == 0) out[c] = cnt;
      w.a = na;
      w.b = nb;
    }
  }
}

// Crossing point of edge e (0 top, 1 right, 2 bottom, 3 left) of the cell with
// corners tl, tr, br, bl, in cell-local (x, y); the same interpolation as
// edge_point, without branches.
__device__ __forceinline__ float2 edge_point_sel(float tl, float tr, float br, float bl, int e, float thr) {
  const float va = e == 1 ? tr : e == 2 ? bl : tl;
  const float vb = e == 0 ? tr : e == 3 ? bl : br;
  const float da = va - thr, db = vb - thr;
  const float t = da / (da - db);
  const float ax = e == 1 ? 1.f : 0.f, ay = e == 2 ? 1.f : 0.f;
  const bool horiz = (e & 1) == 0;
  return make_float2(ax + (horiz ? t : 0.f), ay + (horiz ? 0.f : t));
}

// Emit: the warp's segments of a chunk are handed out one per lane in
// rounds of 32 (most chunks need one): segment s belongs to the first lane
// whose inclusive count exceeds s (a binary search over the warp scan), and
// that lane's pixels are read from its slot in shared memory.
constexpr int kEmitWarps = 8;

__global__ void __launch_bounds__(32 * kEmitWarps, 4) k_ms_emit4(const float* __restrict__ img, int n, int planes,
                                                                 float thr, const long long* __restrict__ chunk_start,
                                                                 const long long* __restrict__ plane_start,
                                                                 long long capacity, float4* __restrict__ seg,
                                                                 int* __restrict__ cell_id) {
  __shared__ uint16_t tab[32];
  // per warp: value v of lane l at [v][l] (row i pixels 4l .. 4l + 4 as
  // v = 0..4, row i + 1 as v = 5..9); the odd row length keeps the reads of
  // different lanes and values on different banks
  __shared__ float px[kEmitWarps][10][33];
  if (threadIdx.x < 32) tab[threadIdx.x] = kSegTable[threadIdx.x];
  __syncthreads();
  const int chunks = n / 128, p = blockIdx.y, lane = threadIdx.x & 31;
  float(*mine)[33] = px[threadIdx.x >> 5];
  const float* plane = img + (size_t)p * n * n;
  const long long p0 = plane_start[p];
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
    RowWalk w = row_walk_begin(plane, n, i, lane);
    const long long* starts = chunk_start + ((size_t)p * n + i) * chunks;
    for (int c = 0; c < chunks; ++c) {
      const Chunk2 nx = row_walk_next(w, c, chunks);
      const long long cbase = p0 + __ldg(starts + c);
      float a4, b4;
      fifth_corner(w.a, w.b, nx.a, nx.b, lane, &a4, &b4);
      const unsigned top = inside5(w.a, a4, thr), bot = inside5(w.b, b4, thr);
      const int cnt = segments4(top, bot);
      int x = cnt;  // inclusive warp scan
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const int total = __shfl_sync(0xffffffffu, x, 31);
      if (total > 0) {  // uniform
        mine[0][lane] = w.a.x;
        mine[1][lane] = w.a.y;
        mine[2][lane] = w.a.z;
        mine[3][lane] = w.a.w;
        mine[4][lane] = a4;
        mine[5][lane] = w.b.x;
        mine[6][lane] = w.b.y;
        mine[7][lane] = w.b.z;
        mine[8][lane] = w.b.w;
        mine[9][lane] = b4;
        __syncwarp();
        for (int s0 = 0; s0 < total; s0 += 32) {
          const int s = min(s0 + lane, total - 1);
          int L = 0;  // owner lane: the number of lanes whose inclusive count is <= s
#pragma unroll
          for (int step = 16; step > 0; step >>= 1)
            if (__shfl_sync(0xffffffffu, x, L + step - 1) <= s) L += step;
          const int excl = __shfl_sync(0xffffffffu, x - cnt, L);
          const unsigned tb = __shfl_sync(0xffffffffu, top | bot << 5, L);
          if (s0 + lane < total) {
            const unsigned t5 = tb & 31u, b5 = tb >> 5, v = t5 ^ b5;
            const unsigned h = (t5 ^ (t5 >> 1)) + ((b5 ^ (b5 >> 1)) << 8) + (v << 16) + ((v >> 1) << 24);
            int q = s - excl, k = 0;  // the owner's cell k and its segment q
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
              const int ck = int(((h >> kk) & 1u) + ((h >> (kk + 8)) & 1u) + ((h >> (kk + 16)) & 1u) +
                                 ((h >> (kk + 24)) & 1u)) >> 1;
              if (k == kk && q >= ck) {
                q -= ck;
                k = kk + 1;
              }
            }
            const Cell cl{mine[k][L], mine[k + 1][L], mine[5 + k + 1][L], mine[5 + k][L]};
            const uint16_t ent = tab[cell_case(cl, thr)];
            const int s_e = (ent >> (4 * q)) & 3, e_e = (ent >> (4 * q + 2)) & 3;
            const float2 pa = edge_point_sel(cl.tl, cl.tr, cl.br, cl.bl, s_e, thr);
            const float2 pb = edge_point_sel(cl.tl, cl.tr, cl.br, cl.bl, e_e, thr);
            const long long o = cbase + s;
            const int j = c * 128 + 4 * L + k;
            if (o < capacity) {
              seg[o] = make_float4(j + pa.x, i + pa.y, j + pb.x, i + pb.y);
              if (cell_id) cell_id[o] = i * n + j;
            }
          }
        }
        __syncwarp();  // slots reusable
      }
      w.a = nx.a;
      w.b = nx.b;
    }
  }
}

// ---- Eq. (6) at control points ----------------------------------------------------------------
__device__ __forceinline__ float bilin(float a, float b, float c, float d, float fx, float fy) {
  return (1.f - fy) * ((1.f - fx) * a + fx * b) + fy * ((1.f - fx) * c + fx * d);
}

// Eq. (6) at point r (pixels) of plane I.
__device__ __forceinline__ float epe_at(const float* __restrict__ I, int n, float2 r, float inv_pixel, float thr) {
  const float fj = floorf(r.x), fi = floorf(r.y);
  const float fx = r.x - fj, fy = r.y - fi;
  auto wrap = [&](int v) { return ((v % n) + n) % n; };
  const int j0 = int(fj), i0 = int(fi);
  float v[4][4];  // rows i0-1 .. i0+2, columns j0-1 .. j0+2
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float* row = I + (size_t)wrap(i0 - 1 + a) * n;
#pragma unroll
    for (int b = 0; b < 4; ++b) v[a][b] = ((a == 0 || a == 3) && (b == 0 || b == 3)) ? 0.f : __ldg(row + wrap(j0 - 1 + b));
  }
  const float e = bilin(v[1][1], v[1][2], v[2][1], v[2][2], fx, fy);
  // central differences at the four corners (per pixel)
  const float gx = bilin(0.5f * (v[1][2] - v[1][0]), 0.5f * (v[1][3] - v[1][1]), 0.5f * (v[2][2] - v[2][0]),
                         0.5f * (v[2][3] - v[2][1]), fx, fy);
  const float gy = bilin(0.5f * (v[2][1] - v[0][1]), 0.5f * (v[2][2] - v[0][2]), 0.5f * (v[3][1] - v[1][1]),
                         0.5f * (v[3][2] - v[1][2]), fx, fy);
  const float g = sqrtf(gx * gx + gy * gy) * inv_pixel;
  return g > 0.f ? -(e - thr) / g : __int_as_float(0x7fc00000);
}

// One thread per control point, every plane in turn.
__global__ void k_epe(const float* __restrict__ img, int planes, int n, int m, float inv_pixel, float thr,
                      const float2* __restrict__ pts, float* __restrict__ epe) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const float2 r = pts[k];
  for (int p = 0; p < planes; ++p) epe[(size_t)p * m + k] = epe_at(img + (size_t)p * n * n, n, r, inv_pixel, thr);
}

// All clips' points in one launch: point k belongs to the last clip c with
// start[c] <= k (empty clips are passed over), whose planes follow one another
// in img.  Whatever start holds, c stays in [0, clips).
__global__ void k_epe_batch(const float* __restrict__ img, int clips, int planes, int n, long long m, float inv_pixel,
                            float thr, const float2* __restrict__ pts, const long long* __restrict__ start,
                            float* __restrict__ epe) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= m) return;
  int lo = 0, hi = clips - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= k)
      lo = mid;
    else
      hi = mid - 1;
  }
  const float2 r = pts[k];
  const float* I = img + (size_t)lo * planes * n * n;
  for (int p = 0; p < planes; ++p) epe[(size_t)p * m + k] = epe_at(I + (size_t)p * n * n, n, r, inv_pixel, thr);
}

__global__ void k_epe_focus(const float* __restrict__ epe, int m, int f0, int fp, int fn, float tol_neg,
                            float tol_pos, float* __restrict__ avg, float* __restrict__ eff) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const float e0 = epe[(size_t)f0 * m + k];
  const float a = (e0 + epe[(size_t)fp * m + k] + epe[(size_t)fn * m + k]) / 3.f;
  if (avg) avg[k] = a;
  if (eff) eff[k] = e0 > tol_pos ? e0 - tol_pos : e0 < tol_neg ? e0 - tol_neg : a;
}

}  // namespace

// Units the count pass produces per plane: rows (one-cell-per-thread path) or
// 128-cell chunks (rows a multiple of 128).
static bool contour_vec(int n) { return n % 128 == 0 && n <= 65536; }
static size_t contour_units(int n) { return contour_vec(n) ? size_t(n) * (n / 128) : size_t(n); }

size_t contour_workspace_bytes(int planes, int n) {
  const size_t units = size_t(planes) * contour_units(n);
  return (units * sizeof(int) + 255) / 256 * 256 + (units * sizeof(long long) + 255) / 256 * 256 +
         size_t(planes) * sizeof(long long);
}

cudaError_t launch_contours(const float* img, int planes, int n, float thr, float4* seg, int* cell_id,
                            long long capacity, long long* plane_start, void* ws, cudaStream_t st) {
  const bool vec = contour_vec(n) && (reinterpret_cast<uintptr_t>(img) & 15) == 0;
  const size_t per_plane = vec ? contour_units(n) : size_t(n);
  // the workspace is sized for the larger (vector) layout when n allows it
  const size_t sized = size_t(planes) * contour_units(n);
  char* w = static_cast<char*>(ws);
  int* count = reinterpret_cast<int*>(w);
  long long* start = reinterpret_cast<long long*>(w + (sized * sizeof(int) + 255) / 256 * 256);
  long long* plane_total = reinterpret_cast<long long*>(w + (sized * sizeof(int) + 255) / 256 * 256 +
                                                        (sized * sizeof(long long) + 255) / 256 * 256);
  if (vec) {
    const int blocks = (n + 7) / 8;  // a warp per row of cells
    k_ms_count4<<<dim3(blocks, planes), 256, 0, st>>>(img, n, planes, thr, count);
    k_ms_scan<<<planes, 1024, 0, st>>>(count, int(per_plane), start, plane_total);
    k_ms_planes<<<1, 1, 0, st>>>(plane_total, planes, plane_start);
    k_ms_emit4<<<dim3(blocks, planes), 256, 0, st>>>(img, n, planes, thr, start, plane_start, capacity, seg, cell_id);
  } else {
    k_ms_count<<<dim3(n, planes), kRowThreads, 0, st>>>(img, n, thr, count);
    k_ms_scan<<<planes, kRowThreads, 0, st>>>(count, n, start, plane_total);
    k_ms_planes<<<1, 1, 0, st>>>(plane_total, planes, plane_start);
    k_ms_emit<<<dim3(n, planes), kRowThreads, 0, st>>>(img, n, thr, start, plane_start, capacity, seg, cell_id);
  }
  return cudaGetLastError();
}

cudaError_t launch_epe(const float* img, int planes, int n, float pixel_nm, float thr, const float2* pts, int m,
                       float* epe, cudaStream_t st) {
  k_epe<<<(m + 255) / 256, 256, 0, st>>>(img, planes, n, m, 1.0f / pixel_nm, thr, pts, epe);
  return cudaGetLastError();
}

cudaError_t launch_epe_batch(const float* img, int clips, int planes, int n, float pixel_nm, float thr,
                             const float2* pts, const long long* start, long long m, float* epe, cudaStream_t st) {
  k_epe_batch<<<unsigned((m + 255) / 256), 256, 0, st>>>(img, clips, planes, n, m, 1.0f / pixel_nm, thr, pts, start,
                                                        epe);
  return cudaGetLastError();
}

cudaError_t launch_epe_focus(const float* epe, int m, int f0, int fp, int fn, float tol_neg, float tol_pos,
                             float* avg, float* eff, cudaStream_t st) {
  k_epe_focus<<<(m + 255) / 256, 256, 0, st>>>(epe, m, f0, fp, fn, tol_neg, tol_pos, avg, eff);
  return cudaGetLastError();
}

}  // namespace litho
