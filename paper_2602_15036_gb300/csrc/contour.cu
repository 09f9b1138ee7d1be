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
// Three launches, all deterministic: per row of cells the number of segments,
// one CTA scanning the row counts of every plane into global offsets, and per
// row again the segments written at those offsets in row-major cell order
// (saddle segments ordered by their start edge).  A row CTA walks its row in
// chunks of one cell per thread, so the corner loads and the segment stores
// of a warp are contiguous; a block scan per chunk places the segments.
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

__device__ __forceinline__ uint16_t cell_entry(const Cell& c, float thr) {
  const int cs = (c.tl >= thr) | (c.tr >= thr) << 1 | (c.br >= thr) << 2 | (c.bl >= thr) << 3;
  if (cs == 5 || cs == 10) {
    const float centre = ((c.tl + c.tr) + (c.br + c.bl)) * 0.25f;
    if (!(centre >= thr)) return kSegTable[16 + cs];
  }
  return kSegTable[cs];
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

// Exclusive block scan of one int per thread; returns the thread's offset, *total the sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[kRowThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < kRowThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kRowThreads / 32) warp_sums[lane] = s;  // inclusive
  }
  __syncthreads();
  const int before = (w > 0 ? warp_sums[w - 1] : 0) + x - v;
  *total = warp_sums[kRowThreads / 32 - 1];
  __syncthreads();  // warp_sums reusable
  return before;
}

__global__ void __launch_bounds__(kRowThreads) k_ms_count(const float* __restrict__ img, int n, float thr,
                                                          int* __restrict__ row_count) {
  const int i = blockIdx.x, p = blockIdx.y;
  const float* plane = img + (size_t)p * n * n;
  int cnt = 0;
  for (int j = threadIdx.x; j < n; j += kRowThreads) cnt += cell_entry(load_cell(plane, n, i, j), thr) >> 8;
  int total;
  block_exclusive_scan(cnt, &total);
  if (threadIdx.x == 0) row_count[(size_t)p * n + i] = total;
}

// One CTA: exclusive scan of all rows' counts (planes * n of them) into
// row_start, and plane_start[p] = row_start[p n], plane_start[planes] = total.
// Chunks of one row per thread (contiguous loads and stores), a block scan
// per chunk, the running total carried from chunk to chunk.
__global__ void __launch_bounds__(kRowThreads) k_ms_scan(const int* __restrict__ row_count, long long rows, int n,
                                                         int planes, long long* __restrict__ row_start,
                                                         long long* __restrict__ plane_start) {
  long long run = 0;
  for (long long r0 = 0; r0 < rows; r0 += kRowThreads) {
    const long long r = r0 + threadIdx.x;
    const int c = r < rows ? row_count[r] : 0;
    int chunk;
    const int before = block_exclusive_scan(c, &chunk);
    if (r < rows) row_start[r] = run + before;
    run += chunk;
  }
  __syncthreads();
  if (threadIdx.x == 0) plane_start[planes] = run;
  for (int p = threadIdx.x; p < planes; p += kRowThreads) plane_start[p] = row_start[(long long)p * n];
}

__global__ void __launch_bounds__(kRowThreads) k_ms_emit(const float* __restrict__ img, int n, float thr,
                                                         const long long* __restrict__ row_start,
                                                         long long capacity, float4* __restrict__ seg,
                                                         int* __restrict__ cell_id) {
  const int i = blockIdx.x, p = blockIdx.y;
  const float* plane = img + (size_t)p * n * n;
  long long base = row_start[(size_t)p * n + i];
  for (int j0 = 0; j0 < n; j0 += kRowThreads) {  // uniform trip count: every thread takes part in each scan
    const int j = j0 + threadIdx.x;
    Cell c{0.f, 0.f, 0.f, 0.f};
    uint16_t ent = 0;
    if (j < n) {
      c = load_cell(plane, n, i, j);
      ent = cell_entry(c, thr);
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

// ---- Eq. (6) at control points ----------------------------------------------------------------
__device__ __forceinline__ float bilin(float a, float b, float c, float d, float fx, float fy) {
  return (1.f - fy) * ((1.f - fx) * a + fx * b) + fy * ((1.f - fx) * c + fx * d);
}

// One thread per control point, every plane in turn.
__global__ void k_epe(const float* __restrict__ img, int planes, int n, int m, float inv_pixel, float thr,
                      const float2* __restrict__ pts, float* __restrict__ epe) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const float2 r = pts[k];
  for (int p = 0; p < planes; ++p) {
  const float* I = img + (size_t)p * n * n;
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
  epe[(size_t)p * m + k] = g > 0.f ? -(e - thr) / g : __int_as_float(0x7fc00000);
  }
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

size_t contour_workspace_bytes(int planes, int n) {
  const size_t rows = size_t(planes) * n;
  return (rows * sizeof(int) + 255) / 256 * 256 + rows * sizeof(long long);
}

cudaError_t launch_contours(const float* img, int planes, int n, float thr, float4* seg, int* cell_id,
                            long long capacity, long long* plane_start, void* ws, cudaStream_t st) {
  const size_t rows = size_t(planes) * n;
  int* row_count = static_cast<int*>(ws);
  long long* row_start =
      reinterpret_cast<long long*>(static_cast<char*>(ws) + (rows * sizeof(int) + 255) / 256 * 256);
  k_ms_count<<<dim3(n, planes), kRowThreads, 0, st>>>(img, n, thr, row_count);
  k_ms_scan<<<1, kRowThreads, 0, st>>>(row_count, (long long)rows, n, planes, row_start, plane_start);
  k_ms_emit<<<dim3(n, planes), kRowThreads, 0, st>>>(img, n, thr, row_start, capacity, seg, cell_id);
  return cudaGetLastError();
}

cudaError_t launch_epe(const float* img, int planes, int n, float pixel_nm, float thr, const float2* pts, int m,
                       float* epe, cudaStream_t st) {
  k_epe<<<(m + 255) / 256, 256, 0, st>>>(img, planes, n, m, 1.0f / pixel_nm, thr, pts, epe);
  return cudaGetLastError();
}

cudaError_t launch_epe_focus(const float* epe, int m, int f0, int fp, int fn, float tol_neg, float tol_pos,
                             float* avg, float* eff, cudaStream_t st) {
  k_epe_focus<<<(m + 255) / 256, 256, 0, st>>>(epe, m, f0, fp, fn, tol_neg, tol_pos, avg, eff);
  return cudaGetLastError();
}

}  // namespace litho
