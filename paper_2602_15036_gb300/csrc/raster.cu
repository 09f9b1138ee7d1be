// Area-coverage rasterisation of rectangle masks: m[i][j] = area of the union
// of the rectangles [x0, x1) x [y0, y1) inside pixel [j, j+1) x [i, i+1)
// (pixel units, periodic with period N, overlaps counted once).  The grey-
// level mask is the object of Eq. (1) for shapes off the pixel grid.
//
// Five launches per batch: every rectangle is split at the period into at
// most four pieces and each piece counted into the 16 x 16-pixel tiles it
// touches (atomics), one CTA per clip scans the tile counts, one thread
// places the clips' lists one after another, the pieces are filed into their
// tiles' lists, and one CTA per tile computes its 256 pixels.  The lists fit
// the workspace by construction: a rectangle with sides of at most S pixels
// reaches at most (ceil(S/16) + 5)^2 tiles; a larger or empty rectangle
// marks its clip, whose mask is then written as NaN.  A pixel's value is
// exact up to FP32 rounding: empty and fully covered pixels are recognised
// directly; otherwise the pixel is swept in x
// between consecutive piece edges, and in each slab the union length in y of
// the pieces spanning it is measured by walking up through their intervals.
// The result does not depend on the order of a tile's list.
#include <cstdint>

#include "litho_internal.h"

namespace litho {

namespace {

constexpr int kTile = 16, kTileThreads = kTile * kTile;
// tile kernel: 64 threads, 4 pixels each, and a 256-piece cache (larger
// lists are read from global memory), so that 32 tiles fit on an SM
constexpr int kRastThreads = 64, kRastPix = kTile * kTile / kRastThreads, kTileCache = 256;

// Pieces of rectangle r (x0, y0, x1, y1) after the shift into [0, n) and the
// split at n; calls f(piece) for each nonempty one.
template <class F>
__device__ __forceinline__ void for_pieces(float4 r, int n, F&& f) {
  const float fn = float(n);
  const float sx = floorf(r.x / fn) * fn, sy = floorf(r.y / fn) * fn;
  const float x0 = r.x - sx, x1 = r.z - sx, y0 = r.y - sy, y1 = r.w - sy;
  const float xa[2] = {x0, 0.f}, xb[2] = {fminf(x1, fn), x1 - fn};
  const float ya[2] = {y0, 0.f}, yb[2] = {fminf(y1, fn), y1 - fn};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      if (xb[a] > xa[a] && yb[b] > ya[b]) f(make_float4(xa[a], ya[b], xb[a], yb[b]));
}

template <bool FILL>
__global__ void k_rast_bin(const float4* __restrict__ rects, const long long* __restrict__ rect_start, int n,
                           long long max_rects, float max_side, int* __restrict__ count, const int* __restrict__ tile_start,
                           const long long* __restrict__ clip_base, int* __restrict__ cursor,
                           float4* __restrict__ list, int* __restrict__ bad) {
  const int c = blockIdx.y, tiles = n / kTile;
  if (!FILL && blockIdx.x == 0 && threadIdx.x == 0 && rect_start[c + 1] - rect_start[c] > max_rects) bad[c] = 1;
  const long long r = rect_start[c] + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rect_start[c + 1]) return;
  const float4 rc = rects[r];
  // NaN-safe: anything but 0 < side <= max_side marks the clip
  if (!(rc.z - rc.x > 0.f && rc.z - rc.x <= max_side && rc.w - rc.y > 0.f && rc.w - rc.y <= max_side)) {
    if (!FILL) bad[c] = 1;
    return;
  }
  for_pieces(rc, n, [&](float4 p) {
    // tiles of the first and last pixel the piece reaches (p.x, p.y in [0, n))
    const int tx0 = int(p.x) / kTile, tx1 = min(n - 1, int(ceilf(p.z)) - 1) / kTile;
    const int ty0 = int(p.y) / kTile, ty1 = min(n - 1, int(ceilf(p.w)) - 1) / kTile;
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx) {
        const size_t t = (size_t)c * tiles * tiles + (size_t)ty * tiles + tx;
        if (!FILL) {
          atomicAdd(count + t, 1);
        } else {
          list[clip_base[c] + tile_start[t] + atomicAdd(cursor + t, 1)] = p;
        }
      }
  });
}

// One CTA per clip: exclusive scan of its tile counts (cursor cleared).
__global__ void __launch_bounds__(kTileThreads) k_rast_scan(const int* __restrict__ count, int tiles2, int* __restrict__ tile_start,
                                                            int* __restrict__ cursor, int* __restrict__ total) {
  __shared__ int warp_sums[kTileThreads / 32];
  const int c = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t base = (size_t)c * tiles2;
  int run = 0;
  for (int t0 = 0; t0 < tiles2; t0 += kTileThreads) {
    const int t = t0 + threadIdx.x;
    const int v = t < tiles2 ? count[base + t] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
      int s = lane < kTileThreads / 32 ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      if (lane < kTileThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    if (t < tiles2) {
      tile_start[base + t] = run + (w > 0 ? warp_sums[w - 1] : 0) + x - v;
      cursor[base + t] = 0;
    }
    run += warp_sums[kTileThreads / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) total[c] = run;
}

// Offsets of the clips' lists: clip_base[c] = sum of the totals before c.
__global__ void k_rast_base(const int* __restrict__ total, int b, long long* __restrict__ clip_base) {
  long long run = 0;
  for (int c = 0; c < b; ++c) {
    clip_base[c] = run;
    run += total[c];
  }
  clip_base[b] = run;
}

// 1 when one piece covers the unit pixel at (px, py), 0 when none reaches
// into it, else -1 (a grey pixel: pixel_area measures it).
__device__ __forceinline__ float pixel_class(const float4* pcs, int np, float px, float py) {
  const float X1 = px + 1.f, Y1 = py + 1.f;
  bool any = false;
  for (int k = 0; k < np; ++k) {
    const float4 p = pcs[k];
    if (p.x <= px && p.z >= X1 && p.y <= py && p.w >= Y1) return 1.f;
    any |= p.x < X1 && p.z > px && p.y < Y1 && p.w > py;
  }
  return any ? -1.f : 0.f;
}

// Union area of the pieces within the unit pixel at (px, py).
__device__ float pixel_area(const float4* pcs, int np, float px, float py) {
  const float X1 = px + 1.f, Y1 = py + 1.f;
  float area = 0.f, xa = px;
  while (xa < X1) {
    float xb = X1;  // next piece edge above xa
    for (int k = 0; k < np; ++k) {
      const float4 p = pcs[k];
      if (p.y >= Y1 || p.w <= py) continue;
      if (p.x > xa && p.x < xb) xb = p.x;
      if (p.z > xa && p.z < xb) xb = p.z;
    }
    // union length in y of the pieces spanning [xa, xb)
    float len = 0.f, y = py;
    while (y < Y1) {
      float top = -1.f, next = Y1;
      for (int k = 0; k < np; ++k) {
        const float4 p = pcs[k];
        if (p.x > xa || p.z < xb) continue;
        if (p.y <= y && p.w > y) top = fmaxf(top, fminf(p.w, Y1));
        else if (p.y > y && p.y < next) next = p.y;
      }
      if (top > y) {
        len += top - y;
        y = top;
      } else {
        y = next;
      }
    }
    area += (xb - xa) * len;
    xa = xb;
  }
  return area;
}

__global__ void __launch_bounds__(kRastThreads) k_rast_tiles(const float4* __restrict__ list, const int* __restrict__ count,
                                                             const int* __restrict__ tile_start,
                                                             const long long* __restrict__ clip_base,
                                                             const int* __restrict__ bad, int n,
                                                             float* __restrict__ mask) {
  __shared__ float4 cache[kTileCache];
  __shared__ int grey[kTile * kTile];
  __shared__ int n_grey;
  const int tiles = n / kTile, c = blockIdx.y, t = blockIdx.x;
  const size_t ti = (size_t)c * tiles * tiles + t;
  const int ty = t / tiles, tx = t % tiles;
  // pixel q = threadIdx.x + r * kRastThreads of the tile (row q / 16, column q % 16)
  auto at = [&](int q) -> float* { return mask + ((size_t)c * n + ty * kTile + q / kTile) * n + tx * kTile + q % kTile; };
  // the flag and the tile's list are fetched together (a flagged clip's
  // counts are read but its list is not)
  const int flagged = bad[c], np = count[ti];
  const float4* pcs = list + clip_base[c] + tile_start[ti];
  if (flagged) {  // uniform across the block
#pragma unroll
    for (int r = 0; r < kRastPix; ++r) *at(threadIdx.x + r * kRastThreads) = __int_as_float(0x7fc00000);
    return;
  }
  if (threadIdx.x == 0) n_grey = 0;
  if (np <= kTileCache) {
    for (int k = threadIdx.x; k < np; k += kRastThreads) cache[k] = pcs[k];
    pcs = cache;
  }
  __syncthreads();
  // empty and fully covered pixels at once; the grey ones are gathered so
  // that whole warps run their sweeps
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < kRastPix; ++r) {
    const int q = threadIdx.x + r * kRastThreads;
    const float cls = pixel_class(pcs, np, float(tx * kTile + q % kTile), float(ty * kTile + q / kTile));
    const unsigned m = __ballot_sync(0xffffffffu, cls < 0.f);
    int slot = 0;
    if (lane == 0 && m) slot = atomicAdd(&n_grey, __popc(m));
    slot = __shfl_sync(0xffffffffu, slot, 0) + __popc(m & ((1u << lane) - 1u));
    if (cls < 0.f)
      grey[slot] = q;
    else
      *at(q) = cls;
  }
  __syncthreads();
  for (int g = threadIdx.x; g < n_grey; g += kRastThreads) {
    const int q = grey[g];
    *at(q) = pixel_area(pcs, np, float(tx * kTile + q % kTile), float(ty * kTile + q / kTile));
  }
}

// Workspace: per-tile counts, starts and cursors, the clips' flags, totals and
// list offsets, then the piece lists.
struct RasterLayout {
  int *count, *tile_start, *cursor, *bad, *total;
  long long* clip_base;
  float4* list;
  size_t bytes;
};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

RasterLayout raster_layout(int b, int n, long long max_rects, int max_side, void* ws) {
  char* p = static_cast<char*>(ws);
  const size_t tiles2 = size_t(n / kTile) * (n / kTile) * b;
  const long long per_rect = raster_tiles_per_rect(max_side);
  RasterLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    void* q = p ? p + o : nullptr;
    o += up256(bytes);
    return q;
  };
  L.count = static_cast<int*>(take(tiles2 * sizeof(int)));
  L.tile_start = static_cast<int*>(take(tiles2 * sizeof(int)));
  L.cursor = static_cast<int*>(take(tiles2 * sizeof(int)));
  L.bad = static_cast<int*>(take(size_t(b) * sizeof(int)));
  L.total = static_cast<int*>(take(size_t(b) * sizeof(int)));
  L.clip_base = static_cast<long long*>(take(size_t(b + 1) * sizeof(long long)));
  L.list = static_cast<float4*>(take(size_t(b) * size_t(max_rects) * size_t(per_rect) * sizeof(float4)));
  L.bytes = o;
  return L;
}

}  // namespace

// Tiles one rectangle with sides of at most s pixels can reach once split at
// the period: at most ceil(s/16) + 5 per axis.
long long raster_tiles_per_rect(int s) {
  const long long a = (s + kTile - 1) / kTile + 5;
  return a * a;
}

size_t raster_workspace_bytes(int b, int n, long long max_rects, int max_side) {
  return raster_layout(b, n, max_rects, max_side, nullptr).bytes;
}

cudaError_t launch_raster(const float4* rects, const long long* rect_start, int b, long long max_rects,
                          int max_side, int n, float* mask, void* ws, cudaStream_t st) {
  const RasterLayout L = raster_layout(b, n, max_rects, max_side, ws);
  const int tiles = n / kTile;
  const size_t tiles2 = size_t(tiles) * tiles;
  cudaError_t e = cudaMemsetAsync(L.count, 0, tiles2 * b * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.bad, 0, size_t(b) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (max_rects > 0) {
    const dim3 grid(unsigned((max_rects + 255) / 256), b);
    k_rast_bin<false><<<grid, 256, 0, st>>>(rects, rect_start, n, max_rects, float(max_side), L.count, nullptr, nullptr,
                                            nullptr, nullptr, L.bad);
  }
  k_rast_scan<<<b, kTileThreads, 0, st>>>(L.count, int(tiles2), L.tile_start, L.cursor, L.total);
  k_rast_base<<<1, 1, 0, st>>>(L.total, b, L.clip_base);
  if (max_rects > 0) {
    const dim3 grid(unsigned((max_rects + 255) / 256), b);
    k_rast_bin<true><<<grid, 256, 0, st>>>(rects, rect_start, n, max_rects, float(max_side), L.count, L.tile_start,
                                           L.clip_base, L.cursor, L.list, L.bad);
  }
  k_rast_tiles<<<dim3(unsigned(tiles2), b), kRastThreads, 0, st>>>(L.list, L.count, L.tile_start, L.clip_base, L.bad,
                                                                   n, mask);
  return cudaGetLastError();
}

}  // namespace litho
