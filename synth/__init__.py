"""Seeded synthetic inputs shared by the FP64 oracle, the tests and the benchmark.

This module only draws random numbers and rasterises shapes; it holds none of
the imaging, resist or gradient arithmetic.  Both sides of every parity test
take their inputs from here, so a mask or a theta field seen by the CUDA path
is bit-identical to the one seen by the oracle.

Random numbers come from the counter form of SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
i-th draw of a stream with seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15)
modulo 2**64, with the published 64-bit finaliser as `mix`.

The paper's IMEC layouts are not available, so these generators stand in for
them (Manhattan rectangles for the OPC clips, smooth blobs for the curvilinear
ILT clips).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws `count` 64-bit words, positions start..start+count-1 of stream `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def words(self, count: int) -> np.ndarray:
        w = splitmix64(self.seed, self.pos, count)
        self.pos += count
        return w

    def uniform(self, count: int) -> np.ndarray:
        """U[0,1) doubles from the top 53 bits."""
        return (self.words(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def integers(self, lo: int, hi: int, count: int) -> np.ndarray:
        """U{lo..hi} inclusive (modulo reduction; the bias is below 2**-50)."""
        span = np.uint64(hi - lo + 1)
        return (self.words(count) % span).astype(np.int64) + lo


def rasterize_rects(n: int, rects: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
    """OR-rasterises axis-aligned rectangles (x0, y0, w, h) in pixels, periodic wrap.

    A pixel is covered when its centre lies inside the rectangle; with integer
    corners that is pixels x0..x0+w-1 by y0..y0+h-1.
    """
    m = np.zeros((n, n), dtype=np.float32) if out is None else out
    for x0, y0, w, h in rects:
        xs = (np.arange(x0, x0 + w) % n)
        ys = (np.arange(y0, y0 + h) % n)
        m[np.ix_(ys, xs)] = 1.0
    return m


def random_rect_mask(n: int, seed: int, count: int = 40, side_lo: int = 5, side_hi: int = 15) -> np.ndarray:
    """`count` rectangles with sides U{side_lo..side_hi} px, corners U over the grid.

    Draw order per rectangle: width, height, x0, y0.
    """
    st = Stream(seed)
    rects = []
    for _ in range(count):
        w, h = st.integers(side_lo, side_hi, 2)
        x0, y0 = st.integers(0, n - 1, 2)
        rects.append((int(x0), int(y0), int(w), int(h)))
    return rasterize_rects(n, np.array(rects))


def manhattan_rects(n: int, seed: int, density: float = 0.35, side_lo: int = 5, side_hi: int = 15,
                    block: int = 64):
    """Rectangles as in `random_rect_mask`, added in blocks of `block` until the
    covered fraction reaches `density` (checked after each block).  Returns
    (rects [R][4] as integer (x0, y0, w, h), the centre-sampled mask).

    Draw order per block: `block` (width, height) pairs, then `block` (x0, y0)
    pairs.  Coverage is counted incrementally (newly covered pixels per rectangle).
    """
    st = Stream(seed)
    m = np.zeros((n, n), dtype=np.float32)
    covered = 0
    target = density * n * n
    rects = []
    while covered < target:
        wh = st.integers(side_lo, side_hi, 2 * block).reshape(block, 2)
        xy = st.integers(0, n - 1, 2 * block).reshape(block, 2)
        for (w, h), (x0, y0) in zip(wh, xy):
            rects.append((int(x0), int(y0), int(w), int(h)))
            if x0 + w <= n and y0 + h <= n:
                view = m[y0:y0 + h, x0:x0 + w]
                covered += int(view.size - np.count_nonzero(view))
                view[...] = 1.0
            else:
                ix = np.ix_(np.arange(y0, y0 + h) % n, np.arange(x0, x0 + w) % n)
                covered += int(w * h - np.count_nonzero(m[ix]))
                m[ix] = 1.0
    return np.array(rects, dtype=np.int64).reshape(-1, 4), m


def manhattan_mask(n: int, seed: int, density: float = 0.35, side_lo: int = 5, side_hi: int = 15,
                   block: int = 64) -> np.ndarray:
    """The centre-sampled mask of `manhattan_rects`."""
    return manhattan_rects(n, seed, density, side_lo, side_hi, block)[1]


def blob_field(n: int, pixel_nm: float, seed: int, count: int = 60, r_lo_nm: float = 30.0,
               r_hi_nm: float = 80.0) -> np.ndarray:
    """Sum of `count` periodic Gaussian blobs, normalised to [0, 1].

    Centres U over the grid (in pixels), radii U[r_lo, r_hi] nm used as the
    Gaussian standard deviation.  Distances wrap around the clip.
    Draw order per blob: cx, cy, radius.
    """
    st = Stream(seed)
    u = st.uniform(3 * count).reshape(count, 3)
    j = np.arange(n, dtype=np.float64)
    b = np.zeros((n, n), dtype=np.float64)
    for cx, cy, ru in u:
        cx *= n
        cy *= n
        r = (r_lo_nm + (r_hi_nm - r_lo_nm) * ru) / pixel_nm
        dx = np.abs(j - cx)
        dx = np.minimum(dx, n - dx)
        dy = np.abs(j - cy)
        dy = np.minimum(dy, n - dy)
        b += np.exp(-0.5 * (dy[:, None] ** 2 + dx[None, :] ** 2) / (r * r))
    b -= b.min()
    mx = b.max()
    if mx > 0:
        b /= mx
    return b


def ilt_clip(n: int, pixel_nm: float, seed: int):
    """ILT inputs: theta0 = 2 (B - 0.5) and target = [B >= 0.5] from one blob field B."""
    b = blob_field(n, pixel_nm, seed)
    target = (b >= 0.5).astype(np.float32)
    theta0 = (2.0 * (b - 0.5)).astype(np.float32)
    return theta0, target


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Plain U[lo, hi) doubles, for property tests."""
    st = Stream(seed)
    return lo + (hi - lo) * st.uniform(int(np.prod(shape))).reshape(shape)


def edge_sites(target: np.ndarray, stride: int = 1) -> np.ndarray:
    """Control points on the edges of a binary target raster: the midpoint of
    every pixel boundary whose two pixels differ (periodic), as (x, y) in pixel
    units (x = column, y = row), vertical boundaries (x = j + 0.5) first, each
    set in row-major order, then every `stride`-th point.  Input construction
    only (the targets' segment control points); float64 [M][2]."""
    t = np.asarray(target) != 0
    i, j = np.nonzero(t != np.roll(t, -1, axis=1))
    vert = np.stack([j + 0.5, i.astype(np.float64)], axis=1)
    i, j = np.nonzero(t != np.roll(t, -1, axis=0))
    horz = np.stack([j.astype(np.float64), i + 0.5], axis=1)
    pts = np.concatenate([vert, horz], axis=0)
    return pts[::stride].copy()
