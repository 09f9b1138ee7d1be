"""Oracle area-coverage rasterisation of rectangle masks (FP64).

Test infrastructure only (see the package docstring).

The mask m of Eq. (1) as a grey level per pixel: the fraction of pixel (i, j)
= [j, j+1) x [i, i+1) (x = column, y = row, pixel units) covered by the union
of axis-aligned rectangles [x0, x1) x [y0, y1), periodic with period N (a
rectangle running past N continues at 0).  Overlapping rectangles count
once (an OR of the shapes, as the centre-sampled rasteriser does for whole
pixels).

Written as coordinate compression: every rectangle edge and every pixel
boundary becomes a grid line, each cell of that grid is either inside the
union or not (tested at its centre), and covered cells add their area to the
pixel that contains them.  A pixel's coverage is exact up to the rounding of
the cell areas.
"""
from __future__ import annotations

import numpy as np


def _pieces(rects, n):
    """Split rectangles at the period so that every piece lies in [0, n] x [0, n]."""
    out = []
    for x0, y0, x1, y1 in rects:
        sx = np.floor(x0 / n) * n
        sy = np.floor(y0 / n) * n
        x0, x1, y0, y1 = x0 - sx, x1 - sx, y0 - sy, y1 - sy
        xs = [(x0, min(x1, n))] + ([(0.0, x1 - n)] if x1 > n else [])
        ys = [(y0, min(y1, n))] + ([(0.0, y1 - n)] if y1 > n else [])
        for a, b in xs:
            for c, d in ys:
                if b > a and d > c:
                    out.append((a, c, b, d))
    return np.array(out, dtype=np.float64).reshape(-1, 4)


def coverage(n: int, rects) -> np.ndarray:
    """Exact area coverage [n][n] of the union of rectangles (x0, y0, x1, y1) in pixels
    (widths and heights at most n)."""
    pcs = _pieces(np.asarray(rects, dtype=np.float64).reshape(-1, 4), n)
    grid = np.arange(n + 1, dtype=np.float64)
    xs = np.unique(np.concatenate([grid, pcs[:, 0], pcs[:, 2]]))
    ys = np.unique(np.concatenate([grid, pcs[:, 1], pcs[:, 3]]))
    cx = 0.5 * (xs[:-1] + xs[1:])
    cy = 0.5 * (ys[:-1] + ys[1:])
    inside = np.zeros((len(cy), len(cx)), dtype=bool)
    for x0, y0, x1, y1 in pcs:
        inside |= ((cy >= y0) & (cy < y1))[:, None] & ((cx >= x0) & (cx < x1))[None, :]
    area = np.diff(ys)[:, None] * np.diff(xs)[None, :] * inside
    out = np.zeros((n, n))
    np.add.at(out, (np.floor(cy).astype(int)[:, None], np.floor(cx).astype(int)[None, :]), area)
    return out
