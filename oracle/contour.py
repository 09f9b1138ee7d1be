"""Oracle contours and edge-placement error (FP64, plain Python/numpy).

Test infrastructure only (see the package docstring).

Section II.D: the printed contour is the level set {I_b = T} of the resist
image (Eq. (5)), traced with marching squares.  Readings used here (and by
the library):

* Cells are the N x N squares whose corners are the pixel centres (i, j),
  (i, j+1), (i+1, j+1), (i+1, j) in (row, column) order, periodic.  A corner is
  inside when I_b >= T (the printed side).  Points are (x, y) = (column, row).
* A cell edge whose two corners differ is crossed at the point given by
  linear interpolation of I_b - T along it.  Edges: 0 top (TL-TR), 1 right
  (TR-BR), 2 bottom (BL-BR), 3 left (TL-BL).
* Two crossed edges give one segment.  Four (a saddle: only TL and BR, or
  only TR and BL, inside) give two: when the mean of the four corners is >= T
  the inside corners are joined through the centre (each segment cuts off one
  outside corner), otherwise each segment cuts off one inside corner.
* Orientation: a segment that cuts off one corner q has q on its left when q
  is inside and on its right when q is outside; a segment between opposite
  edges has the inside pair on its left.  "Left of p0 -> p1" means
  cross(p1 - p0, q - p0) > 0 with cross(a, b) = a.x b.y - a.y b.x.
* Output order: cells row-major; the segments of a saddle cell ordered by the
  edge their start point lies on.
* Decisions (inside, and the saddle's centre test) are taken in the image's
  own precision: the threshold is rounded to the image's type, and the centre
  value is ((v_TL + v_TR) + (v_BR + v_BL)) * 0.25 in that type, so an FP32
  image gives the same decisions here as in the FP32 kernel.

Eq. (6): EPE(r) = -(E_eff(r) - E_tgt(r)) / |grad E_eff(r)|, read with E_eff
the resist image I_b, E_tgt(r) = T at a control point r on a target edge
(the target edge is where the latent image should reach the threshold), I_b
and its gradient evaluated by bilinear interpolation of I_b and of its
central differences (periodic), gradients per nm.  Eq. (7): the mean over the
on-focus and the two defocused planes.  Eq. (8): the piecewise rule, with the
boundary values (e0 = tol) taken by the average branch.
"""
from __future__ import annotations

import math

import numpy as np

# corners of a cell relative to its top-left pixel: (dy, dx)
_TL, _TR, _BR, _BL = (0, 0), (0, 1), (1, 1), (1, 0)
_EDGE_CORNERS = {0: (_TL, _TR), 1: (_TR, _BR), 2: (_BL, _BR), 3: (_TL, _BL)}


def _cross(a, b):
    return a[0] * b[1] - a[1] * b[0]


def _cell_segments(v, thr):
    """Segments of one cell.  v[(dy, dx)] are the four corner values and thr the
    threshold, all of the image's type; returns [((x0, y0), (x1, y1), e0, e1)] in
    cell-local coordinates (corner TL at (0, 0))."""
    inside = {c: v[c] >= thr for c in v}
    pts = {}
    for e, (a, b) in _EDGE_CORNERS.items():
        if inside[a] != inside[b]:
            va, vb = float(v[a]) - float(thr), float(v[b]) - float(thr)
            t = va / (va - vb)
            pts[e] = (a[1] + t * (b[1] - a[1]), a[0] + t * (b[0] - a[0]))  # (x, y)
    if not pts:
        return []
    if len(pts) == 2:
        pairs = [tuple(sorted(pts))]
    else:
        quarter = type(thr)(0.25)
        centre_in = ((v[_TL] + v[_TR]) + (v[_BR] + v[_BL])) * quarter >= thr
        # cut off each outside corner when joined through the centre, else each inside corner
        cut = [c for c in (_TL, _TR, _BR, _BL) if inside[c] != centre_in]
        pairs = []
        for q in cut:
            pairs.append(tuple(e for e, (a, b) in _EDGE_CORNERS.items() if q in (a, b)))
    segs = []
    for e0, e1 in pairs:
        p0, p1 = pts[e0], pts[e1]
        (a0, b0), (a1, b1) = _EDGE_CORNERS[e0], _EDGE_CORNERS[e1]
        shared = {a0, b0} & {a1, b1}
        if shared:  # adjacent edges: the segment cuts off the shared corner
            q = shared.pop()
            want = 1.0 if inside[q] else -1.0
        else:       # opposite edges: the inside pair goes on the left
            q = next(c for c in (a0, b0) if inside[c])
            want = 1.0
        qx, qy = q[1], q[0]
        side = _cross((p1[0] - p0[0], p1[1] - p0[1]), (qx - p0[0], qy - p0[1]))
        if side * want < 0:
            p0, p1, e0, e1 = p1, p0, e1, e0
        segs.append((p0, p1, e0, e1))
    segs.sort(key=lambda s: s[2])
    return segs


def marching_squares(iblur, threshold, rows=None):
    """All contour segments of one plane: list of (cell, x0, y0, x1, y1, e0, e1)
    with cell = i N + j, coordinates in pixels (absolute, not wrapped: a cell in
    the last row or column reaches N).  `rows`: only these cell rows i (for
    large planes)."""
    img = np.asarray(iblur)
    if img.dtype not in (np.float32, np.float64):
        img = img.astype(np.float64)
    thr = img.dtype.type(threshold)
    n = img.shape[-1]
    out = []
    for i in (range(n) if rows is None else sorted(rows)):
        for j in range(n):
            v = {(dy, dx): img[(i + dy) % n, (j + dx) % n] for dy, dx in (_TL, _TR, _BR, _BL)}
            for (x0, y0), (x1, y1), e0, e1 in _cell_segments(v, thr):
                out.append((i * n + j, j + x0, i + y0, j + x1, i + y1, e0, e1))
    return out


def bilinear(field, x, y):
    """Periodic bilinear interpolation of field[row][col] at (x, y) = (col, row)."""
    n = field.shape[-1]
    j0, i0 = math.floor(x), math.floor(y)
    fx, fy = x - j0, y - i0
    a = field[i0 % n, j0 % n]
    b = field[i0 % n, (j0 + 1) % n]
    c = field[(i0 + 1) % n, j0 % n]
    d = field[(i0 + 1) % n, (j0 + 1) % n]
    return (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * c + fx * d)


def epe(iblur, points, threshold, pixel_nm):
    """Eq. (6) at control points (x, y) in pixels: -(I_b(r) - T) / |grad I_b(r)|, in nm."""
    img = np.asarray(iblur, dtype=np.float64)
    gx = (np.roll(img, -1, axis=1) - np.roll(img, 1, axis=1)) / 2.0   # d/dx per pixel
    gy = (np.roll(img, -1, axis=0) - np.roll(img, 1, axis=0)) / 2.0
    res = np.empty(len(points))
    for m, (x, y) in enumerate(points):
        e = bilinear(img, x, y)
        g = math.hypot(bilinear(gx, x, y), bilinear(gy, x, y)) / pixel_nm
        res[m] = -(e - threshold) / g if g > 0 else math.nan
    return res


def epe_through_focus(epe_planes, f0, fp, fn, tol_neg, tol_pos):
    """Eqs. (7)-(8) per control point from EPE[plane][point]: (EPE_avg, EPE_eff)."""
    e = np.asarray(epe_planes, dtype=np.float64)
    avg = (e[f0] + e[fp] + e[fn]) / 3.0
    eff = np.empty_like(avg)
    for m in range(e.shape[1]):
        e0 = e[f0, m]
        if e0 > tol_pos:
            eff[m] = e0 - tol_pos
        elif e0 < tol_neg:
            eff[m] = e0 - tol_neg
        else:
            eff[m] = avg[m]
    return avg, eff
