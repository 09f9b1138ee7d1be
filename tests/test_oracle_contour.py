"""Pins of the oracle's marching squares and edge-placement error (section II.D, Eqs. (6)-(8)).

Each pin is fixed by geometry or arithmetic, not by the oracle itself: exact
level lines of linear fields, closed contours whose segments chain end to
start, the count of crossed pixel pairs, the enclosed area of a disk, a hand-
worked saddle cell, the signed distance to a line for Eq. (6), and each
branch of Eq. (8) with hand-computed values.
"""
import math

import numpy as np
import pytest

import synth
from oracle import contour as OC


def _linear(n, a, b, c):
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    return a * x + b * y + c


def test_linear_field_segments_lie_on_the_level_line_with_inside_on_the_left():
    n, a, b, c, thr = 24, 0.031, -0.017, 0.2, 0.4517   # no pixel centre exactly on the level line
    f = _linear(n, a, b, c)
    # keep only cells away from the periodic seam, where the field is linear across the cell
    segs = [s for s in OC.marching_squares(f, thr) if (s[0] // n) < n - 1 and (s[0] % n) < n - 1]
    assert len(segs) > 10
    for _, x0, y0, x1, y1, _, _ in segs:
        assert abs(a * x0 + b * y0 + c - thr) < 1e-12 and abs(a * x1 + b * y1 + c - thr) < 1e-12
        # the gradient points to the inside (f >= T): it must be on the left of p0 -> p1
        assert (x1 - x0) * b - (y1 - y0) * a > 0


def _blobs(n, seed):
    st = synth.Stream(seed)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    f = np.zeros((n, n))
    for cx, cy, r in zip(st.uniform(6) * n, st.uniform(6) * n, 2.0 + 3.0 * st.uniform(6)):
        dx = (x - cx + n / 2) % n - n / 2
        dy = (y - cy + n / 2) % n - n / 2
        f += np.exp(-(dx * dx + dy * dy) / (2 * r * r))
    return f


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_contours_are_closed_and_each_crossed_pixel_pair_gives_one_endpoint(dtype):
    n, thr = 32, 0.5
    f = _blobs(n, 3).astype(dtype)
    segs = OC.marching_squares(f, thr)
    inside = f >= dtype(thr)
    crossed = int(np.sum(inside != np.roll(inside, -1, axis=1)) + np.sum(inside != np.roll(inside, -1, axis=0)))
    assert len(segs) == crossed          # every crossed edge is shared by two cells: one start, one end
    starts = {}
    for s in segs:
        key = (round(s[1] % n, 12), round(s[2] % n, 12))
        assert key not in starts
        starts[key] = s
    for s in segs:                       # every end point is the start of exactly one other segment
        assert (round(s[3] % n, 12), round(s[4] % n, 12)) in starts


def test_disk_area_and_radius():
    n, r0, cx, cy = 64, 12.0, 31.3, 30.6
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    f = -np.hypot(x - cx, y - cy)        # inside: distance <= r0
    segs = OC.marching_squares(f, -r0)
    area = 0.5 * sum(x0 * y1 - x1 * y0 for _, x0, y0, x1, y1, _, _ in segs)
    assert area == pytest.approx(math.pi * r0 * r0, rel=2e-3)   # inscribed polygon: area slightly below
    assert area < math.pi * r0 * r0
    for _, x0, y0, x1, y1, _, _ in segs:
        assert abs(math.hypot(x0 - cx, y0 - cy) - r0) < 0.02


def test_saddle_cell_worked_by_hand():
    # corners TL = 1, TR = 0, BR = 1, BL = 0 around a cell, T = 0.5: a saddle.
    # Centre mean 0.5 >= T: the inside corners are joined, each segment cuts off an
    # outside corner.  Crossings at the edge midpoints: top (0.5, 0), right (1, 0.5),
    # bottom (0.5, 1), left (0, 0.5).  TR (outside) is cut off by top-right and must be
    # on the right; BL (outside) by bottom-left.
    img = np.zeros((4, 4))
    img[1, 1], img[1, 2], img[2, 2], img[2, 1] = 1.0, 0.0, 1.0, 0.0
    segs = [s for s in OC.marching_squares(img, 0.5) if s[0] == 1 * 4 + 1]
    got = [(s[1] - 1, s[2] - 1, s[3] - 1, s[4] - 1) for s in segs]
    assert got == [(0.5, 0.0, 1.0, 0.5), (0.5, 1.0, 0.0, 0.5)]
    # lowering the centre below T separates the inside corners instead
    img[1, 1], img[2, 2] = 0.9, 0.9
    img[1, 2], img[2, 1] = 0.0, 0.0        # mean 0.45 < 0.5: cut off TL and BR (inside, on the left)
    segs = [s for s in OC.marching_squares(img, 0.5) if s[0] == 5]
    t = 0.4 / 0.9                         # crossing distance from the inside corner
    got = [tuple(round(v, 12) for v in (s[1] - 1, s[2] - 1, s[3] - 1, s[4] - 1)) for s in segs]
    want = [tuple(round(v, 12) for v in w) for w in
            [(t, 0.0, 0.0, t),                 # cuts off TL: from top to left, TL on the left
             (1 - t, 1.0, 1.0, 1 - t)]]        # cuts off BR: from bottom to right, BR on the left
    assert got == want


def test_epe_is_the_signed_distance_to_a_linear_level_line():
    n, a, c, thr, pixel = 32, 0.04, 0.1, 0.3, 8.0
    f = _linear(n, a, 0.0, c)
    pts = [(x, y) for x, y in zip([4.25, 5.0, 7.75, 9.5], [3.0, 10.5, 20.25, 7.0])]
    got = OC.epe(f, pts, thr, pixel)
    xstar = (thr - c) / a
    want = [-(x - xstar) * pixel for x, _ in pts]   # -(I - T)/|grad I| with I linear in x
    assert np.allclose(got, want, atol=1e-12)


def test_epe_through_focus_branches():
    e = np.array([[0.8, -0.9, 0.1, 0.5, -0.5],      # on focus
                  [1.0, -1.0, 0.4, 0.2, -0.2],      # positive defocus
                  [0.0, 0.0, -0.2, 0.5, -0.5]])     # negative defocus
    avg, eff = OC.epe_through_focus(e, 0, 1, 2, tol_neg=-0.5, tol_pos=0.5)
    assert np.allclose(avg, [0.6, -1.9 / 3, 0.1, 0.4, -0.4])
    # 0.8 > 0.5 -> 0.3; -0.9 < -0.5 -> -0.4; inside -> average; exactly at a tolerance -> average
    assert np.allclose(eff, [0.3, -0.4, 0.1, 0.4, -0.4])
