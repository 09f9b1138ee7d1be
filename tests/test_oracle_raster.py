"""Pins of the oracle's area-coverage rasteriser.

Fixed independently of it: (1) rectangles on a quarter-pixel lattice are
covered exactly by centre sampling on a 4x finer grid, so coverage equals the
count of covered sub-pixels / 16; (2) integer rectangles give the centre-
sampled binary mask of `synth.rasterize_rects`; (3) the total of two
overlapping rectangles is the union area by inclusion-exclusion; (4) a
rectangle across the period equals its two pieces.
"""
import numpy as np
import pytest

import synth
from oracle import raster as ORA


def _quarter_rects(n, count, seed):
    st = synth.Stream(seed)
    w = st.integers(4, 40, count) / 4.0
    h = st.integers(4, 40, count) / 4.0
    x0 = st.integers(0, 4 * n - 1, count) / 4.0
    y0 = st.integers(0, 4 * n - 1, count) / 4.0
    return np.stack([x0, y0, x0 + w, y0 + h], axis=1)


def test_quarter_lattice_rectangles_match_fine_centre_sampling():
    n, s = 32, 4
    rects = _quarter_rects(n, 25, seed=3)
    fine = np.zeros((n * s, n * s))
    c = (np.arange(n * s) + 0.5) / s              # sub-pixel centres in pixel units
    for x0, y0, x1, y1 in rects:
        for dx in (0, n):                         # the period: test the centres against both copies
            for dy in (0, n):
                inx = (c + dx >= x0) & (c + dx < x1)
                iny = (c + dy >= y0) & (c + dy < y1)
                fine[np.ix_(iny, inx)] = 1.0
    want = fine.reshape(n, s, n, s).sum(axis=(1, 3)) / (s * s)
    got = ORA.coverage(n, rects)
    assert np.abs(got - want).max() < 1e-12
    assert 0.0 < got.mean() < 1.0 and ((got > 0) & (got < 1)).any()


def test_integer_rectangles_give_the_centre_sampled_mask():
    n = 48
    st = synth.Stream(11)
    rects = []
    for _ in range(30):
        w, h = st.integers(2, 9, 2)
        x0, y0 = st.integers(0, n - 1, 2)
        rects.append((int(x0), int(y0), int(w), int(h)))
    want = synth.rasterize_rects(n, np.array(rects))
    got = ORA.coverage(n, [(x, y, x + w, y + h) for x, y, w, h in rects])
    assert np.array_equal(got, want.astype(np.float64))


def test_overlap_counts_once_and_wrap_splits():
    n = 16
    a = (2.25, 3.5, 7.75, 9.0)
    b = (5.5, 1.0, 11.0, 6.25)
    inter = (7.75 - 5.5) * (6.25 - 3.5)
    union = (7.75 - 2.25) * (9.0 - 3.5) + (11.0 - 5.5) * (6.25 - 1.0) - inter
    assert ORA.coverage(n, [a, b]).sum() == pytest.approx(union, abs=1e-12)
    w = (13.5, 14.25, 18.75, 17.5)                # runs past the period in x and y
    parts = [(13.5, 14.25, 16.0, 16.0), (0.0, 14.25, 2.75, 16.0), (13.5, 0.0, 16.0, 1.5), (0.0, 0.0, 2.75, 1.5)]
    assert np.abs(ORA.coverage(n, [w]) - ORA.coverage(n, parts)).max() < 1e-12
    assert ORA.coverage(n, [w]).sum() == pytest.approx(5.25 * 3.25, abs=1e-12)
