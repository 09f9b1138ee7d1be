"""GPU area-coverage rasterisation against the oracle (coordinate compression, FP64).

The kernel computes each pixel's union area in FP32 from FP32 corners; the
bound is 2e-6 per pixel (a few FP32 roundings of areas of at most 1).
Quarter-pixel rectangles, random off-grid rectangles with heavy overlap and
wrap-around, integer rectangles (exact binary mask), empty clips, and a
rectangle too large for max_side (its clip becomes NaN).
"""
import numpy as np
import pytest

import synth
from oracle import raster as ORA

pytestmark = pytest.mark.gpu


def _rects(n, count, seed, lo=1.0, hi=15.0, quarter=False):
    st = synth.Stream(seed)
    if quarter:
        w = st.integers(int(4 * lo), int(4 * hi), count) / 4.0
        h = st.integers(int(4 * lo), int(4 * hi), count) / 4.0
        x0 = st.integers(0, 4 * n - 1, count) / 4.0
        y0 = st.integers(0, 4 * n - 1, count) / 4.0
    else:
        w = lo + (hi - lo) * st.uniform(count)
        h = lo + (hi - lo) * st.uniform(count)
        x0 = n * st.uniform(count)
        y0 = n * st.uniform(count)
    return np.stack([x0, y0, x0 + w, y0 + h], axis=1).astype(np.float32)


def test_rasterize_matches_oracle(litho_lib, cuda):
    L = litho_lib
    n = 96
    clips = [_rects(n, 60, 1, quarter=True), _rects(n, 150, 2), _rects(n, 0, 3),
             _rects(n, 400, 4, lo=0.3, hi=6.0)]          # dense, overlapping, sub-pixel sides
    got = L.litho_rasterize(clips, n, 16).cpu().numpy()
    for c, r in enumerate(clips):
        want = ORA.coverage(n, r.astype(np.float64))
        err = np.abs(got[c] - want).max()
        print(f"clip {c}: {len(r)} rects, max err {err:.2e}, mean cover {want.mean():.3f}")
        assert err <= 2e-6, (c, err)
    assert not got[2].any()


def test_rasterize_integer_rects_is_binary_and_large_rect_marks_clip(litho_lib, cuda):
    L = litho_lib
    n = 64
    st = synth.Stream(8)
    ints = []
    for _ in range(40):
        w, h = st.integers(2, 12, 2)
        x0, y0 = st.integers(0, n - 1, 2)
        ints.append((int(x0), int(y0), int(w), int(h)))
    rects = np.array([(x, y, x + w, y + h) for x, y, w, h in ints], dtype=np.float32)
    too_big = np.array([[1.0, 1.0, 30.0, 3.0]], dtype=np.float32)
    got = L.litho_rasterize([rects, too_big], n, 16).cpu().numpy()
    assert np.array_equal(got[0], synth.rasterize_rects(n, np.array(ints)))
    assert np.isnan(got[1]).all()


def test_rasterize_full_size_manhattan(litho_lib, cuda):
    """2048^2 clip with the Manhattan generator's rectangles shifted by quarter pixels
    (grey edges everywhere): sampled rows against the oracle on a window."""
    L = litho_lib
    n = 2048
    st = synth.Stream(99)
    k = 6000
    w = st.integers(20, 60, k) / 4.0
    h = st.integers(20, 60, k) / 4.0
    x0 = st.integers(0, 4 * n - 1, k) / 4.0
    y0 = st.integers(0, 4 * n - 1, k) / 4.0
    rects = np.stack([x0, y0, x0 + w, y0 + h], axis=1).astype(np.float32)
    got = L.litho_rasterize([rects], n, 16).cpu().numpy()[0]
    # the oracle on a 128 x 128 window: the rectangles clipped to it (those crossing the
    # window edge are cut there, which leaves the window's pixels unchanged)
    lo, size = 960, 128
    sel = []
    for x0_, y0_, x1_, y1_ in rects.astype(np.float64):
        for sx in (0.0, -n):
            for sy in (0.0, -n):
                a, b_, c, d = max(x0_ + sx, lo), max(y0_ + sy, lo), min(x1_ + sx, lo + size), min(y1_ + sy, lo + size)
                if c > a and d > b_:
                    sel.append((a - lo, b_ - lo, c - lo, d - lo))
    want = ORA.coverage(size, np.array(sel))
    assert np.abs(got[lo:lo + size, lo:lo + size] - want).max() <= 2e-6
