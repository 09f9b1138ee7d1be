"""Oracle resist: periodic Gaussian blur, threshold, contour crossings (FP64).

Test infrastructure only (see the package docstring).

Eq. (5): the wafer contour is the level set {r : (I (x) K_resist)(r) = T_eff}.
K_resist is read as a normalised, truncated Gaussian
    g[j] = exp(-(j pixel)^2 / (2 sigma^2)) for |j| <= R = ceil(4 sigma / pixel),  sum g = 1,
applied separably with periodic boundaries (matching the periodic imaging).
A pixel prints when I_blur >= T (ties count as printed, following the ">=" of
Eqs. (16)-(17)).
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_taps(sigma_nm: float, pixel_nm: float):
    r = int(math.ceil(4.0 * sigma_nm / pixel_nm))
    j = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-((j * pixel_nm) ** 2) / (2.0 * sigma_nm * sigma_nm))
    return g / g.sum()


def blur(img, sigma_nm: float, pixel_nm: float):
    """(g (x) I)(y, x) = sum_{a,b} g[a] g[b] I(y - a, x - b), periodic."""
    g = gaussian_taps(sigma_nm, pixel_nm)
    r = (len(g) - 1) // 2
    img = np.asarray(img, dtype=np.float64)
    tmp = np.zeros_like(img)
    for a in range(-r, r + 1):
        tmp += g[a + r] * np.roll(img, a, axis=-1)
    out = np.zeros_like(img)
    for a in range(-r, r + 1):
        out += g[a + r] * np.roll(tmp, a, axis=-2)
    return out


def printed(iblur, threshold: float):
    return (iblur >= threshold).astype(np.uint8)


def crossings(iblur, threshold: float, axis: int):
    """Threshold crossings along `axis` between neighbours j and j+1 (periodic).

    Returns (line, j, t): the crossing sits at j + t, t in [0, 1), found by
    linear interpolation of d = I_blur - T between the two pixels.  `line` is
    the index of the row (axis=1) or column (axis=0).
    """
    d = np.asarray(iblur, dtype=np.float64) - threshold
    if axis == 0:
        d = d.T
    a = d
    b = np.roll(d, -1, axis=1)
    hit = (a >= 0) != (b >= 0)
    line, j = np.nonzero(hit)
    av = a[line, j]
    bv = b[line, j]
    t = av / (av - bv)
    return line, j, t


def edge_placement_difference(iblur_ref, iblur_test, threshold: float, pixel_nm: float, window: int = 2):
    """Largest contour displacement (nm) of `iblur_test` relative to `iblur_ref`.

    For every crossing of the reference along rows and columns, the nearest
    crossing of the test image on the same line within +-window pixels is
    taken; the metric is max |x_test - x_ref| * pixel.  A reference crossing
    with no partner gives +inf.  Used as the edge-placement check between two
    resist images (Eq. (6) measures against a target instead).
    """
    worst = 0.0
    n = iblur_ref.shape[-1]
    for axis in (1, 0):
        lr, jr, tr = crossings(iblur_ref, threshold, axis)
        lt, jt, tt = crossings(iblur_test, threshold, axis)
        pos_t = {}
        for l_, j_, t_ in zip(lt, jt, tt):
            pos_t.setdefault(int(l_), []).append(j_ + t_)
        for l_, j_, t_ in zip(lr, jr, tr):
            xr = j_ + t_
            cand = pos_t.get(int(l_), [])
            best = np.inf
            for xt in cand:
                dd = abs(xt - xr)
                dd = min(dd, n - dd)
                if dd <= window:
                    best = min(best, dd)
            worst = max(worst, best * pixel_nm)
    return worst
