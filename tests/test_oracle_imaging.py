"""Pins for the oracle's imaging (Eqs. (1), (2), (4)).

* a brute-force direct DFT on a 16x16 grid (explicit DFT matrices, no FFT);
* the clear-field closed form (I = dose for Abbe and full-rank SOCS);
* the pixelated 1-D grating closed form (Fourier-series coefficients of a
  periodic line/space pattern, imaged order by order);
* invariants: full-rank SOCS equals Abbe, shift equivariance, mirror symmetry,
  +-defocus symmetry, monotone truncation, linearity in dose.
"""
import numpy as np
import pytest

import synth
from oracle import imaging as I
from oracle import optics as O

DUV = O.Optics(193.0, 1.35, 1.44, O.ANNULAR, 21, 0.6, 0.9)
QUAD = O.Optics(193.0, 1.35, 1.44, O.QUADRUPOLE, 41, pole_sigma=0.8, pole_radius=0.1)


def _direct_abbe(m, opt, pix, z, dose=1.0):
    """Abbe image by explicit DFT matrices, frequencies u in [-N/2, N/2)."""
    n = m.shape[0]
    u = np.arange(n) - n // 2
    j = np.arange(n)
    fwd = np.exp(-2j * np.pi * np.outer(u, j) / n)          # [u, x]
    inv = np.exp(+2j * np.pi * np.outer(j, u) / n)          # [x, u]
    mhat = fwd @ m @ fwd.T / n ** 2                          # [v, u]
    fu = u / (n * pix)
    fy, fx = np.meshgrid(fu, fu, indexing="ij")
    sx, sy, w = O.source_points(opt)
    fna = opt.na / opt.wavelength_nm
    out = np.zeros((n, n))
    for s in range(len(w)):
        p = O.pupil(fx + sx[s] * fna, fy + sy[s] * fna, opt, z)
        e = inv @ (mhat * p) @ inv.T
        out += w[s] * np.abs(e) ** 2
    return dose * out


@pytest.mark.parametrize("z", [0.0, -40.0])
def test_abbe_matches_direct_dft_16x16(z):
    m = synth.random_rect_mask(16, seed=5, count=4, side_lo=2, side_hi=5).astype(np.float64)
    pix = 30.0
    a = I.abbe_image(m, DUV, pix, z, dose=1.3)
    b = _direct_abbe(m, DUV, pix, z, dose=1.3)
    assert np.abs(a - b).max() < 1e-12


def test_socs_full_rank_matches_direct_dft_16x16():
    m = synth.random_rect_mask(16, seed=7, count=4, side_lo=2, side_hi=5).astype(np.float64)
    pix = 30.0
    ns = len(O.source_points(DUV)[0])
    lam, phi, _ = O.socs_kernels(DUV, 16, pix, 25.0, ns)
    assert np.abs(I.socs_image(m, lam, phi) - _direct_abbe(m, DUV, pix, 25.0)).max() < 1e-12


@pytest.mark.parametrize("opt", [DUV, QUAD])
def test_clear_field(opt):
    n, pix = 64, 8.0
    m = np.ones((n, n))
    a = I.abbe_image(m, opt, pix, 30.0, dose=0.7)
    assert np.abs(a - 0.7).max() < 1e-12
    c = O.crop_size(opt, n, pix)
    ns = len(O.source_points(opt)[0])
    lam, phi, _ = O.socs_kernels(opt, n, pix, 30.0, ns, c)
    assert np.abs(I.socs_image(m, lam, phi, dose=0.7) - 0.7).max() < 1e-12
    # truncated: I = sum_k lam_k |Phi_k(0)|^2 <= 1
    k = 5
    it = I.socs_image(m, lam[:k], phi[:k])
    ref = sum(lam[i] * abs(phi[i, c // 2, c // 2]) ** 2 for i in range(k))
    assert np.abs(it - ref).max() < 1e-12
    assert ref <= 1.0 + 1e-12


def _grating_closed_form(n, period, width, opt, pix, z, dose=1.0):
    """I(x) for m(x) = [x mod P < w] from its Fourier-series coefficients
    c_n = exp(-i pi n (w-1)/P) sin(pi n w/P) / (P sin(pi n/P)), c_0 = w/P."""
    sx, sy, w = O.source_points(opt)
    fna = opt.na / opt.wavelength_nm
    orders = np.arange(-(period // 2), period - period // 2)
    cn = np.empty(len(orders), dtype=np.complex128)
    for i, o in enumerate(orders):
        if o == 0:
            cn[i] = width / period
        else:
            cn[i] = (np.exp(-1j * np.pi * o * (width - 1) / period) * np.sin(np.pi * o * width / period)
                     / (period * np.sin(np.pi * o / period)))
    x = np.arange(n)
    out = np.zeros(n)
    for s in range(len(w)):
        p = O.pupil(orders / (period * pix) + sx[s] * fna, 0 * orders + sy[s] * fna, opt, z)
        e = (cn * p) @ np.exp(2j * np.pi * np.outer(orders, x) / period)
        out += w[s] * np.abs(e) ** 2
    return dose * out


@pytest.mark.parametrize("z", [0.0, 50.0])
@pytest.mark.parametrize("period,width", [(16, 8), (12, 5)])
def test_grating_closed_form(z, period, width):
    n, pix = 192 if period == 12 else 256, 8.0
    m = np.zeros((n, n))
    m[:, (np.arange(n) % period) < width] = 1.0
    a = I.abbe_image(m, DUV, pix, z)
    ref = _grating_closed_form(n, period, width, DUV, pix, z)
    assert np.abs(a - ref[None, :]).max() < 1e-12
    # the pattern is genuinely imaged: not a flat field
    assert ref.max() - ref.min() > 0.05


def test_full_rank_socs_equals_abbe_and_truncation_is_monotone():
    n, pix = 64, 8.0
    m = synth.random_rect_mask(n, seed=11, count=12).astype(np.float64)
    c = O.crop_size(QUAD, n, pix)
    lam, phi, _ = O.socs_kernels(QUAD, n, pix, -35.0, 52, c)
    abbe = I.abbe_image(m, QUAD, pix, -35.0)
    full = I.socs_image(m, lam, phi)
    assert np.abs(full - abbe).max() < 1e-10
    prev = np.zeros_like(abbe)
    for k in (1, 4, 8, 20, 52):
        cur = I.socs_image(m, lam[:k], phi[:k])
        assert np.all(cur >= prev - 1e-13)
        assert np.all(cur <= abbe + 1e-12)
        prev = cur


def test_shift_equivariance_mirror_and_defocus_symmetry():
    n, pix = 64, 8.0
    m = synth.random_rect_mask(n, seed=3, count=10).astype(np.float64)
    base = I.abbe_image(m, DUV, pix, 40.0)
    shifted = I.abbe_image(np.roll(m, (5, -9), axis=(0, 1)), DUV, pix, 40.0)
    assert np.abs(shifted - np.roll(base, (5, -9), axis=(0, 1))).max() < 1e-12
    # mirror x -> -x of mask and (symmetric) source mirrors the image
    mir = m[:, (-np.arange(n)) % n]
    im = I.abbe_image(mir, DUV, pix, 40.0)
    assert np.abs(im - base[:, (-np.arange(n)) % n]).max() < 1e-12
    # real mask, point-symmetric source, no aberrations: I(z) = I(-z)
    assert np.abs(I.abbe_image(m, QUAD, pix, 60.0) - I.abbe_image(m, QUAD, pix, -60.0)).max() < 1e-12
    # and defocus does change the image
    assert np.abs(I.abbe_image(m, QUAD, pix, 60.0) - I.abbe_image(m, QUAD, pix, 0.0)).max() > 1e-3
    # linear in dose
    assert np.abs(I.abbe_image(m, DUV, pix, 40.0, dose=2.5) - 2.5 * base).max() < 1e-12


def test_socs_rows_matches_full_image():
    n, pix = 128, 8.0
    m = synth.random_rect_mask(n, seed=21, count=30).astype(np.float64)
    c = O.crop_size(QUAD, n, pix)
    lam, phi, _ = O.socs_kernels(QUAD, n, pix, 50.0, 8, c)
    full = I.socs_image(m, lam, phi, dose=1.1)
    rows = [0, 17, 64, 127]
    mb = I.band(I.mask_spectrum(m), c)
    assert np.abs(I.socs_rows(mb, lam, phi, n, rows, dose=1.1) - full[rows]).max() < 1e-12
