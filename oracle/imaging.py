"""Oracle imaging: mask spectrum, Abbe image, SOCS image (FP64).

Test infrastructure only (see the package docstring).

* Mask spectrum  M(u) = N^-2 sum_x m(x) exp(-2 pi i u.x / N), so that a clear
  mask has M(0) = 1 ("normalised to clear field").  Eq. (1)'s object spectrum
  O(f) is read as this thin-mask spectrum.
* Abbe image     I(x) = D sum_s w_s |sum_u M(u) P(f_u + sigma_s f_NA; z) e^{+2 pi i u.x/N}|^2,
  Eq. (1) with the TCC of Eq. (2) substituted and the missing `i` of Eq. (1)'s
  exponent restored.  Sums over u run over all N^2 bins (the pupil limits them).
* SOCS image     I(x) = D sum_k lam_k |sum_u M(u) Phi_k(u) e^{+2 pi i u.x/N}|^2, Eq. (4)
  with the convolution O (x) Phi_k read as a product in frequency.
The FFTs are numpy's (a library step): np.fft.ifft2 carries 1/N^2, which is
undone where an unnormalised sum is meant.
"""
from __future__ import annotations

import numpy as np

from .optics import Optics, pupil, source_points


def mask_spectrum(m):
    """M = DFT(m) / N^2 on the full grid, FFT index order."""
    n = m.shape[-1]
    return np.fft.fft2(np.asarray(m, dtype=np.float64)) / (n * n)


def crop_index(n: int, c: int):
    """Grid indices (FFT order) of the centred crop u in [-C/2, C/2)."""
    return (np.arange(c) - c // 2) % n


def band(mfull, c: int):
    """C x C centred crop [v][u] of a full-grid spectrum."""
    idx = crop_index(mfull.shape[-1], c)
    return mfull[np.ix_(idx, idx)]


def embed(spec_crop, n: int):
    """Places a C x C crop into a zero N x N spectrum."""
    c = spec_crop.shape[-1]
    idx = crop_index(n, c)
    s = np.zeros((n, n), dtype=np.complex128)
    s[np.ix_(idx, idx)] = spec_crop
    return s


def inverse_unnormalised(spec_full):
    """sum_u S(u) e^{+2 pi i u.x/N} on the full grid."""
    n = spec_full.shape[-1]
    return np.fft.ifft2(spec_full) * (n * n)


def abbe_image(m, opt: Optics, pixel_nm: float, z_nm: float, dose: float = 1.0):
    """Abbe aerial image: a sum over source points of coherent images."""
    n = m.shape[-1]
    mf = mask_spectrum(m)
    f = np.fft.fftfreq(n, d=pixel_nm)
    fy, fx = np.meshgrid(f, f, indexing="ij")
    sx, sy, w = source_points(opt)
    fna = opt.na / opt.wavelength_nm
    img = np.zeros((n, n))
    for s in range(len(w)):
        p = pupil(fx + sx[s] * fna, fy + sy[s] * fna, opt, z_nm)
        e = inverse_unnormalised(mf * p)
        img += w[s] * (e.real ** 2 + e.imag ** 2)
    return dose * img


def socs_fields(m, phi):
    """Coherent fields E_k(x) for kernels phi[k, C, C] (full grid, complex)."""
    n = m.shape[-1]
    c = phi.shape[-1]
    mb = band(mask_spectrum(m), c)
    return np.stack([inverse_unnormalised(embed(mb * phi[k], n)) for k in range(phi.shape[0])])


def socs_image(m, lam, phi, dose: float = 1.0):
    """SOCS aerial image of Eq. (4) from given kernels (lam[k], phi[k, C, C])."""
    n = m.shape[-1]
    c = phi.shape[-1]
    mb = band(mask_spectrum(m), c)
    img = np.zeros((n, n))
    for k in range(len(lam)):
        if lam[k] == 0.0:
            continue
        e = inverse_unnormalised(embed(mb * phi[k], n))
        img += lam[k] * (e.real ** 2 + e.imag ** 2)
    return dose * img


def socs_rows(mband, lam, phi, n: int, rows, dose: float = 1.0):
    """SOCS image on selected full rows y, from a precomputed band spectrum.

    E_k(y, x) = sum_u [sum_v M(v,u) Phi_k(v,u) e^{2 pi i v y/N}] e^{2 pi i u x/N}:
    the v-sum is done directly for each requested row, the u-sum by a 1-D
    inverse FFT.  Used to check large clips on a sample of rows.
    """
    c = phi.shape[-1]
    v = np.arange(c) - c // 2
    idx = crop_index(n, c)
    rows = np.asarray(rows)
    out = np.zeros((len(rows), n))
    ey = np.exp(2j * np.pi * np.outer(rows, v) / n)          # [rows, C]
    for k in range(len(lam)):
        if lam[k] == 0.0:
            continue
        t = ey @ (mband * phi[k])                               # [rows, C] over u
        s = np.zeros((len(rows), n), dtype=np.complex128)
        s[:, idx] = t
        e = np.fft.ifft(s, axis=1) * n
        out += lam[k] * (e.real ** 2 + e.imag ** 2)
    return dose * out
