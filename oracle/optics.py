"""Oracle optics: source, pupil, band crop and SOCS kernels (FP64).

Test infrastructure only (see the package docstring).

Conventions (paper Section III.A, Eqs. (1)-(3)):
* N x N periodic grid, pixel `pixel_nm`; frequency bin u in [-N/2, N/2) has
  f_u = u / (N * pixel_nm).  Arrays indexed [v][u] are (y-frequency, x-frequency).
* Source points sigma_s in units of the pupil cut-off f_NA = NA / wavelength,
  equal weights w_s with sum 1 (Eq. (2): S is a normalised distribution).
* Pupil P(f; z) = 1[|f| <= f_NA] * exp(i 2 pi z (sqrt((n/lambda)^2 - |f|^2) - n/lambda)),
  a scalar aberration-free pupil with defocus z (nm) in a medium of index n.
  The paper only says the pupil includes the NA cut-off and aberrations; the
  defocus model is our reading.
* TCC(f1, f2) = sum_s w_s P(f1 + sigma_s f_NA) P*(f2 + sigma_s f_NA)  (Eq. (2)).
  With A[u, s] = sqrt(w_s) P(f_u + sigma_s f_NA) this is A A^H, so its nonzero
  eigenpairs are those of the small Gram matrix G = A^H A: G v = lam v gives the
  unit eigenvector Phi = A v / sqrt(lam) of A A^H with the same lam (Eq. (3)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ANNULAR = "annular"
QUADRUPOLE = "quadrupole"


@dataclass(frozen=True)
class Optics:
    wavelength_nm: float = 193.0
    na: float = 1.35
    n_medium: float = 1.44
    kind: str = ANNULAR
    src_grid: int = 21
    sigma_in: float = 0.6
    sigma_out: float = 0.9
    pole_sigma: float = 0.8
    pole_radius: float = 0.1


def source_points(opt: Optics):
    """Source sample points (sx, sy) in units of f_NA and weights w (sum 1).

    Grid points sigma = (i/h, j/h), i, j in [-h, h], h = (src_grid - 1)/2.
    Annular: sigma_in <= |sigma| <= sigma_out (both inclusive).
    Quadrupole: four discs of radius pole_radius centred on the x and y axes at
    distance pole_sigma (inclusive).  The membership tests are done in grid
    units with a relative slack of 1e-12 so that boundary points count.
    """
    h = (opt.src_grid - 1) // 2
    xs, ys = [], []
    for j in range(-h, h + 1):
        for i in range(-h, h + 1):
            r2 = float(i * i + j * j)
            if opt.kind == ANNULAR:
                lo = (opt.sigma_in * h) ** 2
                hi = (opt.sigma_out * h) ** 2
                keep = (r2 >= lo * (1 - 1e-12)) and (r2 <= hi * (1 + 1e-12))
            elif opt.kind == QUADRUPOLE:
                c = opt.pole_sigma * h
                rr = (opt.pole_radius * h) ** 2 * (1 + 1e-12)
                keep = any((i - cx) ** 2 + (j - cy) ** 2 <= rr
                           for cx, cy in ((c, 0.0), (-c, 0.0), (0.0, c), (0.0, -c)))
            else:
                raise ValueError(opt.kind)
            if keep:
                xs.append(i / h)
                ys.append(j / h)
    sx = np.array(xs, dtype=np.float64)
    sy = np.array(ys, dtype=np.float64)
    w = np.full(sx.shape, 1.0 / len(sx))
    return sx, sy, w


def pupil(fx, fy, opt: Optics, z_nm: float):
    """Scalar pupil with NA cut-off (inclusive) and defocus phase, Eq. (2)'s P."""
    f2 = fx * fx + fy * fy
    fna = opt.na / opt.wavelength_nm
    kn = opt.n_medium / opt.wavelength_nm
    inside = f2 <= fna * fna
    kz = np.sqrt(np.maximum(kn * kn - f2, 0.0)) - kn
    return np.where(inside, np.exp(1j * 2.0 * np.pi * z_nm * kz), 0.0)


def band_radius_bins(opt: Optics, n: int, pixel_nm: float) -> int:
    """Largest |u| that can carry light: floor((1 + sigma_max) f_NA N pixel)."""
    sx, sy, _ = source_points(opt)
    smax = float(np.sqrt(sx * sx + sy * sy).max())
    fb = (1.0 + smax) * opt.na / opt.wavelength_nm
    return int(math.floor(fb * n * pixel_nm))


def crop_size(opt: Optics, n: int, pixel_nm: float) -> int:
    """Side C of the centred band crop u in [-C/2, C/2): the smallest multiple of
    32 with C/2 > band radius, capped at N."""
    rb = band_radius_bins(opt, n, pixel_nm)
    c = 2 * rb + 2
    c = ((c + 31) // 32) * 32
    return min(c, n)


def crop_freqs(n: int, c: int):
    """Integer frequencies of the crop, index i <-> u = i - C/2."""
    return np.arange(c) - c // 2


def a_matrix(opt: Optics, n: int, pixel_nm: float, z_nm: float, c: int):
    """A[(v,u), s] = sqrt(w_s) P(f_(u,v) + sigma_s f_NA; z) over the C x C crop."""
    sx, sy, w = source_points(opt)
    fna = opt.na / opt.wavelength_nm
    u = crop_freqs(n, c) / (n * pixel_nm)
    fy, fx = np.meshgrid(u, u, indexing="ij")
    fx = fx.reshape(-1, 1) + sx[None, :] * fna
    fy = fy.reshape(-1, 1) + sy[None, :] * fna
    return pupil(fx, fy, opt, z_nm) * np.sqrt(w)[None, :]


def tcc_trace(opt: Optics, n: int, pixel_nm: float, c: int) -> float:
    """trace(TCC) = sum_s w_s #{u in crop : |f_u + sigma_s f_NA| <= f_NA} (any focus)."""
    sx, sy, w = source_points(opt)
    fna = opt.na / opt.wavelength_nm
    u = crop_freqs(n, c) / (n * pixel_nm)
    fy, fx = np.meshgrid(u, u, indexing="ij")
    tot = 0.0
    for s in range(len(w)):
        gx = fx + sx[s] * fna
        gy = fy + sy[s] * fna
        tot += w[s] * np.count_nonzero(gx * gx + gy * gy <= fna * fna)
    return tot


def socs_kernels(opt: Optics, n: int, pixel_nm: float, z_nm: float, k: int, c: int | None = None,
                 rel_tol: float = 1e-12):
    """Top-k TCC eigenpairs (Eq. (3)) on the C x C crop.

    Returns (lam[k], phi[k, C, C]) with lam descending.  Modes whose eigenvalue
    is at most rel_tol * lam_1 (beyond the rank of the TCC) are returned as
    lam = 0 and phi = 0.
    """
    if c is None:
        c = crop_size(opt, n, pixel_nm)
    a = a_matrix(opt, n, pixel_nm, z_nm, c)
    g = a.conj().T @ a
    lam_all, v = np.linalg.eigh(g)
    order = np.argsort(lam_all)[::-1]
    lam_all = lam_all[order]
    v = v[:, order]
    lam = np.zeros(k)
    phi = np.zeros((k, c * c), dtype=np.complex128)
    top = lam_all[0]
    for i in range(min(k, len(lam_all))):
        if lam_all[i] > rel_tol * top:
            lam[i] = lam_all[i]
            phi[i] = (a @ v[:, i]) / np.sqrt(lam_all[i])
    return lam, phi.reshape(k, c, c), lam_all


def tcc_matrix(opt: Optics, n: int, pixel_nm: float, z_nm: float, c: int):
    """Dense TCC over the crop straight from Eq. (2) (small crops only)."""
    sx, sy, w = source_points(opt)
    fna = opt.na / opt.wavelength_nm
    u = crop_freqs(n, c) / (n * pixel_nm)
    fy, fx = np.meshgrid(u, u, indexing="ij")
    fx = fx.reshape(-1)
    fy = fy.reshape(-1)
    t = np.zeros((c * c, c * c), dtype=np.complex128)
    for s in range(len(w)):
        p = pupil(fx + sx[s] * fna, fy + sy[s] * fna, opt, z_nm)
        t += w[s] * np.outer(p, p.conj())
    return t
