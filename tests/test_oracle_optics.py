"""Pins for the oracle's source sampling, band crop and TCC eigen-kernels.

The paper prints no numerical example, so these pin Eqs. (2)-(3) by lattice
counts, the dense TCC written straight from Eq. (2), trace and PSD properties.
"""
import numpy as np
import pytest

from oracle import optics as O

DUV_ANNULAR = O.Optics(193.0, 1.35, 1.44, O.ANNULAR, 21, 0.6, 0.9)
DUV_QUAD21 = O.Optics(193.0, 1.35, 1.44, O.QUADRUPOLE, 21, pole_sigma=0.8, pole_radius=0.1)
DUV_QUAD41 = O.Optics(193.0, 1.35, 1.44, O.QUADRUPOLE, 41, pole_sigma=0.8, pole_radius=0.1)


def _count_lattice(grid, test):
    h = (grid - 1) // 2
    return sum(1 for i in range(-h, h + 1) for j in range(-h, h + 1) if test(i, j))


def test_source_counts_match_lattice_geometry():
    # annulus 6 <= r <= 9 (grid units) on the 21x21 lattice; quadrupole discs
    assert len(O.source_points(DUV_ANNULAR)[0]) == _count_lattice(21, lambda i, j: 36 <= i * i + j * j <= 81) == 144
    assert len(O.source_points(DUV_QUAD21)[0]) == 20
    assert len(O.source_points(DUV_QUAD41)[0]) == 52
    sx, sy, w = O.source_points(DUV_QUAD41)
    assert abs(w.sum() - 1.0) < 1e-15
    # poles sit on the axes at 0.8 with radius 0.1
    r = np.hypot(sx, sy)
    assert np.all(np.abs(r - 0.8) <= 0.1 + 1e-12)
    assert np.all(np.minimum(np.abs(sx), np.abs(sy)) <= 0.1 + 1e-12)


def test_crop_sizes_of_the_workloads():
    assert O.crop_size(DUV_ANNULAR, 256, 8.0) == 64
    assert O.crop_size(DUV_QUAD41, 2048, 8.0) == 448
    assert O.crop_size(DUV_ANNULAR, 1024, 8.0) == 224
    euv = O.Optics(13.5, 0.33, 1.0, O.ANNULAR, 21, 0.6, 0.9)
    assert O.crop_size(euv, 256, 1.0) == 32
    assert O.crop_size(euv, 2048, 1.0) == 192


def test_pupil_cutoff_and_defocus_phase():
    opt = DUV_ANNULAR
    fna = opt.na / opt.wavelength_nm
    f = np.array([0.0, 0.5 * fna, fna * (1 - 1e-12), fna * (1 + 1e-9)])
    p0 = O.pupil(f, 0 * f, opt, 0.0)
    assert np.allclose(p0, [1, 1, 1, 0])
    # defocus: unit modulus inside, phase 2 pi z (kz - n/lambda) with kz = sqrt((n/l)^2 - f^2)
    z = 37.0
    p = O.pupil(f[:2], 0 * f[:2], opt, z)
    kn = opt.n_medium / opt.wavelength_nm
    ref_phase = 2 * np.pi * z * (np.sqrt(kn ** 2 - (0.5 * fna) ** 2) - kn)
    assert abs(p[0] - 1) < 1e-15
    assert abs(np.angle(p[1]) - ref_phase) < 1e-12


@pytest.mark.parametrize("z", [0.0, 45.0])
def test_tcc_eigen_reconstructs_dense_tcc(z):
    opt = DUV_ANNULAR
    n, pix = 16, 30.0
    c = O.crop_size(opt, n, pix)
    t = O.tcc_matrix(opt, n, pix, z, c)
    # Hermitian PSD (paper: TCC is Hermitian and positive semi-definite)
    assert np.allclose(t, t.conj().T, atol=1e-14)
    ev = np.linalg.eigvalsh(t)
    assert ev.min() > -1e-12
    ns = len(O.source_points(opt)[0])
    lam, phi, lam_all = O.socs_kernels(opt, n, pix, z, ns, c)
    p = phi.reshape(ns, -1)
    recon = (p.T * lam) @ p.conj()
    assert np.abs(recon - t).max() < 1e-12
    # eigenvalues agree with the dense matrix's
    top = np.sort(ev)[::-1][:ns]
    assert np.allclose(np.sort(lam)[::-1], np.where(top > 1e-12 * top[0], top, 0), atol=1e-12)


def test_trace_equals_counted_pupil_overlaps_and_kernels_orthonormal():
    opt = DUV_QUAD41
    n, pix = 128, 8.0
    c = O.crop_size(opt, n, pix)
    lam, phi, lam_all = O.socs_kernels(opt, n, pix, 0.0, 52, c)
    tr = O.tcc_trace(opt, n, pix, c)
    assert abs(lam_all.sum() - tr) < 1e-9 * tr
    assert np.all(lam >= 0)
    assert np.all(np.diff(lam) <= 1e-12)
    p = phi.reshape(52, -1)
    r = int((lam > 0).sum())
    gram = p[:r].conj() @ p[:r].T
    # the weakest modes carry rounding of order eps * lam_1 / lam_k
    assert np.abs(gram - np.eye(r)).max() < 1e-10


# ---- the defocus phase, pinned by Talbot self-imaging ------------------------------------------------
#
# A grating of period p lit by one on-axis plane wave, with only its orders 0 and +-1
# passing the pupil, images itself again after a propagation distance z_T at which the
# first orders have fallen one full cycle behind the zeroth: in a medium of index n the
# axial wavenumbers are n/lambda (order 0) and sqrt((n/lambda)^2 - 1/p^2) (orders +-1),
# so z_T = 1 / (n/lambda - sqrt((n/lambda)^2 - 1/p^2)) (the non-paraxial Talbot length).
# Half-way, the first orders are in antiphase, which is the image shifted by p/2.  These
# are properties of wave propagation, not of any one way of writing the pupil: a
# paraxial defocus, a wrong medium index or a missing factor moves z_T and fails them.

ON_AXIS = O.Optics(193.0, 1.35, 1.44, O.ANNULAR, 21, 0.0, 0.0)   # sigma_in = sigma_out = 0: one point


def _talbot_length(opt, period_nm):
    kn = opt.n_medium / opt.wavelength_nm
    return 1.0 / (kn - np.sqrt(kn * kn - 1.0 / period_nm ** 2))


def _line_grating(n, period, width):
    m = np.zeros((n, n))
    m[:, (np.arange(n) % period) < width] = 1.0
    return m


@pytest.mark.parametrize("n,period,width", [(208, 26, 10), (256, 32, 11)])
def test_defocus_phase_reproduces_the_talbot_self_image(n, period, width):
    from oracle import imaging as I
    pix = 8.0
    opt = ON_AXIS
    sx, sy, _ = O.source_points(opt)
    assert len(sx) == 1 and sx[0] == 0.0 and sy[0] == 0.0
    fna = opt.na / opt.wavelength_nm
    # orders +-1 pass the pupil, +-2 do not
    assert 1.0 / (period * pix) < fna < 2.0 / (period * pix)
    m = _line_grating(n, period, width)
    zt = _talbot_length(opt, period * pix)
    i0 = I.abbe_image(m, opt, pix, 0.0)
    assert i0.max() - i0.min() > 0.1                               # a real pattern, not a flat field
    i_t = I.abbe_image(m, opt, pix, zt)
    i_h = I.abbe_image(m, opt, pix, zt / 2)
    i_q = I.abbe_image(m, opt, pix, zt / 4)
    assert np.abs(i_t - i0).max() < 1e-12
    assert np.abs(i_h - np.roll(i0, -period // 2, axis=1)).max() < 1e-12
    assert np.abs(i_q - i0).max() > 1e-2                           # not periodic at a quarter of z_T
    # the SOCS route (TCC eigen-kernels of Eqs. (2)-(3)) self-images at the same distance
    lam0, phi0, _ = O.socs_kernels(opt, n, pix, 0.0, 1)
    lamt, phit, _ = O.socs_kernels(opt, n, pix, zt, 1)
    assert np.abs(I.socs_image(m, lamt, phit) - I.socs_image(m, lam0, phi0)).max() < 1e-12


def test_planted_paraxial_defocus_misses_the_talbot_length(monkeypatch):
    """A pupil with the paraxial phase -pi lambda z f^2 / n (right sign, right index) puts
    the self-image at 2 n / (lambda f^2), about 13 % beyond the true z_T at this period."""
    from oracle import imaging as I
    n, period, width, pix = 208, 26, 10, 8.0
    opt = ON_AXIS
    m = _line_grating(n, period, width)
    i0 = I.abbe_image(m, opt, pix, 0.0)
    zt = _talbot_length(opt, period * pix)
    orig = O.pupil

    def paraxial(fx, fy, o, z):
        return orig(fx, fy, o, 0.0) * np.exp(-1j * np.pi * o.wavelength_nm * z * (fx * fx + fy * fy) / o.n_medium)

    monkeypatch.setattr(I, "pupil", paraxial)
    assert np.abs(I.abbe_image(m, opt, pix, zt) - i0).max() > 1e-2
