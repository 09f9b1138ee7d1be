"""Pins for the oracle's resist (Eq. (5)) and ILT adjoint gradient.

* resist: brute-force 2-D periodic convolution with the outer-product kernel,
  impulse response, constant preservation, crossing positions of a ramp;
* ILT: central finite differences of the FP64 loss, and the adjoint identity
  <J dm, g> = <dm, J^T g> (the image is quadratic in m, so the central
  difference of I is exact up to rounding).
"""
import numpy as np
import pytest

import synth
from oracle import ilt as L
from oracle import imaging as I
from oracle import optics as O
from oracle import resist as R

DUV = O.Optics(193.0, 1.35, 1.44, O.ANNULAR, 21, 0.6, 0.9)


def test_gaussian_taps():
    g = R.gaussian_taps(10.0, 8.0)
    assert len(g) == 11 and abs(g.sum() - 1) < 1e-15 and np.allclose(g, g[::-1])
    assert len(R.gaussian_taps(10.0, 1.0)) == 81
    # ratio of neighbouring taps is the Gaussian's
    assert abs(g[6] / g[5] - np.exp(-64.0 / 200.0)) < 1e-14


def test_blur_matches_brute_force_2d_convolution():
    n = 16
    img = synth.random_field((n, n), seed=9, lo=0.0, hi=1.0)
    g = R.gaussian_taps(10.0, 8.0)
    r = (len(g) - 1) // 2
    ref = np.zeros_like(img)
    for y in range(n):
        for x in range(n):
            acc = 0.0
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    acc += g[a + r] * g[b + r] * img[(y - a) % n, (x - b) % n]
            ref[y, x] = acc
    assert np.abs(R.blur(img, 10.0, 8.0) - ref).max() < 1e-14
    # impulse -> outer product of the taps; constant -> constant
    d = np.zeros((n, n))
    d[4, 7] = 1.0
    out = R.blur(d, 10.0, 8.0)
    assert abs(out[4 + 2, 7 - 3] - g[r + 2] * g[r - 3]) < 1e-16
    assert np.abs(R.blur(np.full((n, n), 0.37), 10.0, 8.0) - 0.37).max() < 1e-15


def test_crossings_and_edge_placement_difference():
    n = 32
    x = np.arange(n, dtype=np.float64)
    ramp = np.tile(np.where(x < n // 2, x, n - x) / 10.0, (n, 1))   # tent; 0.35 is crossed at 3.5 and 28.5
    line, j, t = R.crossings(ramp, 0.35, axis=1)
    assert np.allclose(sorted(set(np.round(j + t, 12))), [3.5, 28.5])
    assert len(line) == 2 * n
    assert len(R.crossings(ramp, 0.35, axis=0)[0]) == 0
    assert R.edge_placement_difference(ramp, ramp, 0.35, 8.0) == 0.0
    shifted = np.tile(np.where(x < n // 2, x + 0.25, n - x + 0.25) / 10.0, (n, 1))
    d = R.edge_placement_difference(ramp, shifted, 0.35, 8.0)
    assert abs(d - 0.25 * 8.0) < 1e-9


def _small_problem(n=32, pix=16.0, k=6, focus=(-40.0, 0.0)):
    c = O.crop_size(DUV, n, pix)
    kernels = []
    for z in focus:
        lam, phi, _ = O.socs_kernels(DUV, n, pix, z, k, c)
        kernels.append((lam, phi))
    theta, target = synth.ilt_clip(n, pix, seed=42)
    return kernels, theta.astype(np.float64), target.astype(np.float64), pix


def test_adjoint_identity_of_the_intensity_map():
    kernels, theta, _t, pix = _small_problem()
    m = L.sigmoid(4 * theta)
    n = m.shape[0]
    dm = synth.random_field((n, n), seed=1)
    gs = [synth.random_field((n, n), seed=2 + f) for f in range(len(kernels))]
    eps = 1e-3
    lhs = 0.0
    for (lam, phi), g in zip(kernels, gs):
        jp = (I.socs_image(m + eps * dm, lam, phi) - I.socs_image(m - eps * dm, lam, phi)) / (2 * eps)
        lhs += np.sum(jp * g)
    rhs = np.sum(dm * L.intensity_vjp(m, kernels, gs))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_vjp_of_ones_is_the_parseval_closed_form():
    """With dL/dI = 1, L = sum_x I(x) = dose N^2 sum_v D(v) |M(v)|^2 (Parseval), D = sum_k lam_k |Phi_k|^2
    on the band, M = DFT(m)/N^2; so dL/dm = 2 dose Re sum_v D(v) M(v) e^{+2 pi i v.x/N}.  Both sides
    from plain numpy FFTs, against the oracle's image (for L) and its adjoint (for the gradient)."""
    kernels, theta, _t, pix = _small_problem()
    m = L.sigmoid(4 * theta)
    n = m.shape[0]
    dose = 1.7
    mf = np.fft.fft2(m) / (n * n)
    lam, phi = kernels[1]
    c = phi.shape[-1]
    idx = (np.arange(c) - c // 2) % n
    d = np.zeros((n, n))
    d[np.ix_(idx, idx)] = np.einsum("k,kvu->vu", lam, np.abs(phi) ** 2)
    total = dose * n * n * np.sum(d * np.abs(mf) ** 2)
    assert abs(np.sum(I.socs_image(m, lam, phi, dose)) - total) < 1e-10 * total
    closed = 2.0 * dose * np.real(np.fft.ifft2(d * mf) * (n * n))
    got = L.intensity_vjp(m, [(lam, phi)], [np.ones((n, n))], dose)
    assert np.abs(got - closed).max() < 1e-10 * np.abs(closed).max()


def test_gradient_matches_central_finite_differences():
    kernels, theta, target, pix = _small_problem()
    loss, grad = L.loss_and_grad(theta, target, kernels, pixel_nm=pix)
    assert loss > 0
    st = synth.Stream(77)
    pts = list(zip(st.integers(0, 31, 12), st.integers(0, 31, 12)))
    # include the pixels of largest gradient so the check is not vacuous
    flat = np.argsort(np.abs(grad).ravel())[-4:]
    pts += [divmod(int(f), 32) for f in flat]
    fd = L.fd_grad(theta, target, kernels, pts, h=1e-4, pixel_nm=pix)
    ad = np.array([grad[y, x] for y, x in pts])
    scale = np.abs(grad).max()
    assert scale > 1e-3
    assert np.abs(fd - ad).max() < 1e-7 * scale


def test_planted_sign_error_in_adjoint_is_caught(monkeypatch):
    """A conjugation dropped from the adjoint must fail the FD pin."""
    kernels, theta, target, pix = _small_problem()
    def _vjp_without_conj(m, kern, gfields, dose=1.0):
        n = m.shape[-1]
        mf = I.mask_spectrum(m)
        s = None
        for (lam, phi), gf in zip(kern, gfields):
            c = phi.shape[-1]
            mb = I.band(mf, c)
            s = np.zeros((c, c), dtype=np.complex128) if s is None else s
            for k in range(len(lam)):
                e = I.inverse_unnormalised(I.embed(mb * phi[k], n))
                s += lam[k] * phi[k] * I.band(np.fft.fft2(gf * e), c)      # conj(phi) dropped
        return 2.0 * dose / (n * n) * I.inverse_unnormalised(I.embed(s, n)).real

    monkeypatch.setattr(L, "intensity_vjp", _vjp_without_conj)
    _loss, grad = L.loss_and_grad(theta, target, kernels, pixel_nm=pix)
    flat = np.argsort(np.abs(grad).ravel())[-4:]
    pts = [divmod(int(f), 32) for f in flat]
    fd = L.fd_grad(theta, target, kernels, pts, h=1e-4, pixel_nm=pix)
    ad = np.array([grad[y, x] for y, x in pts])
    assert np.abs(fd - ad).max() > 1e-3 * np.abs(fd).max()


def test_planted_defocus_sign_error_is_caught(monkeypatch):
    """A pupil whose defocus term is paraxial-with-wrong-sign must fail the
    grating closed form at z != 0 against the correct pupil."""
    from tests.test_oracle_imaging import _grating_closed_form
    n, pix, period, width = 256, 8.0, 16, 8
    m = np.zeros((n, n))
    m[:, (np.arange(n) % period) < width] = 1.0
    ref = _grating_closed_form(n, period, width, DUV, pix, 50.0)
    orig = O.pupil

    def broken(fx, fy, opt, z):
        return orig(fx, fy, opt, 0.0) * np.exp(1j * np.pi * opt.wavelength_nm * z * (fx * fx + fy * fy)
                                                / opt.n_medium)

    import oracle.imaging as imaging_mod
    monkeypatch.setattr(imaging_mod, "pupil", broken)
    a = I.abbe_image(m, DUV, pix, 50.0)
    assert np.abs(a - ref[None, :]).max() > 1e-4
