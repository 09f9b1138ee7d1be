"""Oracle ILT loss and adjoint gradient (FP64).

Test infrastructure only (see the package docstring).

Pixel-based ILT (the paper's Section I prior art, and the dL/dM input channel
of its Eq. (9)) over several focus planes f with SOCS kernels (lam_kf, Phi_kf):

    m      = sigmoid(alpha * theta)
    I_f    = D sum_k lam_kf |E_kf|^2,      E_kf = sum_u M(u) Phi_kf(u) e^{2 pi i u.x/N}   (Eq. (4))
    Ib_f   = g (x) I_f                                                                  (Eq. (5))
    Z_f    = sigmoid(beta * (Ib_f - t))
    L      = sum_f sum_x (Z_f - target)^2

Adjoint, written out by the chain rule (g is symmetric, so the adjoint of the
periodic blur is the blur itself):

    q_f    = 2 (Z_f - target) * beta * Z_f (1 - Z_f)          dL/dIb_f
    G_f    = g (x) q_f                                         dL/dI_f
    H_kf   = sum_x G_f(x) E_kf(x) e^{-2 pi i u.x/N}            forward DFT, on the crop
    S      = sum_f sum_k lam_kf conj(Phi_kf) H_kf
    dL/dm  = 2 D N^-2 Re sum_u S(u) e^{+2 pi i u.x/N}
    dL/dth = dL/dm * alpha m (1 - m)

The sum over focus planes is unweighted (the paper does not say whether the
planes are summed or averaged).
"""
from __future__ import annotations

import numpy as np

from .imaging import band, embed, inverse_unnormalised, mask_spectrum
from .resist import blur


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def intensity_vjp(m, kernels, gfields, dose: float = 1.0):
    """dL/dm for L with dL/dI_f = gfields[f], I_f the SOCS images of m."""
    n = m.shape[-1]
    mf = mask_spectrum(m)
    s = None
    for (lam, phi), gf in zip(kernels, gfields):
        c = phi.shape[-1]
        mb = band(mf, c)
        if s is None:
            s = np.zeros((c, c), dtype=np.complex128)
        for k in range(len(lam)):
            if lam[k] == 0.0:
                continue
            e = inverse_unnormalised(embed(mb * phi[k], n))
            h = band(np.fft.fft2(gf * e), c)
            s += lam[k] * np.conj(phi[k]) * h
    return 2.0 * dose / (n * n) * inverse_unnormalised(embed(s, n)).real


def forward(theta, target, kernels, dose, alpha, beta, thr, sigma_nm, pixel_nm):
    """Returns (L, per-focus I, Ib, Z) for the ILT objective."""
    m = sigmoid(alpha * np.asarray(theta, dtype=np.float64))
    mf = mask_spectrum(m)
    n = m.shape[-1]
    loss = 0.0
    outs = []
    for lam, phi in kernels:
        c = phi.shape[-1]
        mb = band(mf, c)
        img = np.zeros((n, n))
        for k in range(len(lam)):
            if lam[k] == 0.0:
                continue
            e = inverse_unnormalised(embed(mb * phi[k], n))
            img += lam[k] * (e.real ** 2 + e.imag ** 2)
        img *= dose
        ib = blur(img, sigma_nm, pixel_nm)
        z = sigmoid(beta * (ib - thr))
        loss += float(np.sum((z - target) ** 2))
        outs.append((img, ib, z))
    return loss, m, outs


def loss_and_grad(theta, target, kernels, dose=1.0, alpha=4.0, beta=25.0, thr=0.3, sigma_nm=10.0,
                  pixel_nm=8.0):
    """ILT loss L and dL/dtheta by the adjoint formulas of the module docstring."""
    target = np.asarray(target, dtype=np.float64)
    loss, m, outs = forward(theta, target, kernels, dose, alpha, beta, thr, sigma_nm, pixel_nm)
    gfields = []
    for _img, _ib, z in outs:
        q = 2.0 * (z - target) * beta * z * (1.0 - z)
        gfields.append(blur(q, sigma_nm, pixel_nm))
    dm = intensity_vjp(m, kernels, gfields, dose)
    return loss, dm * alpha * m * (1.0 - m)


def loss_only(theta, target, kernels, **kw):
    args = dict(dose=1.0, alpha=4.0, beta=25.0, thr=0.3, sigma_nm=10.0, pixel_nm=8.0)
    args.update(kw)
    loss, _m, _o = forward(theta, np.asarray(target, dtype=np.float64), kernels, args["dose"], args["alpha"],
                           args["beta"], args["thr"], args["sigma_nm"], args["pixel_nm"])
    return loss


def fd_grad(theta, target, kernels, pixels, h=1e-4, **kw):
    """Central finite differences of L at the given (y, x) pixels."""
    theta = np.asarray(theta, dtype=np.float64)
    out = []
    for (y, x) in pixels:
        tp = theta.copy()
        tp[y, x] += h
        tm = theta.copy()
        tm[y, x] -= h
        out.append((loss_only(tp, target, kernels, **kw) - loss_only(tm, target, kernels, **kw)) / (2 * h))
    return np.array(out)
