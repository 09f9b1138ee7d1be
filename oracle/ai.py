"""Oracle input channels of the AI initialiser and its lithography-consistency
images (Eqs. (9), (15)-(17)), FP64.

Test infrastructure only (see the package docstring).

Readings:

* Eq. (9): M0 = Z_t (the binary target), I0 = the aerial image of the target
  at the nominal focus plane, (dI/dM)0 = the gradient of the total nominal
  intensity sum_x I0(x) with respect to the mask pixels, i.e. the
  vector-Jacobian product of Eq. (4) with a field of ones.  "Each scaled by a
  global normalisation factor so that all values lie within [0, 1]": over the
  batch of clips, I0 is divided by its maximum (it is non-negative) and dI/dM,
  which has either sign, is mapped affinely by its minimum and maximum; the
  target is already 0/1.  A constant channel maps to 0.
* Eq. (16): Z_round = [G_sigma (x) Z_t >= tau_round], with G_sigma the
  normalised, truncated, periodic Gaussian of the resist model (Eq. (5)).
* Eq. (17): Z_print = [I >= tau_print] on the aerial image itself.
* Eq. (15): L_litho = || Z_print - Z_round ||_1 per clip, the number of pixels
  where the two prints differ.
"""
from __future__ import annotations

import numpy as np

from .ilt import intensity_vjp
from .imaging import socs_image
from .resist import blur


def ai_channels(targets, lam, phi, dose: float = 1.0):
    """targets [b][n][n]; lam [K], phi [K][C][C] of the nominal plane -> X [b][3][n][n]."""
    t = np.asarray(targets, dtype=np.float64)
    img = np.stack([socs_image(z, lam, phi, dose) for z in t])
    grad = np.stack([intensity_vjp(z, [(lam, phi)], [np.ones_like(z)], dose) for z in t])
    imax = img.max()
    i0 = img / imax if imax > 0 else np.zeros_like(img)
    lo, hi = grad.min(), grad.max()
    g0 = (grad - lo) / (hi - lo) if hi > lo else np.zeros_like(grad)
    return np.stack([t, i0, g0], axis=1), img, grad


def print_images(targets, images, sigma_nm: float, pixel_nm: float, tau_round: float, tau_print: float):
    """Z_round [b][n][n], Z_print [b][n][n] (0/1) and L_litho [b] (Eqs. (15)-(17))."""
    t = np.asarray(targets, dtype=np.float64)
    zr = np.stack([(blur(z, sigma_nm, pixel_nm) >= tau_round) for z in t]).astype(np.uint8)
    zp = (np.asarray(images, dtype=np.float64) >= tau_print).astype(np.uint8)
    loss = np.abs(zp.astype(np.int64) - zr.astype(np.int64)).reshape(len(t), -1).sum(axis=1)
    return zr, zp, loss
