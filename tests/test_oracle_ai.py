"""Pins of the oracle's AI input channels and print-consistency images (Eqs. (9), (15)-(17)).

The gradient channel is the adjoint of Eq. (4) applied to ones, so it must
equal the derivative of the total intensity: checked by central finite
differences of sum_x I on a few pixels, and by linearity (the total intensity
is quadratic in m, so <grad, m> = 2 sum_x I).  The normalisations are checked
against their definition's extremes; Eqs. (15)-(17) on a hand-made example.
"""
import numpy as np

import synth
from oracle import ai as OA
from oracle import imaging as OI
from tests.gpu_util import DUV_ANNULAR, oracle_kernel_set


def test_gradient_channel_is_the_derivative_of_the_total_intensity():
    n, pixel = 32, 8.0
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [0.0], 6)
    z = synth.random_rect_mask(n, seed=4, count=6, side_lo=3, side_hi=8).astype(np.float64)
    x, img, grad = OA.ai_channels(z[None], lam[0], phi[0])
    total = lambda m: OI.socs_image(m, lam[0], phi[0]).sum()  # noqa: E731
    h = 1e-4
    for (i, j) in [(3, 4), (10, 20), (17, 17), (31, 0)]:
        e = np.zeros_like(z)
        e[i, j] = h
        fd = (total(z + e) - total(z - e)) / (2 * h)
        assert abs(fd - grad[0, i, j]) <= 1e-8 * max(1.0, abs(fd))
    # sum_x I is a quadratic form in m: <d(sum I)/dm, m> = 2 sum I
    assert np.isclose(np.sum(grad[0] * z), 2 * img[0].sum(), rtol=1e-10)
    # channels: target as is, image scaled by its maximum, gradient affinely onto [0, 1]
    assert np.array_equal(x[0, 0], z)
    assert np.isclose(x[0, 1].max(), 1.0) and x[0, 1].min() >= 0.0
    assert np.isclose(x[0, 2].min(), 0.0) and np.isclose(x[0, 2].max(), 1.0)


def test_print_images_and_litho_loss_by_hand():
    n = 16
    t = np.zeros((1, n, n))
    t[0, 4:12, 4:12] = 1.0                        # an 8 x 8 square
    img = np.zeros((1, n, n))
    img[0, 5:12, 4:12] = 0.6                      # prints one row short
    img[0, 0, 0] = 0.6                            # and one stray pixel
    # a blur narrower than a pixel leaves the square as it is (taps 1, ~1e-7, ...)
    zr, zp, loss = OA.print_images(t, img, sigma_nm=1.0, pixel_nm=8.0, tau_round=0.5, tau_print=0.5)
    assert np.array_equal(zr[0], t[0].astype(np.uint8))
    assert loss[0] == 8 + 1
    assert zp.sum() == 7 * 8 + 1
