"""GPU intensity VJP, AI input channels (Eq. (9)) and print images (Eqs. (15)-(17)) vs the oracle.

Bounds: the VJP as the ILT gradient (max |d| <= 1e-4 of max |dm|); channel 1
(image / max) 1e-5; channel 2 (affinely normalised gradient) 1e-4; print
images exact wherever the oracle's value is farther than 1e-5 from the
threshold, and L_litho within the count of such undecided pixels.
"""
import numpy as np
import pytest

import synth
from oracle import ai as OA
from oracle import ilt as OIL
from oracle import imaging as OI
from tests.gpu_util import DUV_ANNULAR, oracle_kernel_set

pytestmark = pytest.mark.gpu


def _setup(n=256, focus=(0.0, 50.0), k=8, b=2):
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, 8.0, list(focus), k)
    targets = np.stack([synth.random_rect_mask(n, seed=600 + i, count=n // 5) for i in range(b)]).astype(np.float32)
    return lam, phi, targets


@pytest.mark.parametrize("precision", ["fft32", "fft32/coarse"])
def test_intensity_vjp_matches_oracle(litho_lib, cuda, precision):
    import torch
    L = litho_lib
    n = 256
    lam, phi, targets = _setup(n)
    kern = L.litho_upload_kernels(n, 8.0, lam, phi)
    if precision.endswith("/coarse"):
        assert 0 < kern.grid(precision) < n
    up = synth.random_field((2, 2, n, n), seed=7).astype(np.float32)
    dm = L.litho_intensity_vjp(kern, torch.from_numpy(targets).to(cuda), torch.from_numpy(up).to(cuda),
                               dose=1.3, precision=precision).cpu().numpy()
    ones = L.litho_intensity_vjp(kern, torch.from_numpy(targets).to(cuda), None, f_first=1, f_count=1,
                                 precision=precision).cpu().numpy()
    for c in range(2):
        m = targets[c].astype(np.float64)
        ref = OIL.intensity_vjp(m, list(zip(lam, phi)), [up[c, 0].astype(np.float64), up[c, 1].astype(np.float64)],
                                dose=1.3)
        assert np.abs(dm[c] - ref).max() <= 1e-4 * np.abs(ref).max()
        ref1 = OIL.intensity_vjp(m, [(lam[1], phi[1])], [np.ones((n, n))])
        assert np.abs(ones[c] - ref1).max() <= 1e-4 * np.abs(ref1).max()


@pytest.mark.parametrize("precision", ["fft32", "fft32/coarse"])
def test_ai_inputs_match_oracle(litho_lib, cuda, precision):
    import torch
    L = litho_lib
    n = 256
    lam, phi, targets = _setup(n, b=3)
    kern = L.litho_upload_kernels(n, 8.0, lam, phi)
    if precision.endswith("/coarse"):
        assert 0 < kern.grid(precision) < n
    x = L.litho_ai_inputs(kern, torch.from_numpy(targets).to(cuda), focus=1, precision=precision).cpu().numpy()
    ref, _, _ = OA.ai_channels(targets, lam[1], phi[1])
    assert np.array_equal(x[:, 0], targets)
    assert np.abs(x[:, 1] - ref[:, 1]).max() <= 1e-5
    assert np.abs(x[:, 2] - ref[:, 2]).max() <= 1e-4
    assert np.isclose(x[:, 1].max(), 1.0) and np.isclose(x[:, 2].min(), 0.0) and np.isclose(x[:, 2].max(), 1.0)


def test_ai_inputs_2048_on_the_1024_point_coarse_grid(litho_lib, cuda):
    """The AI step's clip size: on a 1024-point coarse grid the warp-per-row stage 2 writes the
    coarse image's row spectra for the interpolation itself."""
    import torch
    L = litho_lib
    n = 2048
    lam, phi, targets = _setup(n, focus=(0.0,), k=6, b=1)
    kern = L.litho_upload_kernels(n, 8.0, lam, phi)
    assert kern.grid("fft32/coarse") == 1024
    x = L.litho_ai_inputs(kern, torch.from_numpy(targets).to(cuda), focus=0, precision="fft32/coarse").cpu().numpy()
    ref, _, _ = OA.ai_channels(targets, lam[0], phi[0])
    assert np.array_equal(x[:, 0], targets)
    assert np.abs(x[:, 1] - ref[:, 1]).max() <= 1e-5
    assert np.abs(x[:, 2] - ref[:, 2]).max() <= 1e-4


def test_print_images_match_oracle(litho_lib, cuda):
    import torch
    L = litho_lib
    n, pixel = 256, 8.0
    lam, phi, targets = _setup(n, focus=(0.0,), b=2)
    imgs = np.stack([OI.socs_image(t.astype(np.float64), lam[0], phi[0]) for t in targets])
    zr, zp, loss, blur = L.litho_print_images(torch.from_numpy(targets).to(cuda),
                                              torch.from_numpy(imgs.astype(np.float32)).to(cuda),
                                              pixel, 12.0, 0.5, 0.3)
    rzr, rzp, rloss = OA.print_images(targets, imgs.astype(np.float32), 12.0, pixel, 0.5, 0.3)
    from oracle import resist as OR
    rblur = np.stack([OR.blur(t.astype(np.float64), 12.0, pixel) for t in targets])
    sure_r = np.abs(rblur - 0.5) > 1e-5
    sure_p = np.abs(imgs.astype(np.float32).astype(np.float64) - 0.3) > 1e-5
    zr, zp = zr.cpu().numpy(), zp.cpu().numpy()
    assert np.array_equal(zr[sure_r], rzr[sure_r]) and np.array_equal(zp[sure_p], rzp[sure_p])
    undecided = (~sure_r | ~sure_p).reshape(2, -1).sum(axis=1)
    assert np.all(np.abs(loss.cpu().numpy() - rloss) <= undecided)
    assert rloss.min() > 0
