"""Coarse-grid evaluation (LITHO_GRID_COARSE) against the FP64 oracle.

The fields are evaluated on nc x nc (nc = smallest power of two >= 2C) and
the image is Fourier-interpolated to N x N.  Since I has no frequency at or
beyond C, this is exact up to rounding, so the tolerances are those of the
full-grid paths: 1e-5 (FP32 FFT, split fp16 x3) and 2e-3 (plain fp16).
"""
import numpy as np
import pytest

import synth
from oracle import imaging as OI
from tests.gpu_util import DUV_ANNULAR, DUV_QUAD41, oracle_kernel_set

pytestmark = pytest.mark.gpu

TOL = {"fft32/coarse": 1e-5, "fp16x3/coarse": 1e-5, "bf16x3/coarse": 1e-5, "fp16/coarse": 2e-3}


def _run(L, cuda, lam, phi, n, pixel, masks, precision):
    import torch
    kern = L.litho_upload_kernels(n, pixel, lam, phi)
    out = L.litho_aerial(kern, torch.from_numpy(np.ascontiguousarray(masks, dtype=np.float32)).to(cuda),
                         precision=precision)
    L.litho_check_device(kern)
    return out.cpu().numpy().astype(np.float64), kern


@pytest.mark.parametrize("precision", ["fft32/coarse", "fp16x3/coarse", "fp16/coarse", "bf16x3/coarse"])
@pytest.mark.parametrize("preset,n,focus,k,b", [(DUV_ANNULAR, 256, [0.0], 8, 2),
                                                (DUV_QUAD41, 512, [-50.0, 50.0], 12, 3)])
def test_coarse_grid_matches_oracle(litho_lib, cuda, precision, preset, n, focus, k, b):
    lam, phi = oracle_kernel_set(preset, n, 8.0, focus, k)
    masks = np.stack([synth.random_rect_mask(n, seed=900 + i, count=n // 5) for i in range(b)])
    got, kern = _run(litho_lib, cuda, lam, phi, n, 8.0, masks, precision)
    worst = 0.0
    for i in range(b):
        for f in range(len(focus)):
            worst = max(worst, np.abs(got[i, f] - OI.socs_image(masks[i].astype(np.float64), lam[f], phi[f])).max())
    print(f"{precision} n={n} crop={phi.shape[-1]} max|err|={worst:.3e}")
    assert worst <= TOL[precision]


@pytest.mark.parametrize("precision", ["fft32/coarse", "fp16x3/coarse", "bf16x3/coarse"])
def test_coarse_grid_full_size_rows(litho_lib, cuda, precision):
    n, k, focus = 2048, 24, [-50.0, 0.0, 50.0]
    lam, phi = oracle_kernel_set(DUV_QUAD41, n, 8.0, focus, k)
    masks = np.stack([synth.manhattan_mask(n, seed=1234 + i) for i in range(2)])
    got, _ = _run(litho_lib, cuda, lam, phi, n, 8.0, masks, precision)
    rows = sorted(set(synth.Stream(17).integers(0, n - 1, 6).tolist()) | {0, 1, 1023, n - 1})
    c = phi.shape[-1]
    for i in range(2):
        mb = OI.band(OI.mask_spectrum(masks[i]), c)
        for f in range(3):
            err = np.abs(got[i, f, rows] - OI.socs_rows(mb, lam[f], phi[f], n, rows)).max()
            assert err <= TOL[precision], (i, f, err)


def test_coarse_flag_ignored_when_grid_is_not_smaller(litho_lib, cuda):
    n = 64
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, 16.0, [0.0], 4)
    masks = synth.random_rect_mask(n, seed=1, count=10)[None]
    a, _ = _run(litho_lib, cuda, lam, phi, n, 16.0, masks, "fft32")
    b, _ = _run(litho_lib, cuda, lam, phi, n, 16.0, masks, "fft32/coarse")
    assert np.array_equal(a, b)


def test_coarse_grid_sizes(litho_lib, cuda):
    """Coarse grids per path: the FP32 FFT path takes the smallest power of two >= 2C,
    the tensor-core path also 896 = 16 x 8 x 7 when that is smaller; 0 when not below N."""
    L = litho_lib
    cases = [(2048, 8.0, 448, 1024, 896), (1024, 16.0, 448, 0, 896), (1024, 8.0, 224, 512, 512),
             (256, 8.0, 64, 128, 128), (64, 8.0, 32, 0, 0)]
    for n, pixel, crop, fft, tc in cases:
        lam = np.ones((1, 1))
        phi = np.zeros((1, 1, crop, crop), dtype=np.complex128)
        kern = L.litho_upload_kernels(n, pixel, lam, phi)
        assert (kern.grid("fft32"), kern.grid("fp16x3")) == (fft, tc), (n, crop)


@pytest.mark.parametrize("precision", ["fp16x3/coarse", "fp16/coarse", "fft32/coarse"])
def test_coarse_grid_896_matches_oracle(litho_lib, cuda, precision):
    """1024^2 at 16 nm (band of 448 columns): the tensor-core path evaluates on the
    896 x 896 grid (radix 16, 8, 7 transforms for its operands and the interpolation);
    for the FFT path the flag does not apply (1024 is not below N).  Whole images
    against the oracle."""
    n, pixel, k, focus = 1024, 16.0, 8, [0.0, 60.0]
    lam, phi = oracle_kernel_set(DUV_QUAD41, n, pixel, focus, k)
    assert phi.shape[-1] == 448
    masks = np.stack([synth.random_rect_mask(n, seed=700 + i, count=150, side_lo=3, side_hi=10) for i in range(2)])
    got, kern = _run(litho_lib, cuda, lam, phi, n, pixel, masks, precision)
    assert kern.grid(precision) == (0 if precision.startswith("fft32") else 896)
    worst = 0.0
    for i in range(2):
        for f in range(2):
            worst = max(worst, np.abs(got[i, f] - OI.socs_image(masks[i].astype(np.float64), lam[f], phi[f])).max())
    print(f"{precision} max|err|={worst:.3e}")
    assert worst <= TOL[precision]
