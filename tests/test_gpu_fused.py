"""litho_aerial_resist and the batched FP32 stage launches against the FP64 oracle.

On the coarse grid the resist blur is applied in the frequency domain inside
the interpolation to N x N (the image is band-limited, so this is the periodic
convolution with the truncated taps, exactly up to rounding); the image and
its blur come out of one complex inverse transform.  The blur is held to the
same bound as the image (1e-5 for the FP32 and split paths, 2e-3 for plain
fp16), printed bytes must agree with the oracle wherever the oracle's blurred
value is farther than that bound from the threshold, and contours within
0.1 nm.  Without the coarse grid the call is litho_aerial + litho_resist.
"""
import numpy as np
import pytest

import synth
from oracle import imaging as OI
from oracle import resist as OR
from tests.gpu_util import DUV_ANNULAR, DUV_QUAD41, oracle_kernel_set

pytestmark = pytest.mark.gpu

TOL = {"fft32": 1e-5, "fft32/coarse": 1e-5, "fp16x3/coarse": 1e-5, "fp16/coarse": 2e-3}
THR = 0.3


def _masks(n, b, seed):
    return np.stack([synth.random_rect_mask(n, seed=seed + i, count=n // 5) for i in range(b)]).astype(np.float32)


@pytest.mark.parametrize("precision", ["fft32/coarse", "fp16x3/coarse", "fp16/coarse", "fft32"])
@pytest.mark.parametrize("preset,n,focus,k,b,sigma", [(DUV_ANNULAR, 256, [0.0], 8, 2, 10.0),
                                                      (DUV_QUAD41, 512, [-50.0, 50.0], 12, 3, 6.0)])
def test_aerial_resist_matches_oracle(litho_lib, cuda, precision, preset, n, focus, k, b, sigma):
    import torch
    L = litho_lib
    pixel = 8.0
    lam, phi = oracle_kernel_set(preset, n, pixel, focus, k)
    kern = L.litho_upload_kernels(n, pixel, lam, phi)
    masks = _masks(n, b, 300)
    img, ib, pr = L.litho_aerial_resist(kern, torch.from_numpy(masks).to(cuda), precision=precision, sigma_nm=sigma,
                                        threshold=THR)
    L.litho_check_device(kern)
    img, ib, pr = img.cpu().numpy(), ib.cpu().numpy(), pr.cpu().numpy()
    tol = TOL[precision]
    worst_i = worst_b = worst_epe = 0.0
    for i in range(b):
        for f in range(len(focus)):
            ref = OI.socs_image(masks[i].astype(np.float64), lam[f], phi[f])
            ref_b = OR.blur(ref, sigma, pixel)
            worst_i = max(worst_i, np.abs(img[i, f] - ref).max())
            worst_b = max(worst_b, np.abs(ib[i, f] - ref_b).max())
            sure = np.abs(ref_b - THR) > tol
            assert np.array_equal(pr[i, f][sure], (ref_b[sure] >= THR).astype(np.uint8))
            assert np.array_equal(pr[i, f], (ib[i, f] >= np.float32(THR)).astype(np.uint8))
            if tol <= 1e-5:   # the 0.1 nm contour bound belongs to the 1e-5 paths
                worst_epe = max(worst_epe,
                                OR.edge_placement_difference(ref_b, ib[i, f].astype(np.float64), THR, pixel))
    print(f"{precision} n={n}: image {worst_i:.2e} blur {worst_b:.2e} EPE {worst_epe:.3f} nm")
    assert worst_i <= tol and worst_b <= tol
    assert worst_epe <= 0.1


@pytest.mark.parametrize("precision", ["fft32/coarse", "fp16x3/coarse"])
def test_fused_resist_agrees_with_separate_resist(litho_lib, cuda, precision):
    """Frequency-domain blur inside the interpolation vs the direct blur kernel on the same image."""
    import torch
    L = litho_lib
    n, pixel = 512, 8.0
    lam, phi = oracle_kernel_set(DUV_QUAD41, n, pixel, [0.0, 50.0], 10)
    kern = L.litho_upload_kernels(n, pixel, lam, phi)
    m = torch.from_numpy(_masks(n, 2, 410)).to(cuda)
    img, ib, pr = L.litho_aerial_resist(kern, m, precision=precision, sigma_nm=10.0, threshold=THR)
    img2 = L.litho_aerial(kern, m, precision=precision)
    ib2, _ = L.litho_resist(img2, pixel, 10.0, THR)
    assert (img - img2).abs().max().item() <= 2e-6
    assert (ib - ib2).abs().max().item() <= 2e-6
    assert pr.dtype == torch.uint8 and int(pr.max()) == 1 and int(pr.min()) == 0


def test_aerial_resist_full_size_rows(litho_lib, cuda):
    """Headline shape (2048^2 at 8 nm, quadrupole, K = 24, 3 focus planes, coarse grid,
    fused resist): sampled blurred rows against the oracle, from the oracle's image rows
    y - R .. y + R and the oracle's taps."""
    import torch
    L = litho_lib
    n, pixel, k, focus, sigma = 2048, 8.0, 24, [-50.0, 0.0, 50.0], 10.0
    lam, phi = oracle_kernel_set(DUV_QUAD41, n, pixel, focus, k)
    kern = L.litho_upload_kernels(n, pixel, lam, phi)
    masks = np.stack([synth.manhattan_mask(n, seed=1234 + i) for i in range(2)]).astype(np.float32)
    img, ib, pr = L.litho_aerial_resist(kern, torch.from_numpy(masks).to(cuda), precision="fft32/coarse",
                                        sigma_nm=sigma, threshold=THR)
    ib, pr = ib.cpu().numpy(), pr.cpu().numpy()
    g = OR.gaussian_taps(sigma, pixel)
    r = (len(g) - 1) // 2
    rows = sorted(set(synth.Stream(23).integers(0, n - 1, 3).tolist()) | {0, n - 1})
    c = phi.shape[-1]
    for i in range(2):
        mb = OI.band(OI.mask_spectrum(masks[i].astype(np.float64)), c)
        for f in (0, 2):
            for y in rows:
                ys = [(y + a) % n for a in range(-r, r + 1)]
                band_rows = OI.socs_rows(mb, lam[f], phi[f], n, ys)     # rows y - r .. y + r
                col = sum(g[r - a] * band_rows[r + a] for a in range(-r, r + 1))
                ref = sum(g[b + r] * np.roll(col, b) for b in range(-r, r + 1))
                assert np.abs(ib[i, f, y] - ref).max() <= 1e-5, (i, f, y)
                sure = np.abs(ref - THR) > 1e-5
                assert np.array_equal(pr[i, f, y][sure], (ref[sure] >= THR).astype(np.uint8))


def test_bench_shape_64_clips_sampled_rows(litho_lib, cuda):
    """The benchmark's exact workload and launch shape: 64 clips of 2048^2 (the benchmark's
    masks, seeds 1234..1297) through litho_aerial_resist fft32/coarse in one call, which the
    library runs as 8 stage launches of 8 clips; sampled blurred rows of clips at the start,
    end and inside of several launch groups, all 3 focus planes, against the oracle."""
    import torch
    L = litho_lib
    n, pixel, k, focus, sigma, b = 2048, 8.0, 24, [-50.0, 0.0, 50.0], 10.0, 64
    lam, phi = oracle_kernel_set(DUV_QUAD41, n, pixel, focus, k)
    kern = L.litho_upload_kernels(n, pixel, lam, phi)
    masks = np.stack([synth.manhattan_mask(n, seed=1234 + i) for i in range(b)])
    img, ib, pr = L.litho_aerial_resist(kern, torch.from_numpy(masks).to(cuda), precision="fft32/coarse",
                                        sigma_nm=sigma, threshold=THR)
    L.litho_check_device(kern)
    g = OR.gaussian_taps(sigma, pixel)
    r = (len(g) - 1) // 2
    c = phi.shape[-1]
    worst_i = worst_b = 0.0
    for i in (0, 7, 8, 35, 56, 63):
        y = int(synth.Stream(31 + i).integers(0, n - 1, 1)[0])
        ys = [(y + a) % n for a in range(-r, r + 1)]
        img_i, ib_i, pr_i = img[i, :, y].cpu().numpy(), ib[i, :, y].cpu().numpy(), pr[i, :, y].cpu().numpy()
        mb = OI.band(OI.mask_spectrum(masks[i].astype(np.float64)), c)
        for f in range(3):
            band_rows = OI.socs_rows(mb, lam[f], phi[f], n, ys)           # image rows y - r .. y + r
            worst_i = max(worst_i, np.abs(img_i[f] - band_rows[r]).max())
            col = sum(g[r - a] * band_rows[r + a] for a in range(-r, r + 1))
            ref = sum(g[bb + r] * np.roll(col, bb) for bb in range(-r, r + 1))
            worst_b = max(worst_b, np.abs(ib_i[f] - ref).max())
            sure = np.abs(ref - THR) > 1e-5
            assert np.array_equal(pr_i[f][sure], (ref[sure] >= THR).astype(np.uint8)), (i, f, y)
    print(f"64 x 2048^2 fft32/coarse: image {worst_i:.2e} blur {worst_b:.2e}")
    assert worst_i <= 1e-5 and worst_b <= 1e-5


def test_clip_groups_match_single_clip_calls(litho_lib, cuda):
    """70 clips of 128^2 run as two groups of 35 per stage launch; each clip's image equals
    the image of the same clip imaged alone (bit for bit), and a few match the oracle."""
    import torch
    L = litho_lib
    n, pixel = 128, 8.0
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [0.0, 40.0], 4)
    kern = L.litho_upload_kernels(n, pixel, lam, phi)
    masks = np.stack([synth.random_rect_mask(n, seed=5000 + i, count=12) for i in range(70)]).astype(np.float32)
    dm = torch.from_numpy(masks).to(cuda)
    for precision in ("fft32", "fft32/coarse"):
        batch = L.litho_aerial(kern, dm, precision=precision).cpu().numpy()
        for i in (0, 1, 34, 35, 36, 69):
            alone = L.litho_aerial(kern, dm[i:i + 1].contiguous(), precision=precision).cpu().numpy()
            assert np.array_equal(batch[i], alone[0]), (precision, i)
        for i in (0, 35, 69):
            for f in range(2):
                ref = OI.socs_image(masks[i].astype(np.float64), lam[f], phi[f])
                assert np.abs(batch[i, f] - ref).max() <= 1e-5
