"""GPU parity of the FP32 FFT path and the resist against the FP64 oracle.

Tolerances: 1e-5 absolute intensity (clear field = 1) on the FP32 path,
0.1 nm edge-placement difference at the resist threshold.
"""
import numpy as np
import pytest

import synth
from oracle import imaging as OI
from oracle import resist as OR
from tests.gpu_util import DUV_ANNULAR, DUV_QUAD21, DUV_QUAD41, oracle_kernel_set

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


def _run(litho_lib, cuda, lam, phi, n, pixel, masks, dose=1.0, precision="fft32"):
    import torch
    kern = litho_lib.litho_upload_kernels(n, pixel, lam, phi)
    m = torch.from_numpy(np.ascontiguousarray(masks, dtype=np.float32)).to(cuda)
    out = litho_lib.litho_aerial(kern, m, dose=dose, precision=precision)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), kern


CASES = [
    # preset, n, pixel, focus, k, batch, dose
    (DUV_ANNULAR, 256, 8.0, [0.0], 8, 1, 1.0),          # one clip of the 256^2 correctness workload
    (DUV_ANNULAR, 64, 8.0, [0.0, 40.0], 6, 3, 1.0),
    (DUV_QUAD41, 128, 8.0, [-50.0, 0.0, 50.0], 24, 2, 0.8),
    (DUV_QUAD21, 128, 8.0, [0.0], 24, 1, 1.0),          # rank 20 < K: four zero kernels
    (DUV_ANNULAR, 32, 16.0, [0.0], 5, 2, 1.0),          # crop == N
    (DUV_QUAD41, 512, 8.0, [30.0], 12, 1, 1.0),
    (DUV_ANNULAR, 1024, 8.0, [-60.0], 4, 1, 1.0),
]


@pytest.mark.parametrize("preset,n,pixel,focus,k,b,dose", CASES)
def test_fft32_matches_oracle(litho_lib, cuda, preset, n, pixel, focus, k, b, dose):
    lam, phi = oracle_kernel_set(preset, n, pixel, focus, k)
    masks = np.stack([synth.random_rect_mask(n, seed=100 + i, count=max(8, n // 6)) for i in range(b)])
    got, _ = _run(litho_lib, cuda, lam, phi, n, pixel, masks, dose)
    assert got.shape == (b, len(focus), n, n)
    for i in range(b):
        for f in range(len(focus)):
            ref = OI.socs_image(masks[i].astype(np.float64), lam[f], phi[f], dose)
            err = np.abs(got[i, f] - ref).max()
            assert err <= TOL_FP32, (i, f, err)


def test_clear_and_dark_field(litho_lib, cuda):
    n, pixel, k = 128, 8.0, 10
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [0.0, 50.0], k)
    masks = np.stack([np.ones((n, n)), np.zeros((n, n))])
    got, _ = _run(litho_lib, cuda, lam, phi, n, pixel, masks, dose=1.7)
    c = phi.shape[-1]
    for f in range(2):
        clear = 1.7 * sum(lam[f, j] * abs(phi[f, j, c // 2, c // 2]) ** 2 for j in range(k))
        assert np.abs(got[0, f] - clear).max() <= TOL_FP32
        assert np.abs(got[1, f]).max() == 0.0


def test_full_size_rows_2048_quadrupole_k24(litho_lib, cuda):
    """The 2048^2, K=24, 3-focus workload (two clips) on sampled full rows."""
    n, pixel, k, focus = 2048, 8.0, 24, [-50.0, 0.0, 50.0]
    lam, phi = oracle_kernel_set(DUV_QUAD41, n, pixel, focus, k)
    masks = np.stack([synth.manhattan_mask(n, seed=1234 + i) for i in range(2)])
    assert 0.35 <= masks[0].mean() < 0.4
    got, _ = _run(litho_lib, cuda, lam, phi, n, pixel, masks)
    st = synth.Stream(99)
    rows = sorted(set(st.integers(0, n - 1, 6).tolist()) | {0, n - 1})
    c = phi.shape[-1]
    for i in range(2):
        mb = OI.band(OI.mask_spectrum(masks[i]), c)
        for f in range(len(focus)):
            ref = OI.socs_rows(mb, lam[f], phi[f], n, rows)
            err = np.abs(got[i, f, rows] - ref).max()
            assert err <= TOL_FP32, (i, f, err)
        assert np.isfinite(got[i]).all() and got[i].min() >= 0.0


def test_library_builder_end_to_end(litho_lib, cuda):
    """litho_make_kernels (host FP64 build + upload) images like oracle kernels
    when K closes its eigenvalue cluster."""
    import torch
    L = litho_lib
    n, pixel, k = 256, 8.0, 8
    kern = L.litho_make_kernels(L.make_optics(**DUV_ANNULAR), n, pixel, [0.0], k)
    info = kern.info()
    assert info["gap"][0] > 1e-6 * info["lambda"][0, 0]
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [0.0], k)
    m = synth.random_rect_mask(n, seed=1234)
    out = L.litho_aerial(kern, torch.from_numpy(m[None]).to(cuda)).cpu().numpy()[0, 0]
    ref = OI.socs_image(m.astype(np.float64), lam[0], phi[0])
    assert np.abs(out - ref).max() <= TOL_FP32


def test_host_buffers_path_matches_device_path(litho_lib, cuda):
    import torch
    L = litho_lib
    n, pixel = 256, 8.0
    lam, phi = oracle_kernel_set(DUV_QUAD41, n, pixel, [0.0, 50.0], 6)
    kern = L.litho_upload_kernels(n, pixel, lam, phi)
    masks = np.stack([synth.random_rect_mask(n, seed=7 + i) for i in range(3)]).astype(np.float32)
    dev = L.litho_aerial(kern, torch.from_numpy(masks).to(cuda)).cpu().numpy()
    mh = torch.from_numpy(masks).pin_memory()
    oh = torch.empty((3, 2, n, n), dtype=torch.float32).pin_memory()
    ph = torch.empty((3, 2, n, n), dtype=torch.uint8).pin_memory()
    ws = torch.empty(L.litho_aerial_host_workspace_size(kern, 3), dtype=torch.uint8, device=cuda)
    L.litho_aerial_host(kern, mh, ws, intensity_host=oh, printed_host=ph, sigma_nm=10.0, threshold=0.3)
    assert np.array_equal(oh.numpy(), dev)
    ib, pr = L.litho_resist(torch.from_numpy(dev).to(cuda), pixel, 10.0, 0.3)
    assert np.array_equal(ph.numpy(), pr.cpu().numpy())
    # printed only (pageable numpy output)
    ph2 = np.zeros((3, 2, n, n), dtype=np.uint8)
    L.litho_aerial_host(kern, masks, ws, printed_host=ph2)
    assert np.array_equal(ph2, ph.numpy())


def test_errors_are_reported(litho_lib, cuda):
    import torch
    L = litho_lib
    n = 64
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, 8.0, [0.0], 4)
    kern = L.litho_upload_kernels(n, 8.0, lam, phi)
    m = torch.zeros((1, n, n), dtype=torch.float32, device=cuda)
    small = torch.empty(16, dtype=torch.uint8, device=cuda)
    with pytest.raises(L.LithoError) as e:
        L.litho_aerial(kern, m, workspace=small)
    assert e.value.status == L.ENOMEM
    ws = torch.empty(L.litho_aerial_workspace_size(kern, 1) + 512, dtype=torch.uint8, device=cuda)
    with pytest.raises(L.LithoError) as e:
        L.litho_aerial(kern, m, workspace=ws[8:])
    assert e.value.status == L.EINVAL


# ---- resist --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,pixel,sigma,planes", [(256, 8.0, 10.0, 3), (128, 1.0, 10.0, 2), (64, 8.0, 4.0, 1)])
def test_resist_matches_oracle(litho_lib, cuda, n, pixel, sigma, planes):
    import torch
    img = synth.random_field((planes, n, n), seed=5, lo=0.0, hi=0.6)
    ib, pr = litho_lib.litho_resist(torch.from_numpy(img.astype(np.float32)).to(cuda), pixel, sigma, 0.3)
    ib = ib.cpu().numpy()
    pr = pr.cpu().numpy()
    for p in range(planes):
        ref = OR.blur(img[p].astype(np.float32).astype(np.float64), sigma, pixel)
        assert np.abs(ib[p] - ref).max() <= 1e-6
        sure = np.abs(ref - 0.3) > 1e-5
        assert np.array_equal(pr[p][sure], (ref[sure] >= 0.3).astype(np.uint8))
        assert np.array_equal(pr[p], (ib[p] >= np.float32(0.3)).astype(np.uint8))


def test_aerial_plus_resist_edge_placement_config1(litho_lib, cuda):
    """256^2 annular K=8 clip: GPU contours within 0.1 nm of the oracle's."""
    n, pixel, k = 256, 8.0, 8
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [0.0], k)
    masks = np.stack([synth.random_rect_mask(n, seed=1234 + i) for i in range(4)])
    import torch
    kern = litho_lib.litho_upload_kernels(n, pixel, lam, phi)
    img = litho_lib.litho_aerial(kern, torch.from_numpy(masks).to(cuda))
    ib, _ = litho_lib.litho_resist(img, pixel, 10.0, 0.3)
    ib = ib.cpu().numpy()
    for i in range(4):
        ref_img = OI.socs_image(masks[i].astype(np.float64), lam[0], phi[0])
        ref = OR.blur(ref_img, 10.0, pixel)
        epe = OR.edge_placement_difference(ref, ib[i, 0].astype(np.float64), 0.3, pixel)
        assert epe <= 0.1, epe
        assert len(OR.crossings(ref, 0.3, 1)[0]) > 50
