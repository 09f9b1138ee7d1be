"""GPU parity of the ILT loss and adjoint gradient against the FP64 oracle.

Bar: relative gradient error at most 1e-4 (over all pixels, and per pixel on
64 seeded pixels against the largest gradient), the loss to FP32 accuracy,
and an FP32 finite-difference sanity check at 1e-2.
"""
import numpy as np
import pytest

import synth
from oracle import ilt as OL
from tests.gpu_util import DUV_ANNULAR, oracle_kernel_set

pytestmark = pytest.mark.gpu

PARAMS = dict(dose=1.0, mask_steep=4.0, resist_steep=25.0, threshold=0.3, sigma_nm=10.0)


def _oracle(theta, target, lam, phi, pixel):
    kern = [(lam[f], phi[f]) for f in range(lam.shape[0])]
    return OL.loss_and_grad(theta.astype(np.float64), target.astype(np.float64), kern, dose=PARAMS["dose"],
                            alpha=PARAMS["mask_steep"], beta=PARAMS["resist_steep"], thr=PARAMS["threshold"],
                            sigma_nm=PARAMS["sigma_nm"], pixel_nm=pixel)


def _gpu(litho_lib, cuda, kern, thetas, targets, workspace=None, precision="fft32"):
    import torch
    th = torch.from_numpy(np.ascontiguousarray(thetas, dtype=np.float32)).to(cuda)
    tg = torch.from_numpy(np.ascontiguousarray(targets, dtype=np.float32)).to(cuda)
    g, loss = litho_lib.litho_ilt_grad(kern, th, tg, workspace=workspace, precision=precision, **PARAMS)
    return g.cpu().numpy().astype(np.float64), loss


def _check(g, ref, pts):
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    gmax = np.abs(ref).max()
    per = max(abs(g[y, x] - ref[y, x]) for y, x in pts) / gmax
    return rel, per


@pytest.mark.parametrize("precision", ["fft32", "fft32/coarse"])
@pytest.mark.parametrize("n,pixel,k,focus,b", [(128, 8.0, 6, [-60.0, -30.0, 0.0, 30.0, 60.0], 2),
                                               (256, 8.0, 8, [0.0, 40.0], 1)])
def test_ilt_gradient_matches_oracle(litho_lib, cuda, n, pixel, k, focus, b, precision):
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, focus, k)
    kern = litho_lib.litho_upload_kernels(n, pixel, lam, phi)
    if precision.endswith("/coarse"):
        assert 0 < kern.grid(precision) < n  # the coarse grid is in use
    clips = [synth.ilt_clip(n, pixel, seed=500 + i) for i in range(b)]
    thetas = np.stack([c[0] for c in clips])
    targets = np.stack([c[1] for c in clips])
    g, loss = _gpu(litho_lib, cuda, kern, thetas, targets, precision=precision)
    st = synth.Stream(64)
    pts = list(zip(st.integers(0, n - 1, 64), st.integers(0, n - 1, 64)))
    for i in range(b):
        lo, ref = _oracle(thetas[i], targets[i], lam, phi, pixel)
        assert abs(loss[i] - lo) <= 1e-5 * lo, (loss[i], lo)
        rel, per = _check(g[i], ref, pts)
        print(f"n={n} clip {i}: loss {loss[i]:.6f} vs {lo:.6f}; grad rel l2 {rel:.2e}, per-pixel {per:.2e}")
        assert rel <= 1e-4 and per <= 1e-4


@pytest.mark.parametrize("precision", ["fft32", "fft32/coarse"])
def test_ilt_recompute_mode_equals_full_mode(litho_lib, cuda, precision):
    import torch
    n, pixel = 128, 8.0
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [-40.0, 0.0, 40.0], 6)
    kern = litho_lib.litho_upload_kernels(n, pixel, lam, phi)
    theta, target = synth.ilt_clip(n, pixel, seed=9)
    full, mn = litho_lib.litho_ilt_workspace_size(kern, 1)
    assert mn < full
    g_full, l_full = _gpu(litho_lib, cuda, kern, theta[None], target[None], precision=precision)
    ws = torch.empty(mn, dtype=torch.uint8, device=cuda)
    g_min, l_min = _gpu(litho_lib, cuda, kern, theta[None], target[None], workspace=ws, precision=precision)
    assert abs(l_full[0] - l_min[0]) <= 1e-12 * l_full[0]
    assert np.abs(g_full - g_min).max() <= 1e-6 * np.abs(g_full).max()
    small = torch.empty(mn - 256, dtype=torch.uint8, device=cuda)
    with pytest.raises(litho_lib.LithoError) as e:
        _gpu(litho_lib, cuda, kern, theta[None], target[None], workspace=small, precision=precision)
    assert e.value.status == litho_lib.ENOMEM


@pytest.mark.parametrize("precision", ["fft32", "fft32/coarse"])
def test_ilt_clip_groups_equal_clips_alone(litho_lib, cuda, precision):
    """One call images its clips in groups (a launch covers every clip of a
    group); each clip's gradient is bit-identical and its FP64 loss equal to
    the same clip run alone."""
    n, pixel, b = 128, 8.0, 3
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [-40.0, 0.0, 40.0], 6)
    kern = litho_lib.litho_upload_kernels(n, pixel, lam, phi)
    clips = [synth.ilt_clip(n, pixel, seed=800 + i) for i in range(b)]
    thetas = np.stack([c[0] for c in clips])
    targets = np.stack([c[1] for c in clips])
    g_all, l_all = _gpu(litho_lib, cuda, kern, thetas, targets, precision=precision)
    for i in range(b):
        g_i, l_i = _gpu(litho_lib, cuda, kern, thetas[i:i + 1], targets[i:i + 1], precision=precision)
        assert np.array_equal(g_all[i], g_i[0])
        assert l_all[i] == l_i[0]


def test_ilt_coarse_grid_equals_full_grid(litho_lib, cuda):
    """The coarse-grid adjoint is exact (no product frequency aliases into the
    field band on nc >= 2C), so it agrees with the full-grid gradient to FP32
    rounding: 1e-5 relative, ten times inside the oracle bar."""
    n, pixel = 256, 8.0
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [-50.0, 0.0, 50.0], 8)
    kern = litho_lib.litho_upload_kernels(n, pixel, lam, phi)
    assert 0 < kern.grid("fft32/coarse") < n
    clips = [synth.ilt_clip(n, pixel, seed=700 + i) for i in range(2)]
    thetas = np.stack([c[0] for c in clips])
    targets = np.stack([c[1] for c in clips])
    g_f, l_f = _gpu(litho_lib, cuda, kern, thetas, targets)
    g_c, l_c = _gpu(litho_lib, cuda, kern, thetas, targets, precision="fft32/coarse")
    for i in range(2):
        assert abs(l_c[i] - l_f[i]) <= 1e-5 * l_f[i]
        rel = np.linalg.norm(g_c[i] - g_f[i]) / np.linalg.norm(g_f[i])
        print(f"clip {i}: coarse vs full grid, loss {l_c[i]:.6f} / {l_f[i]:.6f}, grad rel l2 {rel:.2e}")
        assert rel <= 1e-5


def test_ilt_fp32_finite_differences(litho_lib, cuda):
    """Sanity: central FP32 differences of the GPU loss (h = 1e-2) agree to 1e-2."""
    n, pixel = 128, 8.0
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [0.0], 6)
    kern = litho_lib.litho_upload_kernels(n, pixel, lam, phi)
    theta, target = synth.ilt_clip(n, pixel, seed=21)
    g, _ = _gpu(litho_lib, cuda, kern, theta[None], target[None])
    flat = np.argsort(np.abs(g[0]).ravel())[-6:]
    h = 1e-2
    for f in flat:
        y, x = divmod(int(f), n)
        tp = theta.copy()
        tp[y, x] += h
        tm = theta.copy()
        tm[y, x] -= h
        _, lp = _gpu(litho_lib, cuda, kern, tp[None], target[None])
        _, lm = _gpu(litho_lib, cuda, kern, tm[None], target[None])
        fd = (lp[0] - lm[0]) / (2 * h)
        assert abs(fd - g[0, y, x]) <= 1e-2 * np.abs(g).max(), (fd, g[0, y, x])


_ORACLE_1024 = {}


@pytest.mark.parametrize("precision", ["fft32", "fft32/coarse"])
def test_ilt_full_size_1024_k16_five_focus(litho_lib, cuda, precision):
    """The benchmark's clip size and optics, on both grids (the coarse grid's
    1024-point rows keep dL/dI in registers between their two transforms)."""
    n, pixel, k = 1024, 8.0, 16
    focus = [-60.0, -30.0, 0.0, 30.0, 60.0]
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, focus, k)
    kern = litho_lib.litho_upload_kernels(n, pixel, lam, phi)
    if precision.endswith("/coarse"):
        assert 0 < kern.grid(precision) < n
    theta, target = synth.ilt_clip(n, pixel, seed=4000)
    g, loss = _gpu(litho_lib, cuda, kern, theta[None], target[None], precision=precision)
    if not _ORACLE_1024:
        _ORACLE_1024["r"] = _oracle(theta, target, lam, phi, pixel)
    lo, ref = _ORACLE_1024["r"]
    st = synth.Stream(65)
    pts = list(zip(st.integers(0, n - 1, 64), st.integers(0, n - 1, 64)))
    rel, per = _check(g[0], ref, pts)
    print(f"1024 {precision}: loss {loss[0]:.4f} vs {lo:.4f}; grad rel l2 {rel:.2e}, per-pixel {per:.2e}")
    assert abs(loss[0] - lo) <= 1e-5 * lo
    assert rel <= 1e-4 and per <= 1e-4


def test_autograd_function(litho_lib, cuda):
    import torch
    from paper_2602_15036_gb300.autograd import ilt_loss
    n, pixel = 128, 8.0
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [0.0, 50.0], 5)
    kern = litho_lib.litho_upload_kernels(n, pixel, lam, phi)
    clips = [synth.ilt_clip(n, pixel, seed=70 + i) for i in range(2)]
    th = torch.from_numpy(np.stack([c[0] for c in clips])).to(cuda).requires_grad_(True)
    tg = torch.from_numpy(np.stack([c[1] for c in clips])).to(cuda)
    loss = ilt_loss(th, tg, kern)
    (2.0 * loss[0] + 3.0 * loss[1]).backward()
    g, _ = litho_lib.litho_ilt_grad(kern, th.detach(), tg, **PARAMS)
    w = torch.tensor([2.0, 3.0], device=cuda).view(2, 1, 1)
    assert torch.allclose(th.grad, g * w, rtol=0, atol=1e-6 * g.abs().max().item())


def test_ilt_run_resumes_from_checkpoint(litho_lib, cuda, tmp_path):
    """A gradient-descent run through litho_ilt_grad stopped after 3 steps and
    resumed from its checkpoint files equals the run that never stopped."""
    import torch
    from paper_2602_15036_gb300.iltrun import IltRun
    n, pixel = 128, 8.0
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [-40.0, 0.0, 40.0], 6)
    kern = litho_lib.litho_upload_kernels(n, pixel, lam, phi)
    clips = [synth.ilt_clip(n, pixel, seed=900 + i) for i in range(2)]
    theta = torch.from_numpy(np.stack([c[0] for c in clips])).to(cuda)
    target = torch.from_numpy(np.stack([c[1] for c in clips])).to(cuda)
    fn = IltRun.litho_grad_fn(kern, precision="fft32/coarse", **PARAMS)
    full = IltRun(theta.clone(), target, fn)
    full.run(6)
    prefix = str(tmp_path / "ilt")
    IltRun(theta.clone(), target, fn).run(3, checkpoint_prefix=prefix)
    again = IltRun.load(prefix, target, fn, device=cuda)
    again.run(3)
    assert torch.equal(again.theta, full.theta) and again.losses == full.losses
    assert full.losses[-1] < full.losses[0]
