"""Out-of-bounds write checks through the C ABI (compute-sanitizer is not
available here): every output and workspace sits inside a larger buffer whose
guard bytes before and after are filled with a pattern, and the guards must be
intact after the call.  Sizes span several tiles, ragged group tails and the
coarse-grid, grouped and tensor-core paths.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

PAD = 4096          # guard bytes on each side (keeps the 256-byte alignment of the view)
PATTERN = 0xA5


class Guarded:
    """A view of `nbytes` inside a buffer with PAD guard bytes on each side."""

    def __init__(self, cuda, shape, dtype):
        import torch
        self.nbytes = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        self.raw = torch.full((PAD + self.nbytes + PAD,), PATTERN, dtype=torch.uint8, device=cuda)
        self.view = self.raw[PAD:PAD + self.nbytes].view(dtype).view(*shape)

    def intact(self) -> bool:
        import torch
        torch.cuda.synchronize()
        head = self.raw[:PAD]
        tail = self.raw[PAD + self.nbytes:]
        return bool((head == PATTERN).all().item()) and bool((tail == PATTERN).all().item())


def _kernels(L, n, focus, k, kind="quadrupole"):
    optics = (L.make_optics(kind="quadrupole", src_grid=21, pole_sigma=0.8, pole_radius=0.1) if kind == "quadrupole"
              else L.make_optics(kind="annular", src_grid=21, sigma_in=0.6, sigma_out=0.9))
    return L.litho_make_kernels(optics, n, 8.0, focus, k)


def _masks(cuda, n, b, seed=5):
    import torch
    return torch.from_numpy(np.stack([synth.manhattan_mask(n, seed=seed + i) for i in range(b)])).to(cuda)


@pytest.mark.parametrize("precision,n,b", [("fft32", 256, 3), ("fft32/coarse", 256, 3), ("fp16x3/coarse", 512, 5),
                                           ("fp16/coarse", 512, 2)])
def test_aerial_and_resist_stay_in_bounds(litho_lib, cuda, precision, n, b):
    import torch
    L = litho_lib
    kern = _kernels(L, n, [-50.0, 0.0, 50.0], 12)
    m = _masks(cuda, n, b)
    shape = (b, kern.n_focus, n, n)
    out = Guarded(cuda, shape, torch.float32)
    ws = Guarded(cuda, (L.litho_aerial_workspace_size(kern, b, precision),), torch.uint8)
    L.litho_aerial(kern, m, precision=precision, out=out.view, workspace=ws.view)
    assert out.intact() and ws.intact()
    img, ib, pr = Guarded(cuda, shape, torch.float32), Guarded(cuda, shape, torch.float32), Guarded(cuda, shape,
                                                                                                   torch.uint8)
    ws2 = Guarded(cuda, (L.litho_aerial_workspace_size(kern, b, precision),), torch.uint8)
    L.litho_aerial_resist(kern, m, precision=precision, out=img.view, iblur=ib.view, printed=pr.view,
                          workspace=ws2.view)
    assert img.intact() and ib.intact() and pr.intact() and ws2.intact()
    assert torch.isfinite(img.view).all() and torch.isfinite(ib.view).all()


def test_direct_resist_stays_in_bounds(litho_lib, cuda):
    import torch
    L = litho_lib
    n, planes = 384, 3
    x = torch.rand((planes, n, n), device=cuda)
    ib, pr = Guarded(cuda, (planes, n, n), torch.float32), Guarded(cuda, (planes, n, n), torch.uint8)
    L.litho_resist(x, 8.0, sigma_nm=10.0, threshold=0.3, iblur=ib.view, printed=pr.view)
    assert ib.intact() and pr.intact()


@pytest.mark.parametrize("n", [256, 200])
def test_contours_and_epe_stay_in_bounds(litho_lib, cuda, n):
    import torch
    L = litho_lib
    planes = 3
    img = torch.from_numpy(np.stack([synth.blob_field(n, 8.0, seed=30 + p) for p in range(planes)]).astype(
        np.float32)).to(cuda)
    _, _, st = L.litho_contours(img, 0.5, with_cells=False)
    total = int(st[-1])
    seg = Guarded(cuda, (total, 4), torch.float32)          # capacity exactly the segment count
    cell = Guarded(cuda, (total,), torch.int32)
    starts = Guarded(cuda, (planes + 1,), torch.int64)
    ws = Guarded(cuda, (L.contours_workspace_size(planes, n),), torch.uint8)
    L.contours_into(img, planes, n, 0.5, seg.view, cell.view, total, starts.view, ws.view)
    assert seg.intact() and cell.intact() and starts.intact() and ws.intact()
    assert int(starts.view[-1]) == total
    pts = torch.from_numpy(synth.edge_sites((synth.blob_field(n, 8.0, seed=31) >= 0.5)).astype(np.float32)).to(cuda)
    epe = Guarded(cuda, (planes, pts.shape[0]), torch.float32)
    L.litho_epe(img, pts, 8.0, 0.5, out=epe.view)
    assert epe.intact()


def test_raster_stays_in_bounds(litho_lib, cuda):
    import torch
    L = litho_lib
    n, b = 256, 3
    rects = [synth.manhattan_rects(n, seed=40 + i)[0] for i in range(b)]
    flat = np.concatenate([np.stack([r[:, 0], r[:, 1], r[:, 0] + r[:, 2], r[:, 1] + r[:, 3]], axis=1) + 0.25
                           for r in rects]).astype(np.float32)
    counts = [len(r) for r in rects]
    start = torch.from_numpy(np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)).to(cuda)
    d_rects = torch.from_numpy(flat).to(cuda)
    mask = Guarded(cuda, (b, n, n), torch.float32)
    ws = Guarded(cuda, (L.rasterize_workspace_size(b, n, max(counts), 16),), torch.uint8)
    L.rasterize_into(d_rects, start, b, max(counts), 16, n, mask.view, ws.view)
    assert mask.intact() and ws.intact()
    assert torch.isfinite(mask.view).all()


@pytest.mark.parametrize("precision", ["fft32", "fft32/coarse"])
def test_ilt_and_ai_inputs_stay_in_bounds(litho_lib, cuda, precision):
    import torch
    L = litho_lib
    n, b = 256, 3
    kern = _kernels(L, n, [-40.0, 0.0, 40.0], 8, kind="annular")
    clips = [synth.ilt_clip(n, 8.0, seed=60 + i) for i in range(b)]
    theta = torch.from_numpy(np.stack([c[0] for c in clips])).to(cuda)
    target = torch.from_numpy(np.stack([c[1] for c in clips])).to(cuda)
    full, mn = L.litho_ilt_workspace_size(kern, b)
    for size in (full, mn):                                   # grouped, and one plane of one clip at a time
        grad = Guarded(cuda, (b, n, n), torch.float32)
        ws = Guarded(cuda, (size,), torch.uint8)
        L.litho_ilt_grad(kern, theta, target, precision=precision, grad=grad.view, workspace=ws.view)
        assert grad.intact() and ws.intact()
    x = Guarded(cuda, (b, 3, n, n), torch.float32)
    ws = Guarded(cuda, (L.litho_ai_inputs_workspace_size(kern, b),), torch.uint8)
    L.litho_ai_inputs(kern, target, focus=1, precision=precision, out=x.view, workspace=ws.view)
    assert x.intact() and ws.intact()
