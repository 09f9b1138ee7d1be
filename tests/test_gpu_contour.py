"""GPU contours and edge-placement error (section II.D, Eqs. (6)-(8)) against the oracle.

Contours: the inside / saddle decisions are integer results of FP32
comparisons, taken in FP32 on both sides on the same float32 input, so the
segment lists (count, cells, order, start and end edges) must be identical;
the interpolated end points agree to 1e-5 px plus the FP32 rounding of an
absolute coordinate.  EPE: per point |dEPE| <=
1e-3 nm + 1e-4 |EPE| (FP32 interpolation and gradient); Eq. (8)'s branch is
compared wherever the on-focus EPE is farther than that bound from a
tolerance.
"""
import numpy as np
import pytest

import synth
from oracle import contour as OC
from oracle import imaging as OI
from oracle import resist as OR
from tests.gpu_util import DUV_ANNULAR, oracle_kernel_set

pytestmark = pytest.mark.gpu


def _blobs(n, seed, count=40):
    st = synth.Stream(seed)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    f = np.zeros((n, n))
    for cx, cy, r in zip(st.uniform(count) * n, st.uniform(count) * n, 1.5 + 0.04 * n * st.uniform(count)):
        dx = (x - cx + n / 2) % n - n / 2
        dy = (y - cy + n / 2) % n - n / 2
        f += np.exp(-(dx * dx + dy * dy) / (2 * r * r))
    return f.astype(np.float32)


def _compare(seg, cell, start, planes, thr, rows=None):
    """seg/cell: GPU output (numpy); planes: float32 [P][n][n] given to both sides."""
    n = planes.shape[-1]
    for p in range(planes.shape[0]):
        ref = OC.marching_squares(planes[p], thr, rows=rows)
        g_seg = seg[start[p]:start[p + 1]]
        g_cell = cell[start[p]:start[p + 1]]
        if rows is not None:
            keep = np.isin(g_cell // n, list(rows))
            g_seg, g_cell = g_seg[keep], g_cell[keep]
        assert len(g_cell) == len(ref), (p, len(g_cell), len(ref))
        assert np.array_equal(g_cell, np.array([r[0] for r in ref], dtype=np.int32))
        want = np.array([r[1:5] for r in ref], dtype=np.float64).reshape(-1, 4)
        # 1e-5 px, plus the FP32 rounding of an absolute coordinate (two ulps of up to n)
        assert np.all(np.abs(g_seg.astype(np.float64) - want) <= 1e-5 + 2.5e-7 * np.abs(want))


def test_contours_match_oracle_on_images_blobs_and_noise(litho_lib, cuda):
    import torch
    L = litho_lib
    n, pixel, thr = 256, 8.0, 0.3
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [0.0], 8)
    mask = synth.random_rect_mask(n, seed=71, count=50).astype(np.float64)
    img = OR.blur(OI.socs_image(mask, lam[0], phi[0]), 10.0, pixel)
    noise = synth.random_field((n, n), seed=9, lo=0.0, hi=0.6)          # saddles everywhere
    planes = np.stack([img, _blobs(n, 5) * 0.6, noise, np.full((n, n), 0.2)]).astype(np.float32)
    seg, cell, start = L.litho_contours(torch.from_numpy(planes).to(cuda), thr)
    seg, cell = seg.cpu().numpy(), cell.cpu().numpy()
    assert start[3] == start[4]                       # constant plane: no segment
    assert start[4] - start[3] == 0 and start[3] > start[2] > start[1] > 0
    _compare(seg, cell, start, planes, thr)


@pytest.mark.parametrize("n", [96, 64])
def test_contours_rows_not_a_multiple_of_128(litho_lib, cuda, n):
    """Row lengths outside the vectorised kernels' (one cell per thread in chunks)."""
    import torch
    planes = np.stack([_blobs(n, 31), synth.random_field((n, n), seed=32, lo=0.0, hi=1.0).astype(np.float32)])
    seg, cell, start = litho_lib.litho_contours(torch.from_numpy(planes).to(cuda), 0.5)
    _compare(seg.cpu().numpy(), cell.cpu().numpy(), start, planes, 0.5)


def test_contours_capacity_and_chaining(litho_lib, cuda):
    import torch
    L = litho_lib
    n, thr = 128, 0.5
    planes = np.stack([_blobs(n, 11), _blobs(n, 12)])
    full, cells, start = L.litho_contours(torch.from_numpy(planes).to(cuda), thr)
    full = full.cpu().numpy()
    total = int(start[-1])
    # a smaller buffer keeps the first segments and still reports the total
    part, _, start2 = L.litho_contours(torch.from_numpy(planes).to(cuda), thr, capacity=total - 7)
    assert int(start2[-1]) == total and np.array_equal(part.cpu().numpy(), full[:total - 7])
    # closed contours: every end point is the start of exactly one segment of its plane
    for p in range(2):
        s = full[start[p]:start[p + 1]].astype(np.float64) % n
        starts = {(round(a, 4), round(b, 4)) for a, b in s[:, :2]}
        assert len(starts) == len(s)
        assert all((round(a, 4), round(b, 4)) in starts for a, b in s[:, 2:])


def test_contours_full_size_sampled_rows(litho_lib, cuda):
    """2048^2 planes (the headline size): every segment of sampled cell rows."""
    import torch
    L = litho_lib
    n, thr = 2048, 0.5
    planes = np.stack([_blobs(n, 21, count=400), _blobs(n, 22, count=400)])
    seg, cell, start = L.litho_contours(torch.from_numpy(planes).to(cuda), thr)
    rows = sorted(set(synth.Stream(5).integers(0, n - 1, 6).tolist()) | {0, n - 1})
    _compare(seg.cpu().numpy(), cell.cpu().numpy(), start, planes, thr, rows=rows)


def test_epe_and_through_focus_match_oracle(litho_lib, cuda):
    import torch
    L = litho_lib
    n, pixel, thr, sigma = 256, 8.0, 0.3, 10.0
    focus = [0.0, 60.0, -60.0]
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, focus, 8)
    target = synth.random_rect_mask(n, seed=81, count=50)
    planes = np.stack([OR.blur(OI.socs_image(target.astype(np.float64), lam[f], phi[f]), sigma, pixel)
                       for f in range(3)]).astype(np.float32)
    pts = synth.edge_sites(target).astype(np.float32)
    assert len(pts) > 500
    epe = L.litho_epe(torch.from_numpy(planes).to(cuda), torch.from_numpy(pts).to(cuda), pixel, thr)
    ref = np.stack([OC.epe(planes[f], pts.astype(np.float64), thr, pixel) for f in range(3)])
    got = epe.cpu().numpy().astype(np.float64)
    bound = 1e-3 + 1e-4 * np.abs(ref)
    assert np.all(np.abs(got - ref) <= bound)
    tol_neg, tol_pos = -2.0, 1.5
    avg, eff = L.litho_epe_through_focus(epe, 0, 1, 2, tol_neg, tol_pos)
    ravg, reff = OC.epe_through_focus(ref, 0, 1, 2, tol_neg, tol_pos)
    assert np.all(np.abs(avg.cpu().numpy() - ravg) <= 1e-3 + 1e-4 * np.abs(ravg))
    clear = (np.abs(ref[0] - tol_neg) > 2 * bound[0]) & (np.abs(ref[0] - tol_pos) > 2 * bound[0])
    assert clear.sum() > 0.9 * len(pts)
    e = eff.cpu().numpy()
    assert np.all(np.abs(e[clear] - reff[clear]) <= 2e-3 + 1e-4 * np.abs(reff[clear]))


def test_epe_flat_image_is_nan_and_errors(litho_lib, cuda):
    import torch
    L = litho_lib
    flat = torch.full((1, 64, 64), 0.5, dtype=torch.float32, device=cuda)
    pts = torch.tensor([[3.5, 7.0], [10.0, 20.5]], dtype=torch.float32, device=cuda)
    assert torch.isnan(L.litho_epe(flat, pts, 8.0, 0.3)).all()
    e = torch.zeros((2, 4), dtype=torch.float32, device=cuda)
    with pytest.raises(L.LithoError) as err:
        L.litho_epe_through_focus(e, 0, 1, 2, -1.0, 1.0)           # plane 2 does not exist
    assert err.value.status == L.EINVAL


def test_epe_batch_equals_per_clip_calls(litho_lib, cuda):
    """One launch over several clips' points (one clip with no points) gives
    each clip's EPE bit-identical to litho_epe on that clip alone."""
    import torch
    L = litho_lib
    n, pixel, thr, planes = 128, 8.0, 0.5, 3
    imgs = np.stack([np.stack([_blobs(n, 40 + 3 * c + p, count=12) for p in range(planes)]) for c in range(4)])
    pts = [synth.edge_sites(imgs[c, 0] >= thr).astype(np.float32) for c in range(4)]
    pts[2] = np.zeros((0, 2), np.float32)
    start = np.concatenate([[0], np.cumsum([len(p) for p in pts])]).astype(np.int64)
    d_img = torch.from_numpy(imgs).to(cuda)
    d_pts = torch.from_numpy(np.concatenate(pts)).to(cuda)
    got = L.litho_epe_batch(d_img, d_pts, torch.from_numpy(start).to(cuda), pixel, thr).cpu().numpy()
    for c in range(4):
        if len(pts[c]) == 0:
            continue
        one = L.litho_epe(d_img[c], torch.from_numpy(pts[c]).to(cuda), pixel, thr).cpu().numpy()
        np.testing.assert_array_equal(got[:, start[c]:start[c + 1]], one)
