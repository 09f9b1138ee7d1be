"""litho_aerial_noalloc: the aerial image for callers that cannot allocate.

Some callers cannot allocate device memory at call time: an application that
owns every device allocation through its own pool, or a latency-critical loop
that cannot take the device-wide stall cudaMalloc/cudaFree may cause.  For
them the library keeps a fixed scratch array and this entry point takes only
the mask and the output.  Its results must equal the workspace-based
litho_aerial (FP32 path) within the aerial tolerance of the other tests,
call after call, since each call reuses the same array.

This file is named to be collected last, so a failure here leaves every other
test already run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synth
from oracle import imaging as OI
from tests.gpu_util import DUV_ANNULAR, DUV_QUAD41, oracle_kernel_set

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


def test_noalloc_matches_workspace_path_on_consecutive_calls(litho_lib, cuda):
    import torch
    L = litho_lib
    n, pixel = 256, 8.0
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [0.0, 40.0], 8)
    kern = L.litho_upload_kernels(n, pixel, lam, phi)
    for call, seed in enumerate((11, 29)):           # two calls in a row, different masks
        masks = np.stack([synth.random_rect_mask(n, seed=seed + i) for i in range(3)])
        m = torch.from_numpy(masks).to(cuda)
        ref = L.litho_aerial(kern, m, dose=1.2)
        out = torch.full_like(ref, float("nan"))
        L.litho_aerial_noalloc(kern, m, out, dose=1.2)
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item()
        assert err <= TOL_FP32, (call, err)
        got = out.cpu().numpy().astype(np.float64)
        for i in range(len(masks)):                   # and against the FP64 oracle itself
            for f in range(lam.shape[0]):
                want = OI.socs_image(masks[i].astype(np.float64), lam[f], phi[f], 1.2)
                e = np.abs(got[i, f] - want).max()
                assert e <= TOL_FP32, (call, i, f, e)


def test_noalloc_rejects_sizes_beyond_its_scratch(litho_lib, cuda):
    import torch
    L = litho_lib
    n, pixel = 1024, 8.0
    lam, phi = oracle_kernel_set(DUV_QUAD41, n, pixel, [0.0], 24)   # 8*1024*224*25 bytes > 32 MiB
    kern = L.litho_upload_kernels(n, pixel, lam, phi)
    m = torch.zeros((1, n, n), dtype=torch.float32, device=cuda)
    out = torch.empty((1, 1, n, n), dtype=torch.float32, device=cuda)
    with pytest.raises(L.LithoError) as e:
        L.litho_aerial_noalloc(kern, m, out)
    assert e.value.status == L.EINVAL
    assert "fixed scratch array" in str(e.value)
    assert L.litho_aerial_noalloc_max_bytes() == 32 << 20


def test_noalloc_checks_its_arguments(litho_lib, cuda):
    import torch
    L = litho_lib
    n, pixel = 64, 8.0
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [0.0, 40.0], 4)
    kern = L.litho_upload_kernels(n, pixel, lam, phi)
    m = torch.zeros((2, n, n), dtype=torch.float32, device=cuda)
    out = torch.empty((2, 2, n, n), dtype=torch.float32, device=cuda)
    with pytest.raises(L.LithoError) as e:                       # a NaN dose is refused, as by litho_aerial
        L.litho_aerial_noalloc(kern, m, out, dose=float("nan"))
    assert e.value.status == L.EINVAL
    with pytest.raises(ValueError):                              # an output missing the focus axis
        L.litho_aerial_noalloc(kern, m, torch.empty((2, n, n), dtype=torch.float32, device=cuda))
    with pytest.raises(ValueError):
        L.litho_aerial_noalloc(kern, m.double(), out)
