"""Failure detection on the GPU without a GPU fault.

Every device-side wait of the tensor-core pipeline is bounded; past its limit
it records an error code that the host reads (litho_check_device ->
LITHO_ETIMEOUT) and the kernel returns, so the context stays usable.  The
self-test kernel waits on a barrier that nothing ever signals, with a short
limit, to make that wait run out on purpose.
"""
import numpy as np
import pytest

import synth
from oracle import imaging as OI
from tests.gpu_util import DUV_ANNULAR, oracle_kernel_set

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_device_stays_usable(litho_lib, cuda):
    import torch
    L = litho_lib
    n, pixel = 128, 8.0
    lam, phi = oracle_kernel_set(DUV_ANNULAR, n, pixel, [0.0], 6)
    kern = L.litho_upload_kernels(n, pixel, lam, phi)
    assert L.litho_selftest_wait_limit(kern, 50.0) == L.ETIMEOUT
    assert "gave up" in L.litho_last_error()
    L.litho_check_device(kern)  # flag was cleared: no error now
    m = synth.random_rect_mask(n, seed=8, count=20)
    for prec in ("fft32", "fp16x3"):
        img = L.litho_aerial(kern, torch.from_numpy(m[None]).to(cuda), precision=prec).cpu().numpy()[0, 0]
        assert np.abs(img - OI.socs_image(m.astype(np.float64), lam[0], phi[0])).max() <= 1e-5
    L.litho_check_device(kern)
