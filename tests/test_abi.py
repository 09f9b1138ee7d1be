"""Host-side checks of liblitho.so (no GPU): exported symbols, argument
validation, and the FP64 kernel builder against the oracle's TCC eigen-kernels
(Eqs. (2)-(3))."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import imaging as OI
from oracle import optics as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "litho.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(litho_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(litho_lib):
    names = _declared()
    assert len(names) >= 20
    L = litho_lib.lib()
    for name in names:
        assert hasattr(L, name), name
        assert name in litho_lib._SIGS, f"binding lacks {name}"
    assert "sm_103a" in litho_lib.litho_version()


def test_argument_validation_without_gpu(litho_lib):
    L = litho_lib
    o = L.make_optics(kind="annular")
    with pytest.raises(L.LithoError) as e:
        L.litho_tcc_kernels_host(o, 100, 8.0, 0.0, 8)
    assert e.value.status == L.EINVAL
    bad = L.make_optics(kind="annular", src_grid=20)
    with pytest.raises(L.LithoError) as e:
        L.litho_tcc_kernels_host(bad, 256, 8.0, 0.0, 8)
    assert e.value.status == L.EINVAL and "odd" in str(e.value)
    with pytest.raises(L.LithoError):
        L.litho_tcc_kernels_host(L.make_optics(na=1.6, n_medium=1.44), 256, 8.0, 0.0, 8)


def _oracle_optics(kind, grid):
    if kind == "annular":
        return O.Optics(193.0, 1.35, 1.44, O.ANNULAR, grid, 0.6, 0.9)
    return O.Optics(193.0, 1.35, 1.44, O.QUADRUPOLE, grid, pole_sigma=0.8, pole_radius=0.1)


@pytest.mark.parametrize("kind,grid,n,z,k", [("annular", 21, 256, 0.0, 8), ("quadrupole", 41, 128, 50.0, 24),
                                              ("annular", 21, 64, -30.0, 144)])
def test_host_kernel_builder_matches_oracle(litho_lib, kind, grid, n, z, k):
    L = litho_lib
    lam, phi, info = L.litho_tcc_kernels_host(L.make_optics(kind=kind, src_grid=grid), n, 8.0, z, k)
    oo = _oracle_optics(kind, grid)
    c = O.crop_size(oo, n, 8.0)
    assert phi.shape[-1] == c
    lam_o, phi_o, lam_all = O.socs_kernels(oo, n, 8.0, z, k, c)
    assert np.allclose(lam, lam_o, rtol=1e-10, atol=1e-10 * lam_o[0])
    assert abs(info["trace"] - O.tcc_trace(oo, n, 8.0, c)) < 1e-9 * info["trace"]
    assert info["rank"] == int((lam_all > 1e-12 * lam_all[0]).sum())
    # unit norm, orthogonal
    p = phi.reshape(k, -1)
    r = min(k, info["rank"])
    assert np.abs(p[:r].conj() @ p[:r].T - np.eye(r)).max() < 1e-9
    # images from library kernels equal images from oracle kernels when the cut
    # at k closes its degenerate cluster (the eigenbasis inside a cluster is arbitrary)
    gap = lam_all[k - 1] - (lam_all[k] if k < len(lam_all) else 0.0)
    assert abs(info["gap"] - gap) < 1e-9 * lam_all[0]
    if gap > 1e-9 * lam_all[0]:
        m = synth.random_rect_mask(n, seed=13, count=max(10, n // 8)).astype(np.float64)
        a = OI.socs_image(m, lam, phi)
        b = OI.socs_image(m, lam_o, phi_o)
        assert np.abs(a - b).max() < 1e-10
