"""Helpers shared by the GPU parity tests: oracle kernel sets and optics presets.

Kernels fed to the GPU in parity tests are built by the oracle (FP64) and
uploaded through litho_upload_kernels, so the GPU and the oracle image with the
same kernel data; the library's own builder is checked separately.
"""
import numpy as np

from oracle import optics as O

DUV_ANNULAR = dict(kind="annular", src_grid=21, sigma_in=0.6, sigma_out=0.9)
DUV_QUAD41 = dict(kind="quadrupole", src_grid=41, pole_sigma=0.8, pole_radius=0.1)
DUV_QUAD21 = dict(kind="quadrupole", src_grid=21, pole_sigma=0.8, pole_radius=0.1)


def oracle_optics(preset, wavelength=193.0, na=1.35, n_medium=1.44):
    if preset["kind"] == "annular":
        return O.Optics(wavelength, na, n_medium, O.ANNULAR, preset["src_grid"], preset["sigma_in"],
                        preset["sigma_out"])
    return O.Optics(wavelength, na, n_medium, O.QUADRUPOLE, preset["src_grid"], pole_sigma=preset["pole_sigma"],
                    pole_radius=preset["pole_radius"])


def oracle_kernel_set(preset, n, pixel, focus, k, **opt_kw):
    """lam [F][K], phi [F][K][C][C] from the oracle (FP64)."""
    oo = oracle_optics(preset, **opt_kw)
    c = O.crop_size(oo, n, pixel)
    lams, phis = [], []
    for z in focus:
        lam, phi, _ = O.socs_kernels(oo, n, pixel, z, k, c)
        lams.append(lam)
        phis.append(phi)
    return np.array(lams), np.array(phis)
