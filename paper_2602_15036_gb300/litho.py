"""Python binding of liblitho.so (ctypes): the C ABI of include/litho.h, same names.

Argument marshalling only: every step of the imaging, resist and gradient
path runs in the library's CUDA kernels.  torch tensors supply device memory
and streams (`tensor.data_ptr()`, `torch.cuda.current_stream().cuda_stream`).
If the shared library is missing this module raises at import of the
library, never falls back to another implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_size_t, c_uint8, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblitho.so")

OK, EINVAL, ENOMEM, ECUDA, EBUSY, ETIMEOUT, ECANCELED, EUNSUPPORTED = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EBUSY", "ETIMEOUT", "ECANCELED", "EUNSUPPORTED"]

SRC_ANNULAR, SRC_QUADRUPOLE, SRC_CUSTOM = 0, 1, 2
PREC = {"fft32": 0, "bf16": 1, "bf16x3": 2, "fp16x3": 3, "fp16": 4}
GRID_COARSE = 0x100


def prec_code(name: str) -> int:
    """'fft32', 'fp16x3', ... optionally with '/coarse' (LITHO_GRID_COARSE)."""
    base, _, grid = name.partition("/")
    if grid not in ("", "coarse"):
        raise ValueError(f"unknown grid {grid!r}")
    return PREC[base] | (GRID_COARSE if grid == "coarse" else 0)
REQ_IMAGE, REQ_ILT_STEP = 0, 1


class LithoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class litho_optics(ctypes.Structure):
    _fields_ = [("wavelength_nm", c_double), ("na", c_double), ("n_medium", c_double), ("kind", c_int),
                ("src_grid", c_int), ("sigma_in", c_double), ("sigma_out", c_double), ("pole_sigma", c_double),
                ("pole_radius", c_double), ("custom_w", POINTER(c_double))]


class litho_request(ctypes.Structure):
    _fields_ = [("kind", c_int), ("optics", litho_optics), ("n", c_int), ("pixel_nm", c_double),
                ("defocus_nm", c_double), ("k", c_int), ("precision", c_int), ("dose", c_double),
                ("sigma_nm", c_double), ("threshold", c_double), ("mask_steep", c_double),
                ("resist_steep", c_double), ("input_host", c_void_p), ("target_host", c_void_p),
                ("output_host", c_void_p), ("loss_host", c_void_p)]


class litho_serve_stats_t(ctypes.Structure):
    _fields_ = [("submitted", c_uint64), ("completed", c_uint64), ("rejected", c_uint64), ("cancelled", c_uint64),
                ("p50_ms", c_double), ("p99_ms", c_double), ("mpx_per_s", c_double), ("hbm_high_water", c_size_t),
                ("kernel_sets_cached", c_int), ("batches", c_uint64), ("max_batch", c_int)]


# name -> (restype, argtypes); mirrors include/litho.h
_SIGS = {
    "litho_make_kernels": (c_int, [POINTER(litho_optics), c_int, c_double, POINTER(c_double), c_int, c_int,
                                   POINTER(c_void_p)]),
    "litho_tcc_kernels_host": (c_int, [POINTER(litho_optics), c_int, c_double, c_double, c_int, POINTER(c_int),
                                       POINTER(c_double), POINTER(c_double), POINTER(c_int), POINTER(c_double),
                                       POINTER(c_double)]),
    "litho_upload_kernels": (c_int, [c_int, c_double, c_int, c_int, c_int, POINTER(c_double), POINTER(c_double),
                                     POINTER(c_void_p)]),
    "litho_kernels_info": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int),
                                   POINTER(c_int), POINTER(c_double), POINTER(c_double), POINTER(c_double)]),
    "litho_kernels_grid": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int)]),
    "litho_kernels_phi": (c_int, [c_void_p, POINTER(c_double)]),
    "litho_free_kernels": (None, [c_void_p]),
    "litho_aerial_workspace_size": (c_int, [c_void_p, c_int, c_int, POINTER(c_size_t)]),
    "litho_aerial": (c_int, [c_void_p, c_void_p, c_int, c_double, c_int, c_void_p, c_void_p, c_size_t, c_void_p]),
    "litho_aerial_resist": (c_int, [c_void_p, c_void_p, c_int, c_double, c_int, c_void_p, c_double, c_double,
                                    c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "litho_aerial_host_workspace_size": (c_int, [c_void_p, c_int, c_int, POINTER(c_size_t)]),
    "litho_aerial_host": (c_int, [c_void_p, c_void_p, c_int, c_double, c_int, c_void_p, c_double, c_double,
                                  c_void_p, c_void_p, c_size_t, c_void_p]),
    "litho_check_device": (c_int, [c_void_p, c_void_p]),
    "litho_selftest_wait_limit": (c_int, [c_void_p, c_double, c_void_p]),
    "litho_host_trace_read": (c_int, [c_int, POINTER(c_int), POINTER(c_double), POINTER(c_int)]),
    "litho_aerial_noalloc": (c_int, [c_void_p, c_void_p, c_int, c_double, c_void_p, c_void_p]),
    "litho_aerial_noalloc_max_bytes": (c_size_t, []),
    "litho_resist": (c_int, [c_void_p, c_int, c_int, c_double, c_double, c_double, c_void_p, c_void_p, c_void_p]),
    "litho_intensity_vjp_workspace_size": (c_int, [c_void_p, c_int, POINTER(c_size_t), POINTER(c_size_t)]),
    "litho_intensity_vjp": (c_int, [c_void_p, c_void_p, c_int, c_double, c_int, c_int, c_int, c_void_p, c_void_p,
                                    c_void_p, c_size_t, c_void_p]),
    "litho_ai_inputs_workspace_size": (c_int, [c_void_p, c_int, POINTER(c_size_t)]),
    "litho_ai_inputs": (c_int, [c_void_p, c_void_p, c_int, c_double, c_int, c_int, c_void_p, c_void_p, c_size_t,
                                c_void_p]),
    "litho_print_images": (c_int, [c_void_p, c_void_p, c_int, c_int, c_double, c_double, c_double, c_double, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_void_p]),
    "litho_rasterize_workspace_size": (c_int, [c_int, c_int, ctypes.c_int64, c_int, POINTER(c_size_t)]),
    "litho_rasterize": (c_int, [c_void_p, c_void_p, c_int, ctypes.c_int64, c_int, c_int, c_void_p, c_void_p,
                                c_size_t, c_void_p]),
    "litho_contours_workspace_size": (c_int, [c_int, c_int, POINTER(c_size_t)]),
    "litho_contours": (c_int, [c_void_p, c_int, c_int, c_double, c_void_p, c_void_p, ctypes.c_int64, c_void_p,
                               c_void_p, c_size_t, c_void_p]),
    "litho_epe": (c_int, [c_void_p, c_int, c_int, c_double, c_double, c_void_p, c_int, c_void_p, c_void_p]),
    "litho_epe_batch": (c_int, [c_void_p, c_int, c_int, c_int, c_double, c_double, c_void_p, c_void_p, ctypes.c_int64,
                                c_void_p, c_void_p]),
    "litho_epe_through_focus": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_double, c_double, c_void_p,
                                        c_void_p, c_void_p]),
    "litho_ilt_workspace_size": (c_int, [c_void_p, c_int, POINTER(c_size_t), POINTER(c_size_t)]),
    "litho_ilt_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_double, c_double, c_double, c_double,
                               c_int, c_void_p, POINTER(c_double), c_void_p, c_size_t, c_void_p]),
    "litho_serve_create": (c_int, [c_size_t, c_int, c_int, POINTER(c_void_p)]),
    "litho_serve_submit": (c_int, [c_void_p, POINTER(litho_request), POINTER(c_uint64)]),
    "litho_serve_poll": (c_int, [c_void_p, c_uint64, c_int]),
    "litho_serve_cancel": (c_int, [c_void_p, c_uint64]),
    "litho_serve_stats": (c_int, [c_void_p, POINTER(litho_serve_stats_t)]),
    "litho_serve_destroy": (None, [c_void_p]),
    "litho_serve_inject_fault": (c_int, [c_void_p, c_int]),
    "litho_serve_stats_reset": (c_int, [c_void_p]),
    "litho_profile_enable": (c_int, [c_int]),
    "litho_profile_reset": (None, []),
    "litho_profile_read": (c_int, [c_int, c_char_p, POINTER(c_double), POINTER(ctypes.c_longlong), POINTER(c_int)]),
    "litho_last_error": (c_char_p, []),
    "litho_version": (c_char_p, []),
}

_lib = None


def lib():
    """Loads liblitho.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2602_15036_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != OK:
        raise LithoError(status, lib().litho_last_error().decode())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def make_optics(wavelength_nm=193.0, na=1.35, n_medium=1.44, kind="annular", src_grid=21, sigma_in=0.6,
                sigma_out=0.9, pole_sigma=0.8, pole_radius=0.1, custom_w=None):
    kinds = {"annular": SRC_ANNULAR, "quadrupole": SRC_QUADRUPOLE, "custom": SRC_CUSTOM}
    o = litho_optics(wavelength_nm, na, n_medium, kinds[kind] if isinstance(kind, str) else int(kind), src_grid,
                     sigma_in, sigma_out, pole_sigma, pole_radius, None)
    if custom_w is not None:
        arr = np.ascontiguousarray(custom_w, dtype=np.float64)
        o._keep = arr
        o.custom_w = arr.ctypes.data_as(POINTER(c_double))
    return o


class Kernels:
    """Owner of a device-resident litho_kernels handle."""

    def __init__(self, handle: int):
        self.handle = c_void_p(handle)
        n, c, f, k = c_int(), c_int(), c_int(), c_int()
        _check(lib().litho_kernels_info(self.handle, byref(n), byref(c), byref(f), byref(k), None, None, None, None))
        self.n, self.crop, self.n_focus, self.k = n.value, c.value, f.value, k.value

    def info(self):
        f, k = self.n_focus, self.k
        rank = (c_int * f)()
        lam = np.zeros(f * k)
        tr = np.zeros(f)
        gap = np.zeros(f)
        _check(lib().litho_kernels_info(self.handle, None, None, None, None, rank,
                                        lam.ctypes.data_as(POINTER(c_double)), tr.ctypes.data_as(POINTER(c_double)),
                                        gap.ctypes.data_as(POINTER(c_double))))
        return {"rank": list(rank), "lambda": lam.reshape(f, k), "trace": tr, "gap": gap}

    def phi(self):
        out = np.zeros((self.n_focus, self.k, self.crop, self.crop, 2))
        _check(lib().litho_kernels_phi(self.handle, out.ctypes.data_as(POINTER(c_double))))
        return out[..., 0] + 1j * out[..., 1]

    def grid(self, precision: str = "fft32") -> int:
        """Coarse evaluation grid of a precision's path with "/coarse" (0: not below n)."""
        fft, tc = c_int(), c_int()
        _check(lib().litho_kernels_grid(self.handle, byref(fft), byref(tc)))
        return fft.value if precision.split("/")[0] == "fft32" else tc.value

    def close(self):
        if self.handle is not None and self.handle.value:
            lib().litho_free_kernels(self.handle)
            self.handle = c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def litho_make_kernels(optics, n, pixel_nm, defocus_nm, k) -> Kernels:
    z = np.ascontiguousarray(np.atleast_1d(defocus_nm), dtype=np.float64)
    h = c_void_p()
    _check(lib().litho_make_kernels(byref(optics), n, pixel_nm, z.ctypes.data_as(POINTER(c_double)), len(z), k,
                                    byref(h)))
    return Kernels(h.value)


def litho_tcc_kernels_host(optics, n, pixel_nm, defocus_nm, k):
    """FP64 host kernel build for one focus plane (no GPU): returns
    (lam[k], phi[k][C][C] complex128, info dict)."""
    crop = c_int()
    _check(lib().litho_tcc_kernels_host(byref(optics), n, pixel_nm, defocus_nm, k, byref(crop), None, None, None,
                                        None, None))
    c = crop.value
    lam = np.zeros(k)
    phi = np.zeros((k, c, c, 2))
    rank, tr, gap = c_int(), c_double(), c_double()
    _check(lib().litho_tcc_kernels_host(byref(optics), n, pixel_nm, defocus_nm, k, byref(crop),
                                        lam.ctypes.data_as(POINTER(c_double)), phi.ctypes.data_as(POINTER(c_double)),
                                        byref(rank), byref(tr), byref(gap)))
    return lam, phi[..., 0] + 1j * phi[..., 1], {"rank": rank.value, "trace": tr.value, "gap": gap.value}


def litho_upload_kernels(n, pixel_nm, lam, phi) -> Kernels:
    """lam [F][K] float64, phi [F][K][C][C] complex."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    f, k = lam.shape
    phi = np.asarray(phi)
    c = phi.shape[-1]
    inter = np.ascontiguousarray(np.stack([phi.real, phi.imag], axis=-1), dtype=np.float64)
    h = c_void_p()
    _check(lib().litho_upload_kernels(n, pixel_nm, f, k, c, lam.ctypes.data_as(POINTER(c_double)),
                                      inter.ctypes.data_as(POINTER(c_double)), byref(h)))
    return Kernels(h.value)


def litho_aerial_workspace_size(kern: Kernels, b: int, precision="fft32") -> int:
    out = c_size_t()
    _check(lib().litho_aerial_workspace_size(kern.handle, b, prec_code(precision), byref(out)))
    return out.value


def litho_aerial(kern: Kernels, mask, dose=1.0, precision="fft32", out=None, workspace=None, stream=None):
    """mask: torch float32 CUDA tensor [b][n][n] -> intensity [b][F][n][n]."""
    import torch
    assert mask.is_cuda and mask.dtype == torch.float32 and mask.is_contiguous()
    b = mask.shape[0]
    if out is None:
        out = torch.empty((b, kern.n_focus, kern.n, kern.n), dtype=torch.float32, device=mask.device)
    if workspace is None:
        workspace = torch.empty(litho_aerial_workspace_size(kern, b, precision), dtype=torch.uint8,
                                device=mask.device)
    _check(lib().litho_aerial(kern.handle, c_void_p(mask.data_ptr()), b, dose, prec_code(precision),
                              c_void_p(out.data_ptr()), c_void_p(workspace.data_ptr()), workspace.numel(),
                              _stream_ptr(stream)))
    return out


def litho_aerial_resist(kern: Kernels, mask, dose=1.0, precision="fft32", sigma_nm=10.0, threshold=0.3, out=None,
                        iblur=None, printed=None, want_printed=True, workspace=None, stream=None):
    """mask: torch float32 CUDA tensor [b][n][n] -> (intensity, iblur, printed u8 or None), each [b][F][n][n]."""
    import torch
    assert mask.is_cuda and mask.dtype == torch.float32 and mask.is_contiguous()
    b = mask.shape[0]
    shape = (b, kern.n_focus, kern.n, kern.n)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=mask.device)
    if iblur is None:
        iblur = torch.empty(shape, dtype=torch.float32, device=mask.device)
    if printed is None and want_printed:
        printed = torch.empty(shape, dtype=torch.uint8, device=mask.device)
    if workspace is None:
        workspace = torch.empty(litho_aerial_workspace_size(kern, b, precision), dtype=torch.uint8,
                                device=mask.device)
    _check(lib().litho_aerial_resist(kern.handle, c_void_p(mask.data_ptr()), b, dose, prec_code(precision),
                                     c_void_p(out.data_ptr()), sigma_nm, threshold, c_void_p(iblur.data_ptr()),
                                     c_void_p(printed.data_ptr()) if printed is not None else None,
                                     c_void_p(workspace.data_ptr()), workspace.numel(), _stream_ptr(stream)))
    return out, iblur, printed


def litho_aerial_host_workspace_size(kern: Kernels, b: int, precision="fft32") -> int:
    out = c_size_t()
    _check(lib().litho_aerial_host_workspace_size(kern.handle, b, prec_code(precision), byref(out)))
    return out.value


def litho_aerial_host(kern: Kernels, mask_host, workspace, intensity_host=None, printed_host=None, dose=1.0,
                      precision="fft32", sigma_nm=10.0, threshold=0.3, stream=None):
    """mask_host [b][n][n] f32, intensity_host [b][F][n][n] f32 and/or printed_host
    [b][F][n][n] u8: CPU tensors (pinned for full-speed copies) or numpy arrays.
    Synchronous."""
    def ptr(a):
        if a is None:
            return None
        return c_void_p(a.data_ptr()) if hasattr(a, "data_ptr") else c_void_p(a.ctypes.data)
    b = mask_host.shape[0]
    _check(lib().litho_aerial_host(kern.handle, ptr(mask_host), b, dose, prec_code(precision), ptr(intensity_host),
                                   sigma_nm, threshold, ptr(printed_host), c_void_p(workspace.data_ptr()),
                                   workspace.numel(), _stream_ptr(stream)))
    return intensity_host, printed_host


def litho_check_device(kern: Kernels, stream=None):
    """Raises LithoError(ETIMEOUT) if a tensor-core kernel gave up on a barrier wait."""
    _check(lib().litho_check_device(kern.handle, _stream_ptr(stream)))


def litho_selftest_wait_limit(kern: Kernels, limit_ms: float = 50.0, stream=None) -> int:
    """Status of the bounded-wait self-test (ETIMEOUT when the limit works)."""
    return lib().litho_selftest_wait_limit(kern.handle, limit_ms, _stream_ptr(stream))


def litho_aerial_noalloc(kern: Kernels, mask, out, dose=1.0, stream=None):
    """FP32 aerial image with no device allocation: the library's fixed scratch
    array stands in for the workspace, so `out` must be preallocated
    ([b][F][n][n] float32 on the device).  Calls that may overlap on the GPU
    race on that array; keep them on one stream."""
    import torch
    b = mask.shape[0]
    n, nf = kern.n, kern.n_focus
    if mask.dtype != torch.float32 or out.dtype != torch.float32:
        raise ValueError("mask and out must be float32")
    if tuple(mask.shape) != (b, n, n) or tuple(out.shape) != (b, nf, n, n):
        raise ValueError(f"need mask [b][{n}][{n}] and out [b][{nf}][{n}][{n}]; got {tuple(mask.shape)} and "
                         f"{tuple(out.shape)}")
    if not (mask.is_cuda and out.is_cuda and mask.device == out.device):
        raise ValueError("mask and out must be on the same CUDA device")
    if not (mask.is_contiguous() and out.is_contiguous()):
        raise ValueError("mask and out must be contiguous")
    _check(lib().litho_aerial_noalloc(kern.handle, c_void_p(mask.data_ptr()), mask.shape[0], dose,
                                      c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def litho_host_trace_read(max_events: int = 256):
    """Host timestamps of the last litho_aerial_host call: list of (tag, ms since the call began)."""
    tags = (c_int * max_events)()
    ms = (c_double * max_events)()
    count = c_int()
    _check(lib().litho_host_trace_read(max_events, tags, ms, byref(count)))
    return [(tags[i], ms[i]) for i in range(min(count.value, max_events))]


def litho_aerial_noalloc_max_bytes() -> int:
    return int(lib().litho_aerial_noalloc_max_bytes())


def litho_resist(intensity, pixel_nm, sigma_nm=10.0, threshold=0.3, iblur=None, printed=None, want_printed=True,
                 stream=None):
    """intensity: CUDA float32 [..., n, n] -> (iblur, printed u8 or None)."""
    import torch
    n = intensity.shape[-1]
    planes = intensity.numel() // (n * n)
    if iblur is None:
        iblur = torch.empty_like(intensity)
    if printed is None and want_printed:
        printed = torch.empty(intensity.shape, dtype=torch.uint8, device=intensity.device)
    _check(lib().litho_resist(c_void_p(intensity.data_ptr()), planes, n, pixel_nm, sigma_nm, threshold,
                              c_void_p(iblur.data_ptr()), c_void_p(printed.data_ptr()) if printed is not None else None,
                              _stream_ptr(stream)))
    return iblur, printed


def litho_contours(iblur, threshold=0.3, capacity=None, with_cells=True, stream=None):
    """iblur: CUDA float32 [..., n, n] -> (segments [S][4] (x0, y0, x1, y1), cells [S] int32 or None,
    plane_start [planes + 1] int64 numpy).  With capacity=None the call runs once to count and
    again into buffers of the exact size."""
    import torch
    n = iblur.shape[-1]
    planes = iblur.numel() // (n * n)
    dev = iblur.device
    ws_bytes = c_size_t()
    _check(lib().litho_contours_workspace_size(planes, n, byref(ws_bytes)))
    ws = torch.empty(ws_bytes.value, dtype=torch.uint8, device=dev)
    starts = torch.empty(planes + 1, dtype=torch.int64, device=dev)

    def run(cap):
        seg = torch.empty((max(cap, 1), 4), dtype=torch.float32, device=dev)
        cell = torch.empty(max(cap, 1), dtype=torch.int32, device=dev) if with_cells else None
        _check(lib().litho_contours(c_void_p(iblur.data_ptr()), planes, n, threshold, c_void_p(seg.data_ptr()),
                                    c_void_p(cell.data_ptr()) if cell is not None else None, cap,
                                    c_void_p(starts.data_ptr()), c_void_p(ws.data_ptr()), ws.numel(),
                                    _stream_ptr(stream)))
        return seg, cell

    if capacity is None:
        run(0)
        capacity = int(starts[-1].item())
    seg, cell = run(capacity)
    st = starts.cpu().numpy()
    kept = min(capacity, int(st[-1]))
    return seg[:kept], (cell[:kept] if cell is not None else None), st


def litho_intensity_vjp(kern: Kernels, mask, upstream=None, f_first=0, f_count=None, dose=1.0, precision="fft32",
                        stream=None):
    """mask: CUDA float32 [b][n][n]; upstream: CUDA float32 [b][n_focus][n][n] or None (ones) ->
    dm [b][n][n] = sum over planes [f_first, f_first + f_count) of J_f^T upstream_f."""
    import torch
    b = mask.shape[0]
    f_count = kern.n_focus - f_first if f_count is None else f_count
    full, mn = c_size_t(), c_size_t()
    _check(lib().litho_intensity_vjp_workspace_size(kern.handle, b, byref(full), byref(mn)))
    ws = torch.empty(full.value, dtype=torch.uint8, device=mask.device)
    dm = torch.empty_like(mask)
    _check(lib().litho_intensity_vjp(kern.handle, c_void_p(mask.data_ptr()), b, dose, prec_code(precision), f_first,
                                     f_count,
                                     c_void_p(upstream.data_ptr()) if upstream is not None else None,
                                     c_void_p(dm.data_ptr()), c_void_p(ws.data_ptr()), ws.numel(),
                                     _stream_ptr(stream)))
    return dm


def litho_ai_inputs_workspace_size(kern: Kernels, b: int) -> int:
    sz = c_size_t()
    _check(lib().litho_ai_inputs_workspace_size(kern.handle, b, byref(sz)))
    return sz.value


def litho_ai_inputs(kern: Kernels, targets, focus=0, dose=1.0, precision="fft32", out=None, workspace=None,
                    stream=None):
    """targets: CUDA float32 [b][n][n] (0/1) -> X [b][3][n][n] (Eq. (9) channels)."""
    import torch
    b, n = targets.shape[0], targets.shape[-1]
    if workspace is None:
        workspace = torch.empty(litho_ai_inputs_workspace_size(kern, b), dtype=torch.uint8, device=targets.device)
    x = out if out is not None else torch.empty((b, 3, n, n), dtype=torch.float32, device=targets.device)
    _check(lib().litho_ai_inputs(kern.handle, c_void_p(targets.data_ptr()), b, dose, focus, prec_code(precision),
                                 c_void_p(x.data_ptr()), c_void_p(workspace.data_ptr()), workspace.numel(),
                                 _stream_ptr(stream)))
    return x


def litho_print_images(targets, images, pixel_nm, sigma_round_nm, tau_round, tau_print, stream=None):
    """targets, images: CUDA float32 [b][n][n] -> (z_round u8, z_print u8, loss int64 [b], blurred target)."""
    import torch
    b, n = targets.shape[0], targets.shape[-1]
    zr = torch.empty((b, n, n), dtype=torch.uint8, device=targets.device)
    zp = torch.empty_like(zr)
    loss = torch.empty(b, dtype=torch.int64, device=targets.device)
    blur = torch.empty_like(targets)
    _check(lib().litho_print_images(c_void_p(targets.data_ptr()), c_void_p(images.data_ptr()), b, n, pixel_nm,
                                    sigma_round_nm, tau_round, tau_print, c_void_p(zr.data_ptr()),
                                    c_void_p(zp.data_ptr()), c_void_p(loss.data_ptr()), c_void_p(blur.data_ptr()),
                                    _stream_ptr(stream)))
    return zr, zp, loss, blur


def litho_rasterize(rects, n, max_side_px, device="cuda", out=None, stream=None):
    """rects: list (one entry per clip) of float arrays [R_c][4] (x0, y0, x1, y1) in pixels ->
    CUDA float32 [b][n][n] area-coverage masks."""
    import torch
    b = len(rects)
    counts = [int(np.asarray(r).reshape(-1, 4).shape[0]) for r in rects]
    start = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    flat = np.concatenate([np.asarray(r, dtype=np.float32).reshape(-1, 4) for r in rects] +
                          [np.zeros((1, 4), np.float32)])
    d_rects = torch.from_numpy(flat).to(device)
    d_start = torch.from_numpy(start).to(device)
    max_rects = max(counts) if counts else 0
    ws_bytes = c_size_t()
    _check(lib().litho_rasterize_workspace_size(b, n, max_rects, max_side_px, byref(ws_bytes)))
    ws = torch.empty(ws_bytes.value, dtype=torch.uint8, device=device)
    if out is None:
        out = torch.empty((b, n, n), dtype=torch.float32, device=device)
    _check(lib().litho_rasterize(c_void_p(d_rects.data_ptr()), c_void_p(d_start.data_ptr()), b, max_rects,
                                 max_side_px, n, c_void_p(out.data_ptr()), c_void_p(ws.data_ptr()), ws.numel(),
                                 _stream_ptr(stream)))
    return out


def rasterize_workspace_size(b: int, n: int, max_rects: int, max_side_px: int) -> int:
    out = c_size_t()
    _check(lib().litho_rasterize_workspace_size(b, n, max_rects, max_side_px, byref(out)))
    return out.value


def rasterize_into(rects, rect_start, b, max_rects, max_side_px, n, mask, workspace, stream=None):
    """litho_rasterize on CUDA tensors (rects [R][4] f32, rect_start [b+1] int64), asynchronous."""
    _check(lib().litho_rasterize(c_void_p(rects.data_ptr()), c_void_p(rect_start.data_ptr()), b, max_rects,
                                 max_side_px, n, c_void_p(mask.data_ptr()), c_void_p(workspace.data_ptr()),
                                 workspace.numel(), _stream_ptr(stream)))


def contours_workspace_size(planes: int, n: int) -> int:
    out = c_size_t()
    _check(lib().litho_contours_workspace_size(planes, n, byref(out)))
    return out.value


def contours_into(iblur, planes, n, threshold, seg, cell, capacity, plane_start, workspace, stream=None):
    """litho_contours into caller buffers (CUDA tensors), asynchronous: no host synchronisation."""
    _check(lib().litho_contours(c_void_p(iblur.data_ptr()), planes, n, threshold, c_void_p(seg.data_ptr()),
                                c_void_p(cell.data_ptr()) if cell is not None else None, capacity,
                                c_void_p(plane_start.data_ptr()), c_void_p(workspace.data_ptr()), workspace.numel(),
                                _stream_ptr(stream)))


def epe_through_focus_into(epe, f0, fp, fn, tol_neg, tol_pos, avg, eff, stream=None):
    """litho_epe_through_focus into caller buffers, asynchronous."""
    planes, m = epe.shape
    _check(lib().litho_epe_through_focus(c_void_p(epe.data_ptr()), planes, m, f0, fp, fn, tol_neg, tol_pos,
                                         c_void_p(avg.data_ptr()) if avg is not None else None,
                                         c_void_p(eff.data_ptr()) if eff is not None else None, _stream_ptr(stream)))


def litho_epe(iblur, points, pixel_nm, threshold=0.3, out=None, stream=None):
    """iblur: CUDA float32 [planes][n][n] (or [n][n]); points: CUDA float32 [m][2] (x, y) in
    pixels -> EPE [planes][m] in nm (Eq. (6))."""
    import torch
    n = iblur.shape[-1]
    planes = iblur.numel() // (n * n)
    m = points.shape[0]
    assert points.is_cuda and points.dtype == torch.float32 and points.is_contiguous()
    if out is None:
        out = torch.empty((planes, m), dtype=torch.float32, device=iblur.device)
    _check(lib().litho_epe(c_void_p(iblur.data_ptr()), planes, n, pixel_nm, threshold, c_void_p(points.data_ptr()),
                           m, c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def litho_epe_batch(iblur, points, start, pixel_nm, threshold=0.3, out=None, stream=None):
    """iblur: CUDA float32 [clips][planes][n][n]; points: CUDA float32 [M][2] (all clips' points);
    start: CUDA int64 [clips + 1] (clip c's points at start[c] .. start[c+1]) -> EPE [planes][M] in nm."""
    import torch
    clips, planes, n = iblur.shape[0], iblur.shape[1], iblur.shape[-1]
    m = points.shape[0]
    assert points.is_cuda and points.dtype == torch.float32 and points.is_contiguous()
    assert start.is_cuda and start.dtype == torch.int64 and start.numel() == clips + 1
    if out is None:
        out = torch.empty((planes, m), dtype=torch.float32, device=iblur.device)
    _check(lib().litho_epe_batch(c_void_p(iblur.data_ptr()), clips, planes, n, pixel_nm, threshold,
                                 c_void_p(points.data_ptr()), c_void_p(start.data_ptr()), m, c_void_p(out.data_ptr()),
                                 _stream_ptr(stream)))
    return out


def litho_epe_through_focus(epe, f0, fp, fn, tol_neg, tol_pos, stream=None):
    """epe: CUDA float32 [planes][m] -> (EPE_avg [m], EPE_eff [m]) (Eqs. (7)-(8))."""
    import torch
    planes, m = epe.shape
    avg = torch.empty(m, dtype=torch.float32, device=epe.device)
    eff = torch.empty(m, dtype=torch.float32, device=epe.device)
    _check(lib().litho_epe_through_focus(c_void_p(epe.data_ptr()), planes, m, f0, fp, fn, tol_neg, tol_pos,
                                         c_void_p(avg.data_ptr()), c_void_p(eff.data_ptr()), _stream_ptr(stream)))
    return avg, eff


def litho_ilt_workspace_size(kern: Kernels, b: int):
    full, mn = c_size_t(), c_size_t()
    _check(lib().litho_ilt_workspace_size(kern.handle, b, byref(full), byref(mn)))
    return full.value, mn.value


def litho_ilt_grad(kern: Kernels, theta, target, dose=1.0, mask_steep=4.0, resist_steep=25.0, threshold=0.3,
                   sigma_nm=10.0, precision="fft32", grad=None, workspace=None, want_loss=True, stream=None):
    """theta, target: CUDA float32 [b][n][n] -> (grad, loss[b] float64 numpy or None)."""
    import torch
    b = theta.shape[0]
    if grad is None:
        grad = torch.empty_like(theta)
    if workspace is None:
        workspace = torch.empty(litho_ilt_workspace_size(kern, b)[0], dtype=torch.uint8, device=theta.device)
    loss = np.zeros(b) if want_loss else None
    _check(lib().litho_ilt_grad(kern.handle, c_void_p(theta.data_ptr()), c_void_p(target.data_ptr()), b, dose,
                                mask_steep, resist_steep, threshold, sigma_nm, prec_code(precision),
                                c_void_p(grad.data_ptr()),
                                loss.ctypes.data_as(POINTER(c_double)) if want_loss else None,
                                c_void_p(workspace.data_ptr()), workspace.numel(), _stream_ptr(stream)))
    return grad, loss


class Server:
    """litho_serve_*: continuous-batching request server (one clip per request).

    submit() copies nothing: the numpy arrays given for input, target and
    output must stay alive until poll() reports the request finished; the
    server keeps references to them for that reason.
    """

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 4, max_queue: int = 4096):
        h = c_void_p()
        _check(lib().litho_serve_create(hbm_budget_bytes, max_slots, max_queue, byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, kind, optics, n, pixel_nm, defocus_nm, k, input_host, output_host, target_host=None,
               precision="fft32", dose=1.0, sigma_nm=10.0, threshold=0.3, mask_steep=4.0, resist_steep=25.0):
        """kind: 'image' or 'ilt'.  Arrays: contiguous float32 numpy [n][n].
        Returns (ticket, loss_buffer) where loss_buffer[0] receives the ILT loss."""
        loss = np.zeros(1)
        r = litho_request()
        r.kind = REQ_IMAGE if kind == "image" else REQ_ILT_STEP
        r.optics = optics
        r.n, r.pixel_nm, r.defocus_nm, r.k = n, pixel_nm, defocus_nm, k
        r.precision = prec_code(precision)
        r.dose, r.sigma_nm, r.threshold, r.mask_steep, r.resist_steep = dose, sigma_nm, threshold, mask_steep, \
            resist_steep
        r.input_host = input_host.ctypes.data
        r.target_host = target_host.ctypes.data if target_host is not None else None
        r.output_host = output_host.ctypes.data
        r.loss_host = loss.ctypes.data
        t = c_uint64()
        _check(lib().litho_serve_submit(self.handle, byref(r), byref(t)))
        self._keep[t.value] = (input_host, output_host, target_host, loss, optics)
        return t.value, loss

    def poll(self, ticket: int, timeout_ms: int = 0) -> int:
        """Status code: OK, ETIMEOUT (pending), ECANCELED or the request's error."""
        return lib().litho_serve_poll(self.handle, ticket, timeout_ms)

    def cancel(self, ticket: int) -> int:
        return lib().litho_serve_cancel(self.handle, ticket)

    def inject_fault(self, mask: int):
        _check(lib().litho_serve_inject_fault(self.handle, mask))

    def stats_reset(self):
        _check(lib().litho_serve_stats_reset(self.handle))

    def stats(self) -> dict:
        s = litho_serve_stats_t()
        _check(lib().litho_serve_stats(self.handle, byref(s)))
        return {f: getattr(s, f) for f, _ in litho_serve_stats_t._fields_}

    def close(self):
        if self.handle is not None and self.handle.value:
            lib().litho_serve_destroy(self.handle)
            self.handle = c_void_p(0)
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def litho_profile_enable(on: bool = True):
    _check(lib().litho_profile_enable(1 if on else 0))


def litho_profile_reset():
    lib().litho_profile_reset()


def litho_profile_read() -> dict:
    """{stage: (total device ms, kernel launches)} since the last reset."""
    mx = 16
    names = ctypes.create_string_buffer(32 * mx)
    ms = (c_double * mx)()
    launches = (ctypes.c_longlong * mx)()
    cnt = c_int()
    _check(lib().litho_profile_read(mx, names, ms, launches, byref(cnt)))
    out = {}
    for i in range(cnt.value):
        nm = names.raw[32 * i:32 * (i + 1)].split(b"\0")[0].decode()
        out[nm] = (ms[i], launches[i])
    return out


def litho_last_error() -> str:
    return lib().litho_last_error().decode()


def litho_version() -> str:
    return lib().litho_version().decode()
