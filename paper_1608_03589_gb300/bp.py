"""ctypes binding of libbp.so (include/bp.h): argument marshalling only.

Every operator runs in the library's CUDA kernels; this module checks tensor shapes,
dtypes and devices, passes raw device pointers and the current CUDA stream, and raises
BPError with the library's message on failure.  There is no CPU fallback: if libbp.so
is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from typing import Sequence

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libbp.so")

BP_F32, BP_BF16, BP_F16 = 0, 1, 2
FILTERS = {"ramlak": 0, "ram-lak": 0, "shepp-logan": 1, "shepp_logan": 1, "tikhonov": 2}
_DTYPES = {torch.float32: BP_F32, torch.bfloat16: BP_BF16, torch.float16: BP_F16}

# Every symbol the header declares (checked by the ABI test).
SYMBOLS = ("bp_plan_create", "bp_destroy", "bp_filter", "bp_backproject_direct", "bp_backproject_fourier",
           "bp_radon", "bp_fbp_host", "bp_fbp_fourier", "bp_fbp_direct", "bp_backproject_bst",
           "bp_backproject_bst_windowed", "bp_backproject_logpolar", "bp_backproject_logpolar_partial", "bp_set_fourier_width", "bp_set_direct_workspace", "bp_backproject_batched", "bp_fbp_static", "bp_check", "bp_radon_transpose",
           "bp_backproject_transpose", "bp_autotune", "bp_get_shape", "bp_set_shape", "bp_tune_cache_save",
           "bp_tune_cache_load", "bp_stage_timing", "bp_stage_times", "bp_last_error", "bp_version")
OPS = {"direct": 0, "radon": 1}


class BPError(RuntimeError):
    pass


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load libbp.so (built by __graft_entry__.build() or paper_1608_03589_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise BPError(f"libbp.so not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            vp, i, f, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double
            L.bp_plan_create.argtypes = [i, i, i, ctypes.POINTER(d), d]
            L.bp_plan_create.restype = vp
            L.bp_destroy.argtypes = [vp]
            L.bp_destroy.restype = None
            L.bp_filter.argtypes = [vp, vp, i, vp, i, f, i, vp]
            L.bp_backproject_direct.argtypes = [vp, vp, i, vp, i, i, vp]
            L.bp_backproject_fourier.argtypes = [vp, vp, i, vp, i, vp]
            L.bp_radon.argtypes = [vp, vp, vp, i, i, vp]
            L.bp_fbp_host.argtypes = [vp, vp, vp, i, f, i, vp]
            L.bp_fbp_static.argtypes = [vp, vp, i, vp, i, i, vp]
            L.bp_fbp_fourier.argtypes = [vp, vp, i, vp, i, f, i, vp]
            L.bp_fbp_direct.argtypes = [vp, vp, i, vp, i, f, i, vp]
            L.bp_backproject_bst.argtypes = [vp, vp, i, vp, i, i, vp]
            L.bp_backproject_bst_windowed.argtypes = [vp, vp, i, vp, i, f, i, vp]
            L.bp_backproject_logpolar.argtypes = [vp, vp, i, vp, i, vp]
            L.bp_backproject_logpolar_partial.argtypes = [vp, vp, i, vp, i, f, i, vp]
            L.bp_set_fourier_width.argtypes = [vp, i]
            L.bp_set_direct_workspace.argtypes = [vp, ctypes.c_ulonglong]
            L.bp_check.argtypes = [vp, vp]
            L.bp_radon_transpose.argtypes = [vp, vp, vp, i, i, vp]
            L.bp_backproject_transpose.argtypes = [vp, vp, vp, i, i, vp]
            L.bp_backproject_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i),
                                                 ctypes.POINTER(vp), i, vp]
            ip = ctypes.POINTER(i)
            L.bp_autotune.argtypes = [vp, i, i, i, vp, ip, ctypes.POINTER(f)]
            L.bp_get_shape.argtypes = [vp, i, i, i, ip]
            L.bp_set_shape.argtypes = [vp, i, i, i, ip]
            L.bp_tune_cache_save.argtypes = [ctypes.c_char_p]
            L.bp_tune_cache_load.argtypes = [ctypes.c_char_p]
            L.bp_stage_timing.argtypes = [vp, i]
            L.bp_stage_times.argtypes = [vp, i, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(f), ip, ip]
            for name in ("bp_filter", "bp_backproject_direct", "bp_backproject_fourier", "bp_radon",
                         "bp_fbp_host", "bp_fbp_fourier", "bp_fbp_direct", "bp_backproject_bst", "bp_backproject_bst_windowed",
                         "bp_backproject_logpolar", "bp_backproject_logpolar_partial",
                         "bp_set_fourier_width", "bp_set_direct_workspace",
                         "bp_backproject_batched", "bp_fbp_static",
                         "bp_check",
                         "bp_radon_transpose", "bp_backproject_transpose", "bp_autotune", "bp_get_shape",
                         "bp_set_shape", "bp_tune_cache_save", "bp_tune_cache_load", "bp_stage_timing",
                         "bp_stage_times"):
                getattr(L, name).restype = i
            L.bp_last_error.argtypes = []
            L.bp_last_error.restype = ctypes.c_char_p
            L.bp_version.argtypes = []
            L.bp_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(status: int, what: str) -> None:
    if status != 0:
        msg = lib().bp_last_error().decode(errors="replace")
        raise BPError(f"{what} failed (status {status}): {msg}")


def _stream(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def _cuda(t: torch.Tensor, name: str) -> None:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise BPError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise BPError(f"{name} must be contiguous")


class Plan:
    """Geometry of one slice (N x N image, n_theta x n_det sinogram), see include/bp.h."""

    def __init__(self, N: int, n_det: int, theta, det_spacing: float | None = None,
                 device: torch.device | int | None = None):
        theta = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).ravel())
        self.N, self.n_det, self.n_theta = int(N), int(n_det), int(theta.shape[0])
        self.theta = theta
        self.det_spacing = float(2.0 / n_det if det_spacing is None else det_spacing)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   (device if isinstance(device, int) else device.index or 0))
        with torch.cuda.device(self.device):
            h = lib().bp_plan_create(self.N, self.n_det, self.n_theta,
                                     theta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.det_spacing)
        if not h:
            raise BPError("bp_plan_create failed: " + lib().bp_last_error().decode(errors="replace"))
        self._h = ctypes.c_void_p(h)

    # ------------------------------------------------------------------ helpers
    def _batch(self, t: torch.Tensor, tail: tuple[int, int], name: str) -> int:
        if t.dim() < 2 or tuple(t.shape[-2:]) != tail:
            raise BPError(f"{name} must have shape [..., {tail[0]}, {tail[1]}], got {tuple(t.shape)}")
        if t.device != self.device:
            raise BPError(f"{name} is on {t.device}, plan on {self.device}")
        return int(math.prod(t.shape[:-2])) if t.dim() > 2 else 1

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise BPError("plan is closed")
        return self._h

    # ------------------------------------------------------------------ operators
    def filter(self, sino: torch.Tensor, kind: str | int = "ramlak", param: float = 0.0,
               out: torch.Tensor | None = None) -> torch.Tensor:
        """FBP row filter (eq "fbp"; Section 6 for "tikhonov"), float32 output."""
        _cuda(sino, "sino")
        b = self._batch(sino, (self.n_theta, self.n_det), "sino")
        if sino.dtype not in _DTYPES:
            raise BPError(f"unsupported sinogram dtype {sino.dtype}")
        k = FILTERS[kind] if isinstance(kind, str) else int(kind)
        if out is None:
            out = torch.empty(sino.shape, dtype=torch.float32, device=sino.device)
        _cuda(out, "out")
        with torch.cuda.device(self.device):
            _check(lib().bp_filter(self.handle, sino.data_ptr(), _DTYPES[sino.dtype], out.data_ptr(), k,
                                   float(param), b, _stream(sino)), "bp_filter")
        return out

    def backproject(self, sino: torch.Tensor, out: torch.Tensor | None = None,
                    accumulate: bool = False) -> torch.Tensor:
        """Direct pixel-driven R* with linear interpolation (Section 2, eq "bp_app")."""
        _cuda(sino, "sino")
        b = self._batch(sino, (self.n_theta, self.n_det), "sino")
        if sino.dtype not in _DTYPES:
            raise BPError(f"unsupported sinogram dtype {sino.dtype}")
        if out is None:
            if accumulate:
                raise BPError("accumulate=True needs out")
            out = torch.empty((*sino.shape[:-2], self.N, self.N), dtype=torch.float32, device=sino.device)
        _cuda(out, "out")
        if out.dtype != torch.float32 or out.numel() != b * self.N * self.N:
            raise BPError("out must be float32 with batch x N x N elements")
        with torch.cuda.device(self.device):
            _check(lib().bp_backproject_direct(self.handle, sino.data_ptr(), _DTYPES[sino.dtype], out.data_ptr(),
                                               b, int(bool(accumulate)), _stream(sino)), "bp_backproject_direct")
        return out

    def backproject_fourier(self, sino: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """BST / gridding form of R* (Section 3 eq "bst", Section 5.3)."""
        _cuda(sino, "sino")
        b = self._batch(sino, (self.n_theta, self.n_det), "sino")
        if sino.dtype not in _DTYPES:
            raise BPError(f"unsupported sinogram dtype {sino.dtype}")
        if out is None:
            out = torch.empty((*sino.shape[:-2], self.N, self.N), dtype=torch.float32, device=sino.device)
        _cuda(out, "out")
        if out.dtype != torch.float32 or out.numel() != b * self.N * self.N:
            raise BPError("out must be float32 with batch x N x N elements")
        with torch.cuda.device(self.device):
            _check(lib().bp_backproject_fourier(self.handle, sino.data_ptr(), _DTYPES[sino.dtype], out.data_ptr(),
                                                b, _stream(sino)), "bp_backproject_fourier")
        return out

    def backproject_bst(self, sino: torch.Tensor, oversampling: int = 4,
                        out: torch.Tensor | None = None) -> torch.Tensor:
        """R* by the paper's BST algorithm: polar-to-Cartesian interpolation in frequency with
        K^sigma (Section 5.3 Steps 1-4, bp_backproject_bst); radial oversampling 1, 2, 4, 8."""
        _cuda(sino, "sino")
        b = self._batch(sino, (self.n_theta, self.n_det), "sino")
        if sino.dtype not in _DTYPES:
            raise BPError(f"unsupported sinogram dtype {sino.dtype}")
        if out is None:
            out = torch.empty((*sino.shape[:-2], self.N, self.N), dtype=torch.float32, device=sino.device)
        _cuda(out, "out")
        if out.dtype != torch.float32 or out.numel() != b * self.N * self.N:
            raise BPError("out must be float32 with batch x N x N elements")
        with torch.cuda.device(self.device):
            _check(lib().bp_backproject_bst(self.handle, sino.data_ptr(), _DTYPES[sino.dtype], out.data_ptr(),
                                            int(oversampling), b, _stream(sino)), "bp_backproject_bst")
        return out

    def backproject_bst_windowed(self, sino: torch.Tensor, beta: float, oversampling: int = 1,
                                 out: torch.Tensor | None = None) -> torch.Tensor:
        """The paper's BST algorithm on Kaiser-Bessel-windowed semi-polar half-lines (Section 5.3
        Steps 1-4 with Step 2.1 and eq "w", bp_backproject_bst_windowed): an accuracy variant,
        R* of the windowed projections; beta >= 0 (0 = no window)."""
        _cuda(sino, "sino")
        b = self._batch(sino, (self.n_theta, self.n_det), "sino")
        if sino.dtype not in _DTYPES:
            raise BPError(f"unsupported sinogram dtype {sino.dtype}")
        if out is None:
            out = torch.empty((*sino.shape[:-2], self.N, self.N), dtype=torch.float32, device=sino.device)
        _cuda(out, "out")
        if out.dtype != torch.float32 or out.numel() != b * self.N * self.N:
            raise BPError("out must be float32 with batch x N x N elements")
        with torch.cuda.device(self.device):
            _check(lib().bp_backproject_bst_windowed(self.handle, sino.data_ptr(), _DTYPES[sino.dtype],
                                                     out.data_ptr(), int(oversampling), float(beta), b,
                                                     _stream(sino)), "bp_backproject_bst_windowed")
        return out

    def backproject_logpolar_partial(self, sino: torch.Tensor, sectors: int = 8, a_r: float = 0.25,
                                     out: torch.Tensor | None = None) -> torch.Tensor:
        """R* by partial (sector) log-polar backprojections with a shifted origin (Section 5.2,
        eq "sh_prop"; bp_backproject_logpolar_partial)."""
        _cuda(sino, "sino")
        b = self._batch(sino, (self.n_theta, self.n_det), "sino")
        if sino.dtype not in _DTYPES:
            raise BPError(f"unsupported sinogram dtype {sino.dtype}")
        if out is None:
            out = torch.empty((*sino.shape[:-2], self.N, self.N), dtype=torch.float32, device=sino.device)
        _cuda(out, "out")
        if out.dtype != torch.float32 or out.numel() != b * self.N * self.N:
            raise BPError("out must be float32 with batch x N x N elements")
        with torch.cuda.device(self.device):
            _check(lib().bp_backproject_logpolar_partial(self.handle, sino.data_ptr(), _DTYPES[sino.dtype],
                                                         out.data_ptr(), int(sectors), float(a_r), b,
                                                         _stream(sino)), "bp_backproject_logpolar_partial")
        return out

    def backproject_logpolar(self, sino: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """R* by Andersson's log-polar convolution (Sections 5.1-5.2, bp_backproject_logpolar)."""
        _cuda(sino, "sino")
        b = self._batch(sino, (self.n_theta, self.n_det), "sino")
        if sino.dtype not in _DTYPES:
            raise BPError(f"unsupported sinogram dtype {sino.dtype}")
        if out is None:
            out = torch.empty((*sino.shape[:-2], self.N, self.N), dtype=torch.float32, device=sino.device)
        _cuda(out, "out")
        if out.dtype != torch.float32 or out.numel() != b * self.N * self.N:
            raise BPError("out must be float32 with batch x N x N elements")
        with torch.cuda.device(self.device):
            _check(lib().bp_backproject_logpolar(self.handle, sino.data_ptr(), _DTYPES[sino.dtype], out.data_ptr(),
                                                 b, _stream(sino)), "bp_backproject_logpolar")
        return out

    def set_fourier_width(self, width: int) -> None:
        """Kaiser-Bessel width (6 or 4 grid cells) of the Fourier path's gridding."""
        with torch.cuda.device(self.device):
            _check(lib().bp_set_fourier_width(self.handle, int(width)), "bp_set_fourier_width")

    def set_direct_workspace(self, nbytes: int) -> None:
        """Upper bound in bytes on the four-image direct R*'s row-table workspace (0: a quarter
        of the free device memory); batches beyond it run in chunks."""
        with torch.cuda.device(self.device):
            _check(lib().bp_set_direct_workspace(self.handle, int(nbytes)), "bp_set_direct_workspace")

    def fbp_fourier(self, sino: torch.Tensor, kind: str | int = "ramlak", param: float = 0.0,
                    out: torch.Tensor | None = None) -> torch.Tensor:
        """Filtered backprojection in the Fourier form with the filter fused into the
        projection transforms (bp_fbp_fourier); equals filter() then backproject_fourier()."""
        _cuda(sino, "sino")
        b = self._batch(sino, (self.n_theta, self.n_det), "sino")
        if sino.dtype not in _DTYPES:
            raise BPError(f"unsupported sinogram dtype {sino.dtype}")
        k = FILTERS[kind] if isinstance(kind, str) else int(kind)
        if out is None:
            out = torch.empty((*sino.shape[:-2], self.N, self.N), dtype=torch.float32, device=sino.device)
        _cuda(out, "out")
        if out.dtype != torch.float32 or out.numel() != b * self.N * self.N:
            raise BPError("out must be float32 with batch x N x N elements")
        with torch.cuda.device(self.device):
            _check(lib().bp_fbp_fourier(self.handle, sino.data_ptr(), _DTYPES[sino.dtype], out.data_ptr(), k,
                                        float(param), b, _stream(sino)), "bp_fbp_fourier")
        return out

    def fbp_direct(self, sino: torch.Tensor, kind: str | int = "ramlak", param: float = 0.0,
                   out: torch.Tensor | None = None) -> torch.Tensor:
        """Filtered backprojection in the direct form (bp_fbp_direct): filter() then backproject()
        of the float32 filtered rows, the filter writing the four-image form's row tables
        directly where that form runs."""
        _cuda(sino, "sino")
        b = self._batch(sino, (self.n_theta, self.n_det), "sino")
        if sino.dtype not in _DTYPES:
            raise BPError(f"unsupported sinogram dtype {sino.dtype}")
        k = FILTERS[kind] if isinstance(kind, str) else int(kind)
        if out is None:
            out = torch.empty((*sino.shape[:-2], self.N, self.N), dtype=torch.float32, device=sino.device)
        _cuda(out, "out")
        if out.dtype != torch.float32 or out.numel() != b * self.N * self.N:
            raise BPError("out must be float32 with batch x N x N elements")
        with torch.cuda.device(self.device):
            _check(lib().bp_fbp_direct(self.handle, sino.data_ptr(), _DTYPES[sino.dtype], out.data_ptr(), k,
                                       float(param), b, _stream(sino)), "bp_fbp_direct")
        return out

    def radon(self, img: torch.Tensor, out: torch.Tensor | None = None, fourier: bool = False) -> torch.Tensor:
        """R as the scaled transpose of the direct (or Fourier) R* (eqs "P_theta", "adjoint")."""
        _cuda(img, "img")
        b = self._batch(img, (self.N, self.N), "img")
        if img.dtype != torch.float32:
            raise BPError("img must be float32")
        if out is None:
            out = torch.empty((*img.shape[:-2], self.n_theta, self.n_det), dtype=torch.float32, device=img.device)
        _cuda(out, "out")
        if out.dtype != torch.float32 or out.numel() != b * self.n_theta * self.n_det:
            raise BPError("out must be float32 with batch x n_theta x n_det elements")
        with torch.cuda.device(self.device):
            _check(lib().bp_radon(self.handle, img.data_ptr(), out.data_ptr(), b, int(bool(fourier)), _stream(img)),
                   "bp_radon")
        return out

    def radon_transpose(self, sino: torch.Tensor, out: torch.Tensor | None = None,
                        fourier: bool = False) -> torch.Tensor:
        """R^T sino: exact Euclidean transpose of radon() (bp_radon_transpose)."""
        _cuda(sino, "sino")
        b = self._batch(sino, (self.n_theta, self.n_det), "sino")
        if sino.dtype != torch.float32:
            raise BPError("sino must be float32")
        if out is None:
            out = torch.empty((*sino.shape[:-2], self.N, self.N), dtype=torch.float32, device=sino.device)
        _cuda(out, "out")
        if out.dtype != torch.float32 or out.numel() != b * self.N * self.N:
            raise BPError("out must be float32 with batch x N x N elements")
        with torch.cuda.device(self.device):
            _check(lib().bp_radon_transpose(self.handle, sino.data_ptr(), out.data_ptr(), b, int(bool(fourier)),
                                            _stream(sino)), "bp_radon_transpose")
        return out

    def backproject_transpose(self, img: torch.Tensor, out: torch.Tensor | None = None,
                              fourier: bool = False) -> torch.Tensor:
        """A^T img: exact Euclidean transpose of backproject() / backproject_fourier()."""
        _cuda(img, "img")
        b = self._batch(img, (self.N, self.N), "img")
        if img.dtype != torch.float32:
            raise BPError("img must be float32")
        if out is None:
            out = torch.empty((*img.shape[:-2], self.n_theta, self.n_det), dtype=torch.float32, device=img.device)
        _cuda(out, "out")
        if out.dtype != torch.float32 or out.numel() != b * self.n_theta * self.n_det:
            raise BPError("out must be float32 with batch x n_theta x n_det elements")
        with torch.cuda.device(self.device):
            _check(lib().bp_backproject_transpose(self.handle, img.data_ptr(), out.data_ptr(), b,
                                                  int(bool(fourier)), _stream(img)), "bp_backproject_transpose")
        return out

    def fbp_host(self, sino: torch.Tensor, kind: str | int = "ramlak", param: float = 0.0,
                 out: torch.Tensor | None = None) -> torch.Tensor:
        """Filtered backprojection from host float32 memory to host float32 memory (bp_fbp_host)."""
        if sino.is_cuda or sino.dtype != torch.float32 or not sino.is_contiguous():
            raise BPError("sino must be a contiguous float32 CPU tensor")
        b = int(math.prod(sino.shape[:-2])) if sino.dim() > 2 else 1
        if tuple(sino.shape[-2:]) != (self.n_theta, self.n_det):
            raise BPError("sino shape mismatch")
        if out is None:
            out = torch.empty((*sino.shape[:-2], self.N, self.N), dtype=torch.float32,
                              pin_memory=sino.is_pinned())
        k = FILTERS[kind] if isinstance(kind, str) else int(kind)
        with torch.cuda.device(self.device):
            _check(lib().bp_fbp_host(self.handle, sino.data_ptr(), out.data_ptr(), k, float(param), b,
                                     torch.cuda.current_stream(self.device).cuda_stream), "bp_fbp_host")
        return out

    def check(self) -> None:
        """Synchronise the current stream; raise if a device-side bounded wait gave up (bp_check)."""
        with torch.cuda.device(self.device):
            _check(lib().bp_check(self.handle, torch.cuda.current_stream(self.device).cuda_stream), "bp_check")

    # ------------------------------------------------------------------ launch shapes
    @staticmethod
    def _op_dtype(op: str, dtype) -> tuple[int, int]:
        if op not in OPS:
            raise BPError(f"op must be one of {sorted(OPS)}")
        if isinstance(dtype, torch.dtype):
            if dtype not in _DTYPES:
                raise BPError(f"unsupported dtype {dtype}")
            dtype = _DTYPES[dtype]
        return OPS[op], int(dtype)

    def autotune(self, op: str = "direct", dtype=torch.float32, batch: int = 1) -> tuple[tuple[int, int], float]:
        """Time the candidate launch shapes of op ("direct" R* or "radon" R) and keep the
        fastest for calls with this (dtype, batch); returns (shape, milliseconds)."""
        o, d = self._op_dtype(op, dtype)
        shape = (ctypes.c_int * 2)()
        ms = ctypes.c_float()
        with torch.cuda.device(self.device):
            _check(lib().bp_autotune(self.handle, o, d, int(batch), torch.cuda.current_stream(self.device).cuda_stream,
                                     shape, ctypes.byref(ms)), "bp_autotune")
        return (shape[0], shape[1]), float(ms.value)

    def get_shape(self, op: str = "direct", dtype=torch.float32, batch: int = 1) -> tuple[int, int]:
        """Launch shape (after clamping) a call (op, dtype, batch) uses now."""
        o, d = self._op_dtype(op, dtype)
        shape = (ctypes.c_int * 2)()
        with torch.cuda.device(self.device):
            _check(lib().bp_get_shape(self.handle, o, d, int(batch), shape), "bp_get_shape")
        return shape[0], shape[1]

    def set_shape(self, shape: tuple[int, int], op: str = "direct", dtype=torch.float32, batch: int = 1) -> None:
        """Fix the launch shape of calls (op, dtype, batch) on this plan."""
        o, d = self._op_dtype(op, dtype)
        arr = (ctypes.c_int * 2)(int(shape[0]), int(shape[1]))
        with torch.cuda.device(self.device):
            _check(lib().bp_set_shape(self.handle, o, d, int(batch), arr), "bp_set_shape")

    def stage_timing(self, on: bool = True) -> None:
        """Start (or stop) recording a CUDA event after every kernel of this plan's calls."""
        _check(lib().bp_stage_timing(self.handle, 1 if on else 0), "bp_stage_timing")

    def stage_times(self) -> dict[str, tuple[float, int]]:
        """Per kernel name: (summed milliseconds, launches) since the last read (waits for them)."""
        cap = 64
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_float * cap)()
        launches = (ctypes.c_int * cap)()
        count = ctypes.c_int(0)
        _check(lib().bp_stage_times(self.handle, cap, names, ms, launches, ctypes.byref(count)), "bp_stage_times")
        return {names[j].decode(): (float(ms[j]), int(launches[j])) for j in range(min(cap, count.value))}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            lib().bp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def backproject_batched(plans: Sequence[Plan], sinos: Sequence[torch.Tensor],
                        imgs: Sequence[torch.Tensor] | None = None) -> list[torch.Tensor]:
    """R* of independent slices with (possibly) different geometries in one persistent launch."""
    n = len(plans)
    if n == 0 or len(sinos) != n:
        raise BPError("plans and sinos must be non-empty and of equal length")
    if imgs is None:
        imgs = [torch.empty((p.N, p.N), dtype=torch.float32, device=s.device) for p, s in zip(plans, sinos)]
    for p, s, o in zip(plans, sinos, imgs):
        _cuda(s, "sino")
        _cuda(o, "img")
        if tuple(s.shape[-2:]) != (p.n_theta, p.n_det) or s.numel() != p.n_theta * p.n_det:
            raise BPError("each sinogram must be one n_theta x n_det slice")
        if o.numel() != p.N * p.N or o.dtype != torch.float32:
            raise BPError("each image must be one float32 N x N slice")
        if s.dtype not in _DTYPES:
            raise BPError(f"unsupported sinogram dtype {s.dtype}")
    vp = ctypes.c_void_p
    P = (vp * n)(*[p.handle.value for p in plans])
    S = (vp * n)(*[s.data_ptr() for s in sinos])
    D = (ctypes.c_int * n)(*[_DTYPES[s.dtype] for s in sinos])
    O = (vp * n)(*[o.data_ptr() for o in imgs])
    with torch.cuda.device(plans[0].device):
        _check(lib().bp_backproject_batched(P, S, D, O, n, _stream(sinos[0])), "bp_backproject_batched")
    return list(imgs)


def tune_cache_save(path: str) -> None:
    """Write the process-wide tuning cache (bp_tune_cache_save)."""
    _check(lib().bp_tune_cache_save(os.fsencode(path)), "bp_tune_cache_save")


def tune_cache_load(path: str) -> None:
    """Merge a tuning cache file into the process-wide cache (bp_tune_cache_load)."""
    _check(lib().bp_tune_cache_load(os.fsencode(path)), "bp_tune_cache_load")
