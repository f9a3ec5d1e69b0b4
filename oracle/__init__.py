"""FP64 CPU oracle for the discretised backprojection R*, its transpose R, the FBP filter
and the Fourier-path (band-limited) backprojection.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU
baseline are the only callers.  The oracle shares no code with the CUDA path; the
arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over outputs), and
this module only builds it with gcc and marshals numpy arrays.  The one library
primitive used here is numpy's FFT, to form the projection spectra G_k[m] that the
spectral Fourier-path oracle sums (Section 5.3, Step 2.2).

Each wrapped function cites the passage of arXiv:1608.03589 it follows in oracle.c.  The
paper's own BST algorithm (polar-to-Cartesian interpolation in frequency) is plain numpy in
``bst_interp.py`` (``bp_bst_interp`` below), the same algorithm on windowed semi-polar
half-lines in ``bst_semipolar.py`` (``bp_bst_semipolar``), Andersson's log-polar
backprojection in ``logpolar.py`` (``bp_logpolar``) and its partial (sector) form in
``logpolar_partial.py`` (``bp_logpolar_partial``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

RAMLAK, SHEPP_LOGAN, TIKHONOV = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2 -fopenmp); returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            lp = ctypes.POINTER(ctypes.c_long)
            i, d = ctypes.c_int, ctypes.c_double
            sig = {
                "oracle_num_threads": ([], i),
                "oracle_set_threads": ([i], None),
                "oracle_weights": ([i, dp, dp], i),
                "oracle_bp_linear": ([i, i, i, dp, d, dp, dp], i),
                "oracle_bp_linear_points": ([i, i, i, dp, d, dp, i, lp, dp], i),
                "oracle_radon": ([i, i, i, dp, d, dp, dp], i),
                "oracle_filter_kernel": ([i, d, i, d, dp], i),
                "oracle_filter": ([i, i, d, i, d, dp, dp], i),
                "oracle_bp_trig_dirichlet": ([i, i, i, dp, d, i, dp, dp], i),
                "oracle_bp_trig_points": ([i, i, i, dp, d, i, dp, dp, i, lp, dp], i),
                "oracle_radon_trig_points": ([i, i, i, dp, d, i, dp, i, lp, dp], i),
            }
            for name, (args, res) in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _l(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"{name} failed with code {rc}")


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def fourier_pad(n_det: int) -> int:
    """P: smallest power of two >= 2 n_det (zero padding of each projection row)."""
    P = 1
    while P < 2 * n_det:
        P *= 2
    return P


def weights(theta) -> np.ndarray:
    """Quadrature weights w_k of eq "bp_app" (Section 2), gap-based for any angle set."""
    th, thp = _d(theta)
    w = np.empty_like(th)
    _check(_load().oracle_weights(th.shape[0], thp, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "weights")
    return w


def bp_linear(g, N: int, theta, det_spacing: float) -> np.ndarray:
    """R* with linear interpolation (Section 2, eq "bp_app").  g: [n_theta][n_det] -> [N][N]."""
    g, gp = _d(g)
    th, thp = _d(theta)
    n_theta, n_det = g.shape
    assert th.shape[0] == n_theta
    b = np.empty((N, N), dtype=np.float64)
    _check(_load().oracle_bp_linear(N, n_det, n_theta, thp, float(det_spacing), gp,
                                    b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "bp_linear")
    return b


def bp_linear_points(g, N: int, theta, det_spacing: float, pix) -> np.ndarray:
    """R* (Section 2, eq "bp_app") at the listed flat pixel indices iy*N + ix."""
    g, gp = _d(g)
    th, thp = _d(theta)
    pix, pp = _l(pix)
    n_theta, n_det = g.shape
    out = np.empty(pix.shape[0], dtype=np.float64)
    _check(_load().oracle_bp_linear_points(N, n_det, n_theta, thp, float(det_spacing), gp, pix.shape[0], pp,
                                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "bp_linear_points")
    return out


def radon(f, n_det: int, theta, det_spacing: float) -> np.ndarray:
    """R = (dx^2/dt) diag(1/w) A^T, the scaled transpose of bp_linear (eq "adjoint")."""
    f, fp = _d(f)
    th, thp = _d(theta)
    N = f.shape[0]
    assert f.shape == (N, N)
    g = np.empty((th.shape[0], n_det), dtype=np.float64)
    _check(_load().oracle_radon(N, n_det, th.shape[0], thp, float(det_spacing), fp,
                                g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "radon")
    return g


def filter_kernel(n_det: int, det_spacing: float, kind: int, param: float = 0.0) -> np.ndarray:
    """Spatial filter taps h(n), n = -(n_det-1)..(n_det-1) (Section 3 eq "fbp"; Section 6)."""
    h = np.empty(2 * n_det - 1, dtype=np.float64)
    _check(_load().oracle_filter_kernel(n_det, float(det_spacing), int(kind), float(param),
                                        h.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "filter_kernel")
    return h


def filter_rows(g, det_spacing: float, kind: int, param: float = 0.0) -> np.ndarray:
    """q_j = dt sum_i h(j - i) g_i per row (linear convolution), FP64 direct sum."""
    g, gp = _d(g)
    rows, n_det = g.reshape(-1, g.shape[-1]).shape
    q = np.empty_like(g)
    _check(_load().oracle_filter(rows, n_det, float(det_spacing), int(kind), float(param), gp,
                                 q.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "filter")
    return q


def bp_trig_dirichlet(g, N: int, theta, det_spacing: float, P: int | None = None) -> np.ndarray:
    """Fourier-path backprojection by the spatial Dirichlet-kernel sum (small sizes only)."""
    g, gp = _d(g)
    th, thp = _d(theta)
    n_theta, n_det = g.shape
    P = fourier_pad(n_det) if P is None else int(P)
    b = np.empty((N, N), dtype=np.float64)
    _check(_load().oracle_bp_trig_dirichlet(N, n_det, n_theta, thp, float(det_spacing), P, gp,
                                            b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "bp_trig_dirichlet")
    return b


def half_spectra(g, P: int) -> np.ndarray:
    """G_k[m] = sum_j g_kj exp(-2 pi i m j / P), m = 0..P/2-1 (numpy FFT of the zero-padded rows)."""
    G = np.fft.rfft(np.asarray(g, dtype=np.float64), n=P, axis=-1)
    return G[..., : P // 2]


def bp_trig_points(g, N: int, theta, det_spacing: float, pix, P: int | None = None) -> np.ndarray:
    """Fourier-path backprojection at listed pixels from the projection spectra."""
    g = np.asarray(g, dtype=np.float64)
    n_theta, n_det = g.shape
    P = fourier_pad(n_det) if P is None else int(P)
    G = half_spectra(g, P)
    re, rp = _d(G.real)
    im, ip = _d(G.imag)
    th, thp = _d(theta)
    pix, pp = _l(pix)
    out = np.empty(pix.shape[0], dtype=np.float64)
    _check(_load().oracle_bp_trig_points(N, n_det, n_theta, thp, float(det_spacing), P, rp, ip, pix.shape[0], pp,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "bp_trig_points")
    return out


def radon_trig_points(f, n_det: int, theta, det_spacing: float, kj, P: int | None = None) -> np.ndarray:
    """Transpose of the Fourier-path operator at listed (k*n_det + j) sinogram entries."""
    f, fp = _d(f)
    th, thp = _d(theta)
    kj, kp = _l(kj)
    N = f.shape[0]
    P = fourier_pad(n_det) if P is None else int(P)
    out = np.empty(kj.shape[0], dtype=np.float64)
    _check(_load().oracle_radon_trig_points(N, n_det, th.shape[0], thp, float(det_spacing), P, fp, kj.shape[0], kp,
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "radon_trig_points")
    return out


def rel_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2 in float64."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / (nb if nb > 0 else 1.0)


from .bst_interp import bp_bst_interp, bst_full_period  # noqa: E402  (numpy oracle of Section 5.3)
from .logpolar import bp_logpolar  # noqa: E402  (numpy oracle of Sections 5.1-5.2)
from .bst_semipolar import bp_bst_semipolar  # noqa: E402  (numpy oracle of Section 5.3 with eq "w")
from .logpolar_partial import bp_logpolar_partial  # noqa: E402  (numpy oracle of Section 5.2, sectors)
