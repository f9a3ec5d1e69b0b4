"""Seeded synthetic workloads: random-ellipse phantoms and their analytic sinograms.

This module only *generates inputs*; it holds none of the backprojection, Radon or
filter arithmetic.  It is the one module that both the FP64 oracle tests and the
CUDA path use, so the two see identical data.

Geometry (shared convention, stated here once):
  * image domain [-1, 1]^2 sampled by N x N pixels, pixel centres
    x_i = -1 + (i + 1/2) * (2/N); image array img[iy][ix], y along rows;
  * detector centres t_j = (j - (n_det - 1)/2) * det_spacing, default spacing 2/n_det
    (sinogram grid of Table "tab:symbols", Section 5);
  * sinogram array g[k][j] = projection at angle theta_k, detector bin j.

Phantoms follow the workload recipe of the benchmark configurations: ellipse centres
area-uniform in a disk of radius 0.7, semi-axes U[0.05, 0.4], rotation U[0, pi),
density U[-1, 1]; numpy PCG64 seeded per slice.  The sinogram of an ellipse is its
exact line integral (Radon transform, Section 1, eq "P_theta"), sampled at detector
centres.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def uniform_theta(n_theta: int) -> np.ndarray:
    """theta_k = k * pi / n_theta, k = 0..n_theta-1 (Table "tab:symbols": dtheta = pi/N_theta)."""
    return np.arange(n_theta, dtype=np.float64) * (math.pi / n_theta)


def default_det_spacing(n_det: int) -> float:
    """dt = 2 / N_t (Table "tab:symbols")."""
    return 2.0 / n_det


@dataclass(frozen=True)
class Ellipses:
    cx: np.ndarray
    cy: np.ndarray
    a: np.ndarray      # semi-axis along the rotated x' axis
    b: np.ndarray      # semi-axis along the rotated y' axis
    alpha: np.ndarray  # rotation angle
    rho: np.ndarray    # density

    def __len__(self) -> int:
        return int(self.cx.shape[0])


def random_ellipses(n: int, seed: int, radius: float = 0.7,
                    axes: tuple[float, float] = (0.05, 0.4)) -> Ellipses:
    rng = np.random.Generator(np.random.PCG64(seed))
    r = radius * np.sqrt(rng.uniform(0.0, 1.0, n))
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    a = rng.uniform(axes[0], axes[1], n)
    b = rng.uniform(axes[0], axes[1], n)
    alpha = rng.uniform(0.0, math.pi, n)
    rho = rng.uniform(-1.0, 1.0, n)
    return Ellipses(r * np.cos(phi), r * np.sin(phi), a, b, alpha, rho)


def ellipse_sinogram(e: Ellipses, theta: np.ndarray, n_det: int,
                     det_spacing: float | None = None) -> np.ndarray:
    """Exact line integrals of the ellipse phantom, g[k][j] in float64.

    For one ellipse (centre c, semi-axes a, b, rotation alpha, density rho) the chord
    length along the line x . xi_theta = t is 2ab sqrt(A^2 - t'^2) / A^2 with
    A^2 = a^2 cos^2(theta - alpha) + b^2 sin^2(theta - alpha) and t' = t - c . xi_theta.
    """
    dt = default_det_spacing(n_det) if det_spacing is None else float(det_spacing)
    theta = np.asarray(theta, dtype=np.float64)
    t = (np.arange(n_det, dtype=np.float64) - (n_det - 1) / 2.0) * dt
    g = np.zeros((theta.shape[0], n_det), dtype=np.float64)
    ct = np.cos(theta)[:, None]
    st = np.sin(theta)[:, None]
    for i in range(len(e)):
        th = theta[:, None] - e.alpha[i]
        A2 = (e.a[i] * np.cos(th)) ** 2 + (e.b[i] * np.sin(th)) ** 2
        tp = t[None, :] - (e.cx[i] * ct + e.cy[i] * st)
        rad = A2 - tp * tp
        mask = rad > 0
        chord = np.zeros_like(rad)
        chord[mask] = 2.0 * e.a[i] * e.b[i] * np.sqrt(rad[mask]) / np.broadcast_to(A2, rad.shape)[mask]
        g += e.rho[i] * chord
    return g


def ellipse_image(e: Ellipses, N: int, supersample: int = 1) -> np.ndarray:
    """Point-sampled (optionally supersampled box-averaged) phantom image [N][N] float64."""
    s = int(supersample)
    dx = 2.0 / N
    off = (np.arange(s) + 0.5) / s - 0.5
    xs = (-1.0 + (np.arange(N)[:, None] + 0.5 + off[None, :]) * dx).reshape(-1)
    X = xs[None, :]
    Y = xs[:, None]
    img = np.zeros((N * s, N * s), dtype=np.float64)
    for i in range(len(e)):
        ca, sa = math.cos(e.alpha[i]), math.sin(e.alpha[i])
        xr = (X - e.cx[i]) * ca + (Y - e.cy[i]) * sa
        yr = -(X - e.cx[i]) * sa + (Y - e.cy[i]) * ca
        img += e.rho[i] * ((xr / e.a[i]) ** 2 + (yr / e.b[i]) ** 2 <= 1.0)
    if s > 1:
        img = img.reshape(N, s, N, s).mean(axis=(1, 3))
    return img


def add_gaussian_noise(g: np.ndarray, frac: float, seed: int) -> np.ndarray:
    """g + N(0, (frac * max|g|)^2), seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sigma = frac * float(np.max(np.abs(g)))
    return g + rng.normal(0.0, sigma, g.shape)


def circ_sinogram(theta: np.ndarray, n_det: int, det_spacing: float | None = None) -> np.ndarray:
    """Sinogram of circ(|x|) (Section 4, Example II): g(t, theta) = 2 sqrt(1 - t^2) for |t| <= 1."""
    dt = default_det_spacing(n_det) if det_spacing is None else float(det_spacing)
    t = (np.arange(n_det, dtype=np.float64) - (n_det - 1) / 2.0) * dt
    row = np.where(np.abs(t) <= 1.0, 2.0 * np.sqrt(np.clip(1.0 - t * t, 0.0, None)), 0.0)
    return np.repeat(row[None, :], len(theta), axis=0)


@dataclass(frozen=True)
class Workload:
    """One benchmark-shaped slice: geometry plus the phantom recipe."""
    name: str
    N: int
    n_det: int
    n_theta: int
    n_ellipses: int
    noise_frac: float
    seed: int

    @property
    def theta(self) -> np.ndarray:
        return uniform_theta(self.n_theta)

    @property
    def det_spacing(self) -> float:
        return default_det_spacing(self.n_det)

    @property
    def updates(self) -> int:
        return self.N * self.N * self.n_theta

    def sinogram(self, slice_id: int = 0) -> np.ndarray:
        e = random_ellipses(self.n_ellipses, self.seed + slice_id)
        g = ellipse_sinogram(e, self.theta, self.n_det, self.det_spacing)
        if self.noise_frac > 0:
            g = add_gaussian_noise(g, self.noise_frac, self.seed + 500 + slice_id)
        return g


# Single slice, 256^2 image, 256 bins, 180 angles, 10 ellipses (Ram-Lak filtered in use).
SMALL = Workload("slice256_bins256_ang180", 256, 256, 180, 10, 0.0, 1000)
# Single slice, 2048^2 image, 2048 bins, 1800 angles, 50 ellipses + 1% noise (Shepp-Logan).
LARGE = Workload("slice2048_bins2048_ang1800", 2048, 2048, 1800, 50, 0.01, 2000)


def ellipse_sinogram_torch(e: Ellipses, theta: np.ndarray, n_det: int, det_spacing: float | None = None,
                           device="cuda"):
    """ellipse_sinogram evaluated with torch in float64 on `device` (same formula, for large batches)."""
    import torch

    dt = default_det_spacing(n_det) if det_spacing is None else float(det_spacing)
    th = torch.as_tensor(np.asarray(theta, dtype=np.float64), device=device)
    t = (torch.arange(n_det, dtype=torch.float64, device=device) - (n_det - 1) / 2.0) * dt
    g = torch.zeros((th.shape[0], n_det), dtype=torch.float64, device=device)
    ct = torch.cos(th)[:, None]
    st = torch.sin(th)[:, None]
    for i in range(len(e)):
        a, b = float(e.a[i]), float(e.b[i])
        ang = th[:, None] - float(e.alpha[i])
        A2 = (a * torch.cos(ang)) ** 2 + (b * torch.sin(ang)) ** 2
        tp = t[None, :] - (float(e.cx[i]) * ct + float(e.cy[i]) * st)
        rad = torch.clamp(A2 - tp * tp, min=0.0)
        g += float(e.rho[i]) * (2.0 * a * b) * torch.sqrt(rad) / A2
    return g


# 256 slices of 2048^2 from 2048 bins x 1800 angles, BF16 storage, 30 ellipses per slice.
VOLUME = Workload("volume256_slice2048_bins2048_ang1800_bf16", 2048, 2048, 1800, 30, 0.0, 3000)
VOLUME_SLICES = 256


# Single high-resolution slice: 8192^2 image, 8192 bins, 6000 angles, 30 ellipses.
HIRES = Workload("slice8192_bins8192_ang6000", 8192, 8192, 6000, 30, 0.0, 5999)


def mixed_batch_geometries(n: int = 64, seed: int = 5000):
    """Uneven batch: image side = detector width drawn from {512, 1024, 2048, 4096}, angle
    counts uniform in [360, 3000] (uniform angles on [0, pi))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = rng.choice([512, 1024, 2048, 4096], size=n)
    angles = rng.integers(360, 3001, size=n)
    return [(int(s), int(s), int(a)) for s, a in zip(sizes, angles)]
