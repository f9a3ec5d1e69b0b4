"""FP64 oracle of the paper's BST algorithm on semi-polar half-lines with the Kaiser-Bessel
window of eq "w" (Section 5.3, Steps 1-4 with Step 2.1; the theorem is eq "bst" of Section
3, the kernel K^sigma at the origin eq "kernel"; the polar mesh {s_k} and G_P of the table of
symbols, Section 5).

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU baseline).  Plain
numpy in double precision; numpy's FFT and modified Bessel function I0 are the only library
primitives.

Steps, in the paper's order (image [-1, 1]^2, N pixels, dx = 2/N; detector centres t_j =
(j - (n_det-1)/2) dt; theta_k in [0, pi)):

Step 1   The sinogram becomes the semi-polar half-lines s >= 0 at phi in [0, 2 pi): for each
         projection the ray phi = theta_k carries g(s, theta_k) and the ray theta_k + pi
         carries g(-s, theta_k) (Section 1: g(-s, theta) = g(s, theta + pi)).  They are
         sampled on the polar mesh s_i = i ds, ds = dt, i = 0 .. N_s - 1, N_s = floor(n_det/2)
         + 1 (the mesh reaches the last detector centre), by linear interpolation between
         detector centres (zero off the detector).
Step 2.1 Each half-line is multiplied by the window of eq "w",
             w_i = I0(beta sqrt(1 - ((2 i - N_s + 1) / (N_s - 1))^2)) / I0(beta),
         which tapers both ends of the half-line (s = 0 and s = s_max), beta >= 0 a
         parameter (the paper gives no value; beta = 0 is the identity).  The sample at s = 0
         is shared by the two half-lines of a projection; each takes half of it, so that the
         two one-sided transforms add up to the transform of the full line.
Step 2.2 One-sided transform of each half-line: H_phi(kappa_m) = ds sum_i c_i w_i h_i
         e^{-2 pi i m i / P} at kappa_m = m / (P ds), m < P/2 (c_0 = 1/2, c_i = 1 otherwise),
         P = 2^ceil(log2(2 n_det)) (the full-line form's transform length, so both forms share
         the frequency mesh).
Step 2.3 Times K^sigma = 1/|kappa| (1/dkappa at kappa = 0), eq "kernel".  The BST (eq
         "bst") relates the backprojection's transform to the transform of a full line; a
         one-sided transform alone is the transform of no projection.  With real data the
         line through the half-lines phi and phi + pi has the transform H_phi + conj H_{phi+pi}
         at kappa >= 0 (in the direction of phi), so ray phi carries
         (H_phi + conj H_{phi+pi}) K^sigma.
Step 3   Linear polar-to-Cartesian interpolation on the 2 n_theta rays
         (bst_interp.cartesian_grid_rays).
Step 4   b = Re (1/(M dx))^2 sum_l bhat(l) e^{2 pi i l . x / (M dx)} at the pixel centres.

With beta = 0 and odd n_det (half-line samples on detector centres) this is exactly the
full-line algorithm of bst_interp.bp_bst_interp; with beta > 0 it is that algorithm applied
to the windowed full lines g(t, theta) w(|t|) (the window alters the result: it is the
paper's accuracy variant, not R*).
"""
from __future__ import annotations

import math

import numpy as np

from .bst_interp import _pad, cartesian_grid_rays, grid_size


def halfline_count(n_det: int) -> int:
    """N_s: samples s_i = i ds, i < N_s, on each half-line (the polar mesh {s_k})."""
    return n_det // 2 + 1


def kb_window(n_s: int, beta: float) -> np.ndarray:
    """Step 2.1: the Kaiser-Bessel window of eq "w" on the N_s half-line samples."""
    if n_s == 1:
        return np.ones(1)
    i = np.arange(n_s, dtype=np.float64)
    x = (2.0 * i - n_s + 1.0) / (n_s - 1.0)
    return np.i0(beta * np.sqrt(np.clip(1.0 - x * x, 0.0, None))) / np.i0(beta)


def semipolar_rows(g, det_spacing: float) -> tuple[np.ndarray, np.ndarray]:
    """Step 1: (h_plus, h_minus) [n_theta][N_s], g at t = +s_i and t = -s_i by linear
    interpolation between detector centres (zero off the detector)."""
    g = np.asarray(g, dtype=np.float64)
    n_det = g.shape[-1]
    n_s = halfline_count(n_det)
    s_idx = np.arange(n_s, dtype=np.float64)  # s_i / dt

    def at(u):  # g at fractional detector index u, per row
        j = np.floor(u).astype(np.int64)
        f = u - j
        v0 = np.where((j >= 0) & (j < n_det), g[:, np.clip(j, 0, n_det - 1)], 0.0)
        v1 = np.where((j + 1 >= 0) & (j + 1 < n_det), g[:, np.clip(j + 1, 0, n_det - 1)], 0.0)
        return (1.0 - f) * v0 + f * v1

    c = 0.5 * (n_det - 1)
    return at(c + s_idx), at(c - s_idx)


def halfline_values(h: np.ndarray, w: np.ndarray, det_spacing: float, P: int) -> np.ndarray:
    """Steps 2.1-2.3 for half-lines h [rays][N_s]: K^sigma times the one-sided transform."""
    n_s = h.shape[-1]
    c = np.ones(n_s)
    c[0] = 0.5
    H = P // 2
    T = np.fft.fft(h * (c * w)[None, :], n=P, axis=-1)[..., :H] * det_spacing
    m = np.arange(H, dtype=np.float64)
    dkappa = 1.0 / (P * det_spacing)
    K = np.where(m > 0, 1.0 / (np.maximum(m, 1.0) * dkappa), 1.0 / dkappa)
    return T * K


def bp_bst_semipolar(g, N: int, theta, det_spacing: float, beta: float, M: int | None = None,
                     P: int | None = None) -> np.ndarray:
    """The paper's BST algorithm on the windowed semi-polar half-lines (Steps 1-4), image [N][N]."""
    g = np.asarray(g, dtype=np.float64)
    n_theta, n_det = g.shape
    M = grid_size(N) if M is None else int(M)
    P = _pad(n_det) if P is None else int(P)
    dx = 2.0 / N
    hp, hm = semipolar_rows(g, det_spacing)
    w = kb_window(hp.shape[-1], beta)
    Vp = halfline_values(hp, w, det_spacing, P)
    Vm = halfline_values(hm, w, det_spacing, P)
    th = np.mod(np.asarray(theta, dtype=np.float64), 2.0 * math.pi)
    ang = np.concatenate([th, np.mod(th + math.pi, 2.0 * math.pi)])
    V = np.concatenate([Vp + np.conj(Vm), Vm + np.conj(Vp)])
    order = np.argsort(ang, kind="stable")
    grid = cartesian_grid_rays(ang[order], V[order], N, det_spacing, M, P)
    delta = (N // 2) - (N - 1) / 2.0
    l = np.fft.fftfreq(M, 1.0 / M)
    ph = np.exp(2j * math.pi * delta * l / M)
    Wg = grid * ph[:, None] * ph[None, :] / (M * dx) ** 2
    full = (np.fft.ifft2(Wg) * (M * M)).real
    idx = (np.arange(N) - N // 2) % M
    return np.ascontiguousarray(full[np.ix_(idx, idx)].T)  # img[i_y][i_x]
