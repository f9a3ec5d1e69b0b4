"""FP64 oracle of the paper's own Backprojection-Slice-Theorem algorithm: frequency-domain
interpolation from the polar grid to a Cartesian grid (Section 5.3, Steps 1-4; the theorem
is eq "bst" of Section 3; the kernel K^sigma at the origin is eq "kernel").

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU baseline).  Plain
numpy in double precision; numpy's FFT is the only library primitive (Steps 2.2 and 4).

Steps, in the paper's order, in the conventions of the rest of the oracle (image [-1, 1]^2,
N pixels, dx = 2/N; detector centres t_j = (j - (n_det-1)/2) dt; theta_k in [0, pi)):

Step 1   The full lines t in R, theta in [0, pi) carry the same data as the semi-polar
         half-lines s >= 0, theta in [0, 2 pi) (g(-s, theta) = g(s, theta + pi), Section 1):
         every projection gives a ray theta_k and its opposite theta_k + pi.  Each row is
         zero-padded to P = 2^ceil(log2(2 n_det)); no s = 0 boundary arises, so the window
         of Step 2.1 (eq "w") is the identity.
Step 2.2 G_k[m] = sum_j g_kj exp(-2 pi i m j / P).  With kappa_m = m / (P dt) (cycles per
         unit length) the projection's transform is ghat_k(kappa_m) = dt e^{i pi m (n_det-1)/P}
         G_k[m], m = 0..P/2-1 (the Nyquist bin dropped); on the opposite ray the values are
         the complex conjugates (real projections).
Step 2.3 By the BST the backprojection's transform on the ray is bhat(kappa xi_k) =
         ghat_k(kappa) K^sigma(kappa) with K^sigma = 1/|kappa|, and 1/dkappa at kappa = 0
         (eq "kernel"; dkappa = 1/(P dt) is the radial step).
Step 3   The Cartesian frequency grid nu_l = l / (M dx), l in [-M/2, M/2)^2, M =
         max(2^ceil(log2(2N)), 64) (period M dx of the reconstructed image).  Each node takes the
         value interpolated linearly in radius (fractional sample index |nu_l| / dkappa) and
         linearly in angle between the two rays that bracket its polar angle (angles taken
         cyclically on [0, 2 pi)); samples at or beyond P/2 are zero.  The origin node
         belongs to every ray; it takes the mean of the rays' values there (the paper does
         not say which ray's value to use).
Step 4   b(x_i) = Re sum_l (1/(M dx))^2 bhat(nu_l) exp(2 pi i nu_l . x_i) -- a 2D inverse DFT
         of the grid (the Riemann sum of the inverse Fourier integral), at the N x N pixel
         centres x_i = (i - floor(N/2) + delta) dx, delta = floor(N/2) - (N-1)/2.

The result approximates R* of the band-limited projections; it is not the same
discretisation as the gridding form (which sums the polar samples exactly), and its
distance to that one is what this algorithm's accuracy means.
"""
from __future__ import annotations

import math

import numpy as np


def grid_size(N: int) -> int:
    """M: smallest power of two >= 2N, and at least 64 (the Cartesian frequency grid)."""
    M = 1
    while M < 2 * N:
        M *= 2
    return max(M, 64)


def _pad(n_det: int) -> int:
    P = 1
    while P < 2 * n_det:
        P *= 2
    return P


def polar_values(g, det_spacing: float, P: int) -> np.ndarray:
    """Steps 2.2-2.3: bhat on ray k at kappa_m, m = 0..P/2-1 (complex [n_theta][P/2])."""
    g = np.asarray(g, dtype=np.float64)
    n_det = g.shape[-1]
    H = P // 2
    G = np.fft.fft(g, n=P, axis=-1)[..., :H]
    m = np.arange(H, dtype=np.float64)
    ghat = det_spacing * np.exp(1j * math.pi * m * (n_det - 1) / P) * G
    dkappa = 1.0 / (P * det_spacing)
    K = np.where(m > 0, 1.0 / (np.maximum(m, 1.0) * dkappa), 1.0 / dkappa)
    return ghat * K


def full_circle_rays(theta) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Step 1: the 2 n_theta ray directions theta_k and theta_k + pi in [0, 2 pi), sorted;
    returns (angle, projection index, conjugate flag)."""
    th = np.mod(np.asarray(theta, dtype=np.float64), 2.0 * math.pi)
    n = th.shape[0]
    ang = np.concatenate([th, np.mod(th + math.pi, 2.0 * math.pi)])
    k = np.concatenate([np.arange(n), np.arange(n)])
    conj = np.concatenate([np.zeros(n, bool), np.ones(n, bool)])
    order = np.argsort(ang, kind="stable")
    return ang[order], k[order], conj[order]


def cartesian_grid_rays(ang: np.ndarray, V: np.ndarray, N: int, det_spacing: float, M: int, P: int) -> np.ndarray:
    """Step 3 for explicit rays: ang [R] sorted in [0, 2 pi), V [R][P/2] the values on each ray
    at kappa_m; returns the M x M grid indexed [l_x mod M][l_y mod M]."""
    H = P // 2
    dx = 2.0 / N
    rho = M * dx / (P * det_spacing)  # grid cells per radial sample
    R = ang.shape[0]
    out = np.zeros((M, M), dtype=np.complex128)
    l = np.arange(-M // 2, M // 2)
    ly = l[None, :].astype(np.float64)
    for lx in l:  # one grid row at a time keeps the memory small
        lxf = float(lx)
        r = np.sqrt(lxf * lxf + ly[0] ** 2)
        phi = np.mod(np.arctan2(ly[0], lxf), 2.0 * math.pi)
        # bracketing rays a (angle <= phi, cyclically) and b = a + 1
        a = np.searchsorted(ang, phi, side="right") - 1
        wrap_lo = a < 0  # phi before the first ray: bracket (last ray - 2 pi, first ray)
        a = np.where(wrap_lo, R - 1, a)
        b = (a + 1) % R
        phia = np.where(wrap_lo, ang[a] - 2.0 * math.pi, ang[a])
        phib = np.where((b == 0) & ~wrap_lo, ang[b] + 2.0 * math.pi, ang[b])
        if R == 1:
            tphi = np.zeros_like(phi)
        else:
            tphi = (phi - phia) / (phib - phia)
        mf = r / rho
        m0 = np.floor(mf).astype(np.int64)
        tm = mf - m0

        def sample(j, m):
            ok = m < H
            return np.where(ok, V[j, np.where(ok, m, 0)], 0.0)

        va = (1.0 - tm) * sample(a, m0) + tm * sample(a, m0 + 1)
        vb = (1.0 - tm) * sample(b, m0) + tm * sample(b, m0 + 1)
        out[lx % M, (l % M)] = (1.0 - tphi) * va + tphi * vb
    out[0, 0] = np.mean(V[:, 0])  # the origin node belongs to every ray
    return out


def cartesian_grid(B: np.ndarray, theta, N: int, det_spacing: float, n_det: int, M: int | None = None,
                   P: int | None = None) -> np.ndarray:
    """Step 3: bhat on the Cartesian nodes, as an M x M array indexed [l_x mod M][l_y mod M]
    (ray theta_k carries B[k], ray theta_k + pi its complex conjugate)."""
    M = grid_size(N) if M is None else int(M)
    P = _pad(n_det) if P is None else int(P)
    ang, kk, cj = full_circle_rays(theta)
    V = np.where(cj[:, None], np.conj(B[kk]), B[kk])
    return cartesian_grid_rays(ang, V, N, det_spacing, M, P)


def bst_full_period(g, N: int, theta, det_spacing: float, M: int | None = None, P: int | None = None) -> np.ndarray:
    """Step 4 on the whole period: Re sum_l (1/(M dx))^2 bhat(nu_l) e^{2 pi i l . (i' + delta) / M}
    for all M x M offsets i' (array [i'_x mod M][i'_y mod M])."""
    g = np.asarray(g, dtype=np.float64)
    n_det = g.shape[-1]
    P = _pad(n_det) if P is None else int(P)
    M = grid_size(N) if M is None else int(M)
    dx = 2.0 / N
    B = polar_values(g, det_spacing, P)
    V = cartesian_grid(B, theta, N, det_spacing, n_det, M, P)
    delta = (N // 2) - (N - 1) / 2.0
    l = np.fft.fftfreq(M, 1.0 / M)  # l for index l mod M
    ph = np.exp(2j * math.pi * delta * l / M)
    W = V * ph[:, None] * ph[None, :] / (M * dx) ** 2
    return (np.fft.ifft2(W) * (M * M)).real


def bp_bst_interp(g, N: int, theta, det_spacing: float, M: int | None = None, P: int | None = None) -> np.ndarray:
    """R* by the paper's BST algorithm with polar-to-Cartesian interpolation, image [N][N]."""
    M = grid_size(N) if M is None else int(M)
    full = bst_full_period(g, N, theta, det_spacing, M, P)
    idx = (np.arange(N) - N // 2) % M
    return np.ascontiguousarray(full[np.ix_(idx, idx)].T)  # img[i_y][i_x]
