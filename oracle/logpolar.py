"""FP64 oracle of Andersson's log-polar backprojection as the paper implements it (Section
5.1, Steps 1-4, with the adaptive choice of rho_0 of Section 5.2; the convolution formula is
eq "andersson" of Section 2, the kernel eq "and_kernel", its mesh approximation eq
"calc_and_kernel", the mesh size eq "N_rho").

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU baseline).  Plain
numpy in double precision; numpy's FFT is the only library primitive (the convolution of
Step 3, which the paper also computes with FFTs).

In log-polar coordinates x = e^rho (cos theta, sin theta), s = e^mu, the backprojection is a
convolution over (rho, theta):  [R* g]_L(rho, theta) = int int g_L(mu, phi)
delta(1 - e^{rho - mu} cos(theta - phi)) dmu dphi, with g_L(mu, phi) the sinogram on the
semi-polar half-lines (s >= 0, phi in [0, 2 pi): g_L(mu, phi) = g(e^mu, phi) for phi < pi
and g(-e^mu, phi - pi) otherwise, Section 1).

Meshes (the image is [-1, 1]^2 with N pixels, dx = 2/N; detector pitch dt):
  rho_0   = ln(dx / 2): below half a pixel, as the adaptive rule asks (rho_0 < ln dx);
  top     = ln(s_max), s_max = t_{n_det-1} + dt (the end of the linearly interpolated
            detector: the paper's rho = 0 when the detector ends at 1);
  N_rho   = ceil((top - rho_0) / -ln(1 - dt / s_max)) + 1 nodes mu_i = rho_0 + i drho, so that
            the largest step s_max (1 - e^{-drho}) is at most the detector pitch (eq "N_rho");
  N_phi   = 2^ceil(log2(2 n_theta)) angles phi_j = 2 pi j / N_phi on the full circle;
  output  rho_c = rho_0 + c drho, c < N_out, reaching the farthest pixel centre.

Step 1  g_L on the (mu_i, phi_j) mesh by linear interpolation: along the detector (zero off
        the detector, as R*) and between the two projections that bracket the angle, taken
        cyclically with g(t, theta + pi) = g(-t, theta).
Step 2  the kernel delta(1 - e^{rho'} cos theta') is, at each theta' with cos theta' > 0, a
        unit point mass at rho' = -ln cos theta' (the derivative of the argument there is
        -1); on the mesh it is the hat of unit mass on the two nodes around it.  (The
        indicator of eq "calc_and_kernel", 1/drho on |e^{rho} cos theta - 1| <= drho, puts
        about two nodes of height 1/drho at each angle, twice the mass of the delta.)
Step 3  B(rho_c, theta_b) = dphi sum_j sum_i hat(c - i, b - j) g_L(mu_i, phi_j): linear in rho,
        circular in theta (the dmu of the integral cancels the 1/drho of the point mass).
Step 4  each pixel centre takes B at (ln |x|, atan2(y, x)) by bilinear interpolation (cyclic
        in theta).  The only radius below e^{rho_0} is the centre of an odd image, which has
        no angle: it takes the mean of B over the angles at rho_0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _pow2(n: int) -> int:
    p = 1
    while p < n:
        p *= 2
    return p


@dataclass(frozen=True)
class LogPolarMesh:
    rho0: float
    drho: float
    n_rho: int
    n_phi: int
    n_out: int
    L: int  # convolution length along rho (power of two >= n_rho + n_out)


def mesh(N: int, n_det: int, n_theta: int, det_spacing: float) -> LogPolarMesh:
    dx = 2.0 / N
    dt = float(det_spacing)
    s_max = 0.5 * (n_det - 1) * dt + dt
    rho0 = math.log(0.5 * dx)
    top = math.log(s_max)
    if n_det < 2 or top <= rho0:
        raise ValueError("log-polar mesh needs n_det >= 2 and a detector wider than half a pixel")
    step = -math.log(1.0 - dt / s_max)
    n_rho = int(math.ceil((top - rho0) / step)) + 1
    drho = (top - rho0) / (n_rho - 1)
    r_far = math.sqrt(2.0) * (1.0 - 0.5 * dx)
    n_out = int(math.ceil((math.log(max(r_far, 0.5 * dx)) - rho0) / drho)) + 2
    return LogPolarMesh(rho0, drho, n_rho, _pow2(2 * n_theta), n_out, _pow2(n_rho + n_out))


def _lerp_rows(g, rows, t, dt):
    """Linear interpolation of projection rows at detector positions t (zero off the detector)."""
    n_det = g.shape[1]
    u = t / dt + 0.5 * (n_det - 1)
    j = np.floor(u).astype(np.int64)
    f = u - j
    v0 = np.where((j >= 0) & (j < n_det), g[rows, np.clip(j, 0, n_det - 1)], 0.0)
    v1 = np.where((j + 1 >= 0) & (j + 1 < n_det), g[rows, np.clip(j + 1, 0, n_det - 1)], 0.0)
    return (1.0 - f) * v0 + f * v1


def angle_brackets(theta, n_phi: int):
    """For each phi_j: the two projections (index, detector sign) bracketing the angle and the
    linear weight of the second, on the projection circle with g(t, theta + pi) = g(-t, theta)."""
    th = np.mod(np.asarray(theta, dtype=np.float64), math.pi)
    order = np.argsort(th, kind="stable")
    ths = th[order]
    n = ths.shape[0]
    phi = 2.0 * math.pi * np.arange(n_phi) / n_phi
    tq = np.mod(phi, math.pi)
    sign_q = np.where(phi < math.pi, 1.0, -1.0)
    a = np.searchsorted(ths, tq, side="right") - 1
    ka = np.empty(n_phi, np.int64)
    kb = np.empty(n_phi, np.int64)
    sa = np.empty(n_phi)
    sb = np.empty(n_phi)
    w = np.empty(n_phi)
    for q in range(n_phi):
        if a[q] < 0:  # before the first projection: (last - pi, flipped) .. first
            lo, lo_ang, lo_s = n - 1, ths[n - 1] - math.pi, -1.0
            hi, hi_ang, hi_s = 0, ths[0], 1.0
        elif a[q] == n - 1:  # after the last: last .. (first + pi, flipped)
            lo, lo_ang, lo_s = n - 1, ths[n - 1], 1.0
            hi, hi_ang, hi_s = 0, ths[0] + math.pi, -1.0
        else:
            lo, lo_ang, lo_s = a[q], ths[a[q]], 1.0
            hi, hi_ang, hi_s = a[q] + 1, ths[a[q] + 1], 1.0
        ka[q], kb[q] = order[lo], order[hi]
        sa[q], sb[q] = lo_s * sign_q[q], hi_s * sign_q[q]
        w[q] = (tq[q] - lo_ang) / (hi_ang - lo_ang)
    return ka, sa, kb, sb, w


def sample_logpolar(g, theta, det_spacing: float, m: LogPolarMesh) -> np.ndarray:
    """Step 1: g_L[j][i] on the (phi_j, mu_i) mesh."""
    g = np.asarray(g, dtype=np.float64)
    s = np.exp(m.rho0 + m.drho * np.arange(m.n_rho))
    ka, sa, kb, sb, w = angle_brackets(theta, m.n_phi)
    out = np.empty((m.n_phi, m.n_rho))
    for q in range(m.n_phi):
        va = _lerp_rows(g, np.full(m.n_rho, ka[q]), sa[q] * s, det_spacing)
        vb = _lerp_rows(g, np.full(m.n_rho, kb[q]), sb[q] * s, det_spacing)
        out[q] = (1.0 - w[q]) * va + w[q] * vb
    return out


def kernel_weights(m: LogPolarMesh) -> np.ndarray:
    """Step 2: unit-mass hat of the point mass at rho' = -ln cos theta'_b, [n_phi][n_out]."""
    K = np.zeros((m.n_phi, m.n_out))
    for b in range(m.n_phi):
        c = math.cos(2.0 * math.pi * b / m.n_phi)
        if c <= 0.0:
            continue
        r = -math.log(c) / m.drho
        a0 = int(math.floor(r))
        fr = r - a0
        if a0 < m.n_out:
            K[b, a0] += 1.0 - fr
        if a0 + 1 < m.n_out:
            K[b, a0 + 1] += fr
    return K


def convolve(gL: np.ndarray, K: np.ndarray, m: LogPolarMesh) -> np.ndarray:
    """Step 3: dphi * (K conv gL), linear in rho (first n_out outputs), circular in phi."""
    A = np.zeros((m.n_phi, m.L))
    A[:, : m.n_rho] = gL
    Kp = np.zeros((m.n_phi, m.L))
    Kp[:, : m.n_out] = K
    B = np.fft.ifft2(np.fft.fft2(A) * np.fft.fft2(Kp)).real
    return (2.0 * math.pi / m.n_phi) * B[:, : m.n_out]


def to_cartesian(B: np.ndarray, N: int, m: LogPolarMesh) -> np.ndarray:
    """Step 4: bilinear interpolation of B[phi][rho] at the pixel centres, img[i_y][i_x]."""
    x = -1.0 + (np.arange(N) + 0.5) * (2.0 / N)
    X, Y = np.meshgrid(x, x)  # [i_y][i_x]
    r = np.hypot(X, Y)
    with np.errstate(divide="ignore"):
        c = (np.log(r) - m.rho0) / m.drho
    c = np.clip(np.where(r > 0, c, 0.0), 0.0, m.n_out - 1.0)
    c0 = np.minimum(np.floor(c).astype(np.int64), m.n_out - 2)
    fc = c - c0
    p = np.mod(np.arctan2(Y, X), 2.0 * math.pi) / (2.0 * math.pi / m.n_phi)
    b0 = np.floor(p).astype(np.int64) % m.n_phi
    fb = p - np.floor(p)
    b1 = (b0 + 1) % m.n_phi
    img = ((1 - fb) * ((1 - fc) * B[b0, c0] + fc * B[b0, c0 + 1]) +
           fb * ((1 - fc) * B[b1, c0] + fc * B[b1, c0 + 1]))
    return np.where(r > 0, img, np.mean(B[:, 0]))


def bp_logpolar(g, N: int, theta, det_spacing: float) -> np.ndarray:
    """R* by Andersson's log-polar convolution (Steps 1-4), image [N][N]."""
    g = np.asarray(g, dtype=np.float64)
    m = mesh(N, g.shape[1], g.shape[0], det_spacing)
    gL = sample_logpolar(g, theta, det_spacing, m)
    B = convolve(gL, kernel_weights(m), m)
    return to_cartesian(B, N, m)
