"""FP64 oracle of the partial (sector) log-polar backprojection: Andersson's convolution of
Section 5.1 (Steps 1-4; eq "andersson", the kernel of eq "and_kernel") applied to one sector
of angles at a time after moving the origin away from the object with the shifting property
of the Radon transform (eq "sh_prop"), as Section 5.2 ("Partial Backprojections") describes.

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU baseline).  Plain
numpy in double precision; numpy's FFT is the only library primitive (the 2D convolution of
Step 3, which the paper also computes with FFTs).

The object is the image [-1, 1]^2 (N pixels, dx = 2/N), inside the disk of radius R = sqrt(2).
A line with normal xi_phi at signed distance t carries g(t, phi) for phi in [0, pi) (the
sinogram, zero off the detector).  Every line is counted once by the half-line angles phi in
[0, pi), split into Q sectors; R* is the sum over the sectors of the partial backprojections
    B_q(x) = int_{phi in sector q} g(x . xi_phi, phi) dphi.
Sector q with centre direction phi_c moves the origin to O' = -d xi_{phi_c}: the paper rescales
the object to radius a_r and shifts it by 1 - a_r, i.e. d / R = (1 - a_r) / a_r (a_r = 1/4
by default).  By eq "sh_prop" the sinogram in the new frame is g'(s, phi) = g(s - d cos(phi -
phi_c), phi), and every line through the object with phi in the sector has s >= d cos beta - R
> 0 (beta the sector's half-width): no line is lost near the new origin.  The paper's minimal
s is the distance from the new origin to the object, 1 - 2 a_r in its units (d - R here); the
mesh starts a little lower, at the lowest line any output node of Step 4 sees,
rho_0 = ln((d - R) cos gamma) - 2 drho with gamma = asin(R/d) + beta + 3 dphi (the nodes that
bracket the pixels reach one step beyond the object).

Meshes:
  phi_j   = j dphi, dphi = pi / n_half, n_half = 2^ceil(log2 n_theta) (half of the full-circle
            mesh of the log-polar method), sector q: j in [q K, (q + 1) K), K = n_half / Q,
            centre phi_c = (q K + (K - 1)/2) dphi, half-width beta = (K - 1)/2 dphi;
  mu_i    = rho_0 + i drho, i < N_rho, up to ln(d + R) with the outermost step at most the
            detector pitch (eq "N_rho");
  output  rho nodes c in [c_lo, N_rho) on the same lattice, covering ln(d - R) .. ln(d + R),
          angle nodes a on the phi lattice covering phi_c +- asin(R / d).
Step 1  g'_L(mu_i, phi_j) = g(e^{mu_i} - d cos(phi_j - phi_c), phi_j) by linear interpolation
        along the detector and between the projections that bracket phi_j (cyclic, with
        g(t, theta + pi) = g(-t, theta)).
Step 2  at angular lag theta' = b dphi the kernel delta(1 - e^{rho'} cos theta') is the unit
        point mass at rho' = -ln cos theta' (cos theta' > 0 for every lag used), the hat of
        unit mass on the two nodes around it.
Step 3  B(rho_c, theta_a) = dphi sum_j sum_i hat(c - i, a - j) g'_L(mu_i, phi_j): linear in rho
        and in angle (the sector is not periodic), by zero-padded 2D FFTs.
Step 4  each pixel x takes B at (ln |x - O'|, the angle of x - O') by bilinear interpolation;
        the sectors add up.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .logpolar import _lerp_rows, _pow2, angle_brackets

R_OBJECT = math.sqrt(2.0)  # radius of the disk holding the image [-1, 1]^2


@dataclass(frozen=True)
class SectorMesh:
    Q: int          # sectors over [0, pi)
    a_r: float      # rescaling ratio: d = R (1 - a_r) / a_r
    d: float        # shift of the origin
    n_half: int     # angle nodes over [0, pi)
    K: int          # angle nodes per sector
    dphi: float
    rho0: float
    drho: float
    n_rho: int      # input mesh mu_i, i < n_rho
    c_lo: int       # first output rho node (same lattice)
    n_out: int      # output rho nodes c_lo .. c_lo + n_out - 1
    a_lo: int       # first output angle node, relative to the sector's first input node
    n_aout: int     # output angle nodes
    b_lo: int       # smallest angular lag a - j
    b_hi: int       # largest angular lag
    kmax: int       # largest radial kernel lag (nodes)
    Lr: int         # FFT length along rho
    Lp: int         # FFT length along phi


def sector_mesh(N: int, n_det: int, n_theta: int, det_spacing: float, Q: int = 8, a_r: float = 0.25) -> SectorMesh:
    dt = float(det_spacing)
    n_half = _pow2(max(n_theta, 1))
    if Q < 1 or n_half % Q:
        raise ValueError("Q must divide the number of angle nodes over [0, pi)")
    if not (0.0 < a_r < 0.5):
        raise ValueError("a_r must lie in (0, 1/2)")
    K = n_half // Q
    dphi = math.pi / n_half
    R = R_OBJECT
    d = R * (1.0 - a_r) / a_r
    beta = 0.5 * (K - 1) * dphi
    alpha = math.asin(R / d)
    gamma = alpha + beta + 3.0 * dphi  # largest angle between an output node and a sector node
    if gamma >= 0.5 * math.pi:
        raise ValueError("sector too wide for the shift: use more sectors or a smaller a_r")
    step = -math.log(1.0 - dt / (d + R))
    # every output node used by Step 4 lies at radius >= (d - R) e^{-drho} and within gamma of
    # every sector angle, so its lines have s >= (d - R) e^{-drho} cos gamma
    rho0, top = math.log((d - R) * math.cos(gamma)) - 2.0 * step, math.log(d + R)
    n_rho = int(math.ceil((top - rho0) / step)) + 1
    drho = (top - rho0) / (n_rho - 1)
    c_lo = int(math.floor((math.log(d - R) - rho0) / drho))
    n_out = n_rho - c_lo
    A = alpha / dphi
    a_lo = int(math.floor(0.5 * (K - 1) - A)) - 1
    a_hi = int(math.ceil(0.5 * (K - 1) + A)) + 1
    n_aout = a_hi - a_lo + 1
    b_lo, b_hi = a_lo - (K - 1), a_hi
    kmax = int(math.floor(-math.log(math.cos(max(-b_lo, b_hi) * dphi)) / drho)) + 1
    Lr = _pow2(n_rho + kmax + 1)
    Lp = _pow2(max(b_hi - b_lo + 1, n_aout, K))
    return SectorMesh(Q, a_r, d, n_half, K, dphi, rho0, drho, n_rho, c_lo, n_out, a_lo, n_aout, b_lo, b_hi, kmax,
                      Lr, Lp)


def sector_centre(m: SectorMesh, q: int) -> float:
    return (q * m.K + 0.5 * (m.K - 1)) * m.dphi


def sample_sector(g, theta, det_spacing: float, m: SectorMesh, q: int) -> np.ndarray:
    """Step 1: g'_L[j'][i] for the sector's angle nodes j' < K and mu_i, i < n_rho."""
    g = np.asarray(g, dtype=np.float64)
    ka, sa, kb, sb, w = angle_brackets(theta, 2 * m.n_half)
    phic = sector_centre(m, q)
    s = np.exp(m.rho0 + m.drho * np.arange(m.n_rho))
    out = np.empty((m.K, m.n_rho))
    for jp in range(m.K):
        j = q * m.K + jp
        t = s - m.d * math.cos(j * m.dphi - phic)
        va = _lerp_rows(g, np.full(m.n_rho, ka[j]), sa[j] * t, det_spacing)
        vb = _lerp_rows(g, np.full(m.n_rho, kb[j]), sb[j] * t, det_spacing)
        out[jp] = (1.0 - w[j]) * va + w[j] * vb
    return out


def sector_kernel(m: SectorMesh) -> np.ndarray:
    """Step 2: K[b - b_lo][dc], the unit-mass hat of the point mass at -ln cos(b dphi) / drho."""
    Kk = np.zeros((m.b_hi - m.b_lo + 1, m.kmax + 2))
    for b in range(m.b_lo, m.b_hi + 1):
        r = -math.log(math.cos(b * m.dphi)) / m.drho
        a0 = int(math.floor(r))
        Kk[b - m.b_lo, a0] += 1.0 - (r - a0)
        Kk[b - m.b_lo, a0 + 1] += r - a0
    return Kk


def convolve_sector(G: np.ndarray, Kk: np.ndarray, m: SectorMesh) -> np.ndarray:
    """Step 3: B[a - a_lo][c - c_lo] = dphi sum_j' sum_i K[a - j'][c - i] G[j'][i], linear in both."""
    A = np.zeros((m.Lp, m.Lr))
    A[:m.K, :m.n_rho] = G
    Kp = np.zeros((m.Lp, m.Lr))
    for bi in range(Kk.shape[0]):
        Kp[(bi + m.b_lo) % m.Lp, :Kk.shape[1]] = Kk[bi]
    C = np.fft.ifft2(np.fft.fft2(A) * np.fft.fft2(Kp)).real
    rows = np.arange(m.a_lo, m.a_lo + m.n_aout) % m.Lp
    return m.dphi * C[np.ix_(rows, np.arange(m.c_lo, m.c_lo + m.n_out))]


def to_cartesian_sector(B: np.ndarray, N: int, m: SectorMesh, q: int) -> np.ndarray:
    """Step 4: bilinear interpolation of B at the pixel centres in the sector's frame, img[i_y][i_x]."""
    x = -1.0 + (np.arange(N) + 0.5) * (2.0 / N)
    X, Y = np.meshgrid(x, x)  # [i_y][i_x]
    phic = sector_centre(m, q)
    ux, uy = math.cos(phic), math.sin(phic)
    px, py = X + m.d * ux, Y + m.d * uy          # x - O'
    rho = 0.5 * np.log(px * px + py * py)
    ang = phic + np.arctan2(-uy * px + ux * py, ux * px + uy * py)  # angle of x - O' near phi_c
    c = (rho - m.rho0) / m.drho - m.c_lo
    a = ang / m.dphi - (q * m.K + m.a_lo)
    c0 = np.floor(c).astype(np.int64)
    a0 = np.floor(a).astype(np.int64)
    fc, fa = c - c0, a - a0
    assert c0.min() >= 0 and c0.max() <= m.n_out - 2 and a0.min() >= 0 and a0.max() <= m.n_aout - 2
    return ((1 - fa) * ((1 - fc) * B[a0, c0] + fc * B[a0, c0 + 1]) +
            fa * ((1 - fc) * B[a0 + 1, c0] + fc * B[a0 + 1, c0 + 1]))


def bp_logpolar_partial(g, N: int, theta, det_spacing: float, Q: int = 8, a_r: float = 0.25) -> np.ndarray:
    """R* by partial log-polar backprojections over Q sectors (Steps 1-4 per sector), image [N][N]."""
    g = np.asarray(g, dtype=np.float64)
    m = sector_mesh(N, g.shape[1], g.shape[0], det_spacing, Q, a_r)
    Kk = sector_kernel(m)
    img = np.zeros((N, N))
    for q in range(m.Q):
        B = convolve_sector(sample_sector(g, theta, det_spacing, m, q), Kk, m)
        img += to_cartesian_sector(B, N, m, q)
    return img
