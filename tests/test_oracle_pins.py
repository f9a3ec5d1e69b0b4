"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula: each compares it with a closed form,
an invariant, a library routine that computes the same special case, or a second,
independent evaluation.  CPU only.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from paper_1608_03589_gb300 import synth


def _rand_theta(rng, n):
    return np.sort(rng.uniform(0.0, math.pi, n))


# ----------------------------------------------------------------------------------- weights
def test_weights_uniform_equal_dtheta():
    # Table "tab:symbols": dtheta = pi / N_theta for theta_k = k pi / N_theta.
    for n in (1, 2, 7, 180, 1800):
        w = oracle.weights(synth.uniform_theta(n))
        assert np.allclose(w, math.pi / n, rtol=0, atol=1e-14)


def test_weights_nonuniform_sum_to_pi_and_gap_rule():
    rng = np.random.default_rng(3)
    th = rng.uniform(-3.0, 7.0, 11)
    w = oracle.weights(th)
    assert abs(w.sum() - math.pi) < 1e-13
    # Angles equal mod pi define the same line set: shifting one by pi changes nothing.
    th2 = th.copy()
    th2[4] += math.pi
    assert np.allclose(oracle.weights(th2), w, atol=1e-13)


# ----------------------------------------------------------------------------------- R*
def _bp_by_numpy_interp(g, N, theta, dt, w):
    """R* via np.interp on the zero-extended row: a library routine for the same lerp."""
    n_theta, n_det = g.shape
    dx = 2.0 / N
    xs = -1.0 + (np.arange(N) + 0.5) * dx
    X, Y = np.meshgrid(xs, xs)  # X varies along columns, Y along rows
    b = np.zeros((N, N))
    knots = np.arange(-1, n_det + 1, dtype=np.float64)
    for k in range(n_theta):
        u = (X * math.cos(theta[k]) + Y * math.sin(theta[k])) / dt + (n_det - 1) / 2.0
        row = np.concatenate([[0.0], g[k], [0.0]])
        b += w[k] * np.interp(u, knots, row, left=0.0, right=0.0)
    return b


@pytest.mark.parametrize("N,n_det,n_theta,dt_scale", [(8, 8, 5, 1.0), (9, 13, 7, 0.8), (16, 11, 3, 1.7), (7, 41, 6, 0.3)])
def test_bp_linear_matches_library_interp(N, n_det, n_theta, dt_scale):
    rng = np.random.default_rng(N * 100 + n_det)
    g = rng.normal(size=(n_theta, n_det))
    theta = _rand_theta(rng, n_theta)
    dt = dt_scale * 2.0 / n_det
    ref = _bp_by_numpy_interp(g, N, theta, dt, oracle.weights(theta))
    b = oracle.bp_linear(g, N, theta, dt)
    assert np.max(np.abs(b - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_bp_constant_sinogram_is_pi_c():
    # sum_k w_k = pi, so R* of g == c is pi * c wherever every projection stays on the detector.
    N, n_det, n_theta = 64, 64, 37
    theta = synth.uniform_theta(n_theta)
    dt = 2.0 / n_det
    b = oracle.bp_linear(np.full((n_theta, n_det), 2.5), N, theta, dt)
    xs = -1.0 + (np.arange(N) + 0.5) * (2.0 / N)
    R = np.hypot(xs[None, :], xs[:, None])
    inside = R <= (n_det - 1) * dt / 2.0
    assert inside.sum() > 2000
    assert np.max(np.abs(b[inside] - 2.5 * math.pi)) < 1e-12


def test_bp_points_equal_full():
    rng = np.random.default_rng(5)
    g = rng.normal(size=(9, 21))
    theta = _rand_theta(rng, 9)
    b = oracle.bp_linear(g, 17, theta, 0.1)
    pix = rng.choice(17 * 17, 40, replace=False)
    assert np.array_equal(oracle.bp_linear_points(g, 17, theta, 0.1, pix), b.ravel()[pix])


@pytest.mark.parametrize("n", [128, 256])
def test_bp_circ_is_4E(n):
    # Section 4, Example II: g = 2 sqrt(1 - t^2); b(r) = int_0^pi 2 sqrt(1 - r^2 cos^2) = 4 E(r).
    theta = synth.uniform_theta(2 * n)
    g = synth.circ_sinogram(theta, n)
    b = oracle.bp_linear(g, n, theta, 2.0 / n)
    xs = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    r = np.hypot(xs[None, :], xs[:, None])
    m = r <= 0.9
    exact = 4.0 * special.ellipe(r[m] ** 2)
    err = np.max(np.abs(b[m] - exact)) / (2 * math.pi)
    # Linear interpolation of the concave chord profile: error O(dt^2).
    assert err < 3.0 / n ** 2 * 10


def test_bp_gaussian_closed_form():
    # Isotropic Gaussian f = exp(-|x|^2 / (2 s^2)): g(t) = sqrt(2 pi) s exp(-t^2/(2 s^2)) and
    # B g(x) = sqrt(2 pi) s pi exp(-r^2/(4 s^2)) I0(r^2/(4 s^2)).
    s, n = 0.15, 128
    theta = synth.uniform_theta(256)
    dt = 2.0 / n
    t = (np.arange(n) - (n - 1) / 2) * dt
    g = np.repeat((math.sqrt(2 * math.pi) * s * np.exp(-t * t / (2 * s * s)))[None, :], 256, axis=0)
    xs = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    r2 = xs[None, :] ** 2 + xs[:, None] ** 2
    z = r2 / (4 * s * s)
    exact = math.sqrt(2 * math.pi) * s * math.pi * special.i0e(z)  # i0e(z) = exp(-z) I0(z)
    b_lin = oracle.bp_linear(g, n, theta, dt)
    b_trig = oracle.bp_trig_dirichlet(g, n, theta, dt)
    e_lin = oracle.rel_l2(b_lin, exact)
    e_trig = oracle.rel_l2(b_trig, exact)
    assert e_lin < 2e-3          # O(dt^2 / s^2) lerp error
    assert e_trig < 1e-9         # band-limited interpolant of a well-resolved Gaussian
    assert e_trig < e_lin * 1e-4


# ----------------------------------------------------------------------------------- R
def test_adjoint_identity_weighted_and_euclidean():
    # eq "adjoint" (Section 1), discrete: sum_k w_k dt <Rf, g>_k = dx^2 <f, R* g>.
    rng = np.random.default_rng(11)
    N, n_det, n_theta = 23, 31, 13
    theta = _rand_theta(rng, n_theta)
    dt = 1.3 * 2.0 / n_det
    f = rng.normal(size=(N, N))
    g = rng.normal(size=(n_theta, n_det))
    w = oracle.weights(theta)
    Rf = oracle.radon(f, n_det, theta, dt)
    Bg = oracle.bp_linear(g, N, theta, dt)
    dx = 2.0 / N
    lhs = float(np.sum(w[:, None] * dt * Rf * g))
    rhs = float(dx * dx * np.sum(f * Bg))
    scale = np.linalg.norm(w[:, None] * dt * Rf) * np.linalg.norm(g)
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_radon_pixel_mass_is_dx2():
    # Hat weights of one pixel sum to one: sum_j (R delta_p)_{kj} dt = dx^2 for interior pixels.
    N, n_det = 32, 48
    theta = synth.uniform_theta(17)
    dt = 2.0 / n_det
    for p in [(8, 8), (5, 20), (23, 24), (16, 16)]:  # |x| < 1 - dt: always on the detector
        f = np.zeros((N, N))
        f[p] = 1.0
        g = oracle.radon(f, n_det, theta, dt)
        dx = 2.0 / N
        assert np.allclose(g.sum(axis=1) * dt, dx * dx, rtol=1e-14, atol=0)
        # Support: exactly the two bins around u for non-integer u.
        assert np.all((g > 0).sum(axis=1) <= 2)


def test_radon_converges_to_analytic_ellipses():
    # R of the pixelised phantom approximates the exact line integrals (eq "P_theta").
    e = synth.random_ellipses(6, seed=77)
    errs = []
    for N in (64, 128, 256):
        theta = synth.uniform_theta(45)
        img = synth.ellipse_image(e, N, supersample=4)
        g = oracle.radon(img, N, theta, 2.0 / N)
        ga = synth.ellipse_sinogram(e, theta, N, 2.0 / N)
        errs.append(oracle.rel_l2(g, ga))
    assert errs[-1] < 0.02
    assert errs[0] > errs[1] > errs[2]


# ----------------------------------------------------------------------------------- filter
def _response(h, dt, nu):
    n = np.arange(h.shape[0]) - (h.shape[0] - 1) // 2
    return dt * np.sum(h[None, :] * np.cos(2 * math.pi * nu[:, None] * n[None, :] * dt), axis=1)


def test_filter_frequency_responses():
    # Section 3 eq "fbp" (|nu|), Shepp-Logan |nu| sinc(nu dt), Section 6 |nu|/(1 + lambda |nu|).
    n_det = 2048
    dt = 2.0 / n_det
    nu = np.linspace(0.02, 0.48, 24) / dt
    h = oracle.filter_kernel(n_det, dt, oracle.RAMLAK)
    assert np.max(np.abs(_response(h, dt, nu) - np.abs(nu))) < 2e-3 / dt
    h = oracle.filter_kernel(n_det, dt, oracle.SHEPP_LOGAN)
    exact = np.sin(math.pi * nu * dt) / (math.pi * dt)
    assert np.max(np.abs(_response(h, dt, nu) - exact)) < 2e-3 / dt
    lam = 0.02
    h = oracle.filter_kernel(256, 2.0 / 256, oracle.TIKHONOV, lam)
    dt2 = 2.0 / 256
    nu2 = np.linspace(0.02, 0.48, 12) / dt2
    exact = nu2 / (1 + lam * nu2)
    assert np.max(np.abs(_response(h, dt2, nu2) - exact)) < 2e-2 / dt2


def test_ramlak_dc_gain_closed_form():
    # sum_n h(n) = 1/(4 dt^2) - (2/(pi^2 dt^2)) sum_{odd n <= L} 1/n^2  ->  0 as L -> inf.
    n_det, dt = 501, 0.01
    h = oracle.filter_kernel(n_det, dt, oracle.RAMLAK)
    odd = np.arange(1, n_det, 2, dtype=np.float64)
    tail = 2.0 / (math.pi ** 2 * dt * dt) * (math.pi ** 2 / 8 - np.sum(1.0 / odd ** 2))
    assert abs(h.sum() - tail) < 1e-9 * h.max()


def test_filter_rows_equals_fft_linear_convolution():
    rng = np.random.default_rng(2)
    n_det, dt = 77, 0.03
    g = rng.normal(size=(5, n_det))
    for kind, par in ((oracle.RAMLAK, 0.0), (oracle.SHEPP_LOGAN, 0.0), (oracle.TIKHONOV, 0.1)):
        h = oracle.filter_kernel(n_det, dt, kind, par)
        L = 256
        H = np.fft.rfft(h, L)
        full = np.fft.irfft(np.fft.rfft(g, L, axis=1) * H[None, :], L, axis=1)
        ref = dt * full[:, n_det - 1: 2 * n_det - 1]
        q = oracle.filter_rows(g, dt, kind, par)
        assert np.max(np.abs(q - ref)) < 1e-10 * np.max(np.abs(ref))


def test_fbp_reconstructs_ellipse_phantom():
    # Section 3, eq "fbp": B F R f = f.  Analytic sinogram, Ram-Lak, compare inside the FOV.
    e = synth.random_ellipses(5, seed=9)
    N = 128
    theta = synth.uniform_theta(256)
    dt = 2.0 / N
    g = synth.ellipse_sinogram(e, theta, N, dt)
    q = oracle.filter_rows(g, dt, oracle.RAMLAK)
    rec = oracle.bp_linear(q, N, theta, dt)
    ref = synth.ellipse_image(e, N, supersample=4)
    assert oracle.rel_l2(rec, ref) < 0.2


# ----------------------------------------------------------------------------------- Fourier path
def test_trig_interpolation_property_closed_form():
    # One angle theta = 0, N = n_det, dx = dt: u(x_i) = i exactly.  D_P(0) = (P-1)/P and
    # D_P(v) = -(-1)^v / P at other integers (Nyquist bin dropped), so
    # T(i) = g_i - (1/P) sum_j (-1)^(i-j) g_j.
    rng = np.random.default_rng(8)
    n = 16
    g = rng.normal(size=(1, n))
    P = oracle.fourier_pad(n)
    b = oracle.bp_trig_dirichlet(g, n, np.array([0.0]), 2.0 / n)
    sgn = (-1.0) ** np.arange(n)
    T = g[0] - sgn * np.sum(sgn * g[0]) / P
    assert np.allclose(b, math.pi * T[None, :], atol=1e-12)
    pix = np.arange(n * n)
    bs = oracle.bp_trig_points(g, n, np.array([0.0]), 2.0 / n, pix)
    assert np.allclose(bs, b.ravel(), atol=1e-11)


def test_trig_spatial_and_spectral_agree():
    rng = np.random.default_rng(21)
    N, n_det, n_theta = 24, 20, 9
    g = rng.normal(size=(n_theta, n_det))
    theta = _rand_theta(rng, n_theta)
    b = oracle.bp_trig_dirichlet(g, N, theta, 0.09)
    pix = np.arange(N * N)
    assert np.max(np.abs(oracle.bp_trig_points(g, N, theta, 0.09, pix) - b.ravel())) < 1e-10


def test_trig_adjoint_identity():
    rng = np.random.default_rng(12)
    N, n_det, n_theta = 12, 15, 7
    theta = _rand_theta(rng, n_theta)
    dt = 0.15
    f = rng.normal(size=(N, N))
    g = rng.normal(size=(n_theta, n_det))
    w = oracle.weights(theta)
    kj = np.arange(n_theta * n_det)
    Rf = oracle.radon_trig_points(f, n_det, theta, dt, kj).reshape(n_theta, n_det)
    Bg = oracle.bp_trig_dirichlet(g, N, theta, dt)
    dx = 2.0 / N
    lhs = float(np.sum(w[:, None] * dt * Rf * g))
    rhs = float(dx * dx * np.sum(f * Bg))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(w[:, None] * dt * Rf) * np.linalg.norm(g)
