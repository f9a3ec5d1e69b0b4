"""Pins of the FP64 oracle of the partial (sector) log-polar backprojection (Section 5.2,
"Partial Backprojections", with eq "sh_prop"; Section 5.1 Steps 1-4 per sector): each step
against an independent evaluation, the kernel's mass and centre, the exact value pi of R* of
a constant sinogram at every pixel (the origin problem of the adaptive-rho_0 form is gone),
and convergence to the C oracle's R* of a phantom.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import logpolar_partial as lpp
from paper_1608_03589_gb300 import synth


def test_mesh_geometry():
    m = lpp.sector_mesh(64, 64, 90, 2.0 / 64, Q=8, a_r=0.25)
    assert m.n_half == 128 and m.K == 16 and abs(m.d - 3.0 * math.sqrt(2.0)) < 1e-15
    # the mesh starts below every line that an output node of the sector sees and ends at the
    # farthest line of the object
    beta = 0.5 * (m.K - 1) * m.dphi
    gamma = math.asin(math.sqrt(2.0) / m.d) + beta + 3 * m.dphi
    assert math.exp(m.rho0) < (m.d - math.sqrt(2.0)) * math.exp(-m.drho) * math.cos(gamma)
    assert math.exp(m.rho0) < m.d * math.cos(beta) - math.sqrt(2.0)
    assert abs(m.rho0 + (m.n_rho - 1) * m.drho - math.log(m.d + math.sqrt(2.0))) < 1e-12
    # eq "N_rho": the outermost step is at most the detector pitch
    top = math.exp(m.rho0 + (m.n_rho - 1) * m.drho)
    assert top * (1.0 - math.exp(-m.drho)) <= 2.0 / 64 + 1e-15
    with pytest.raises(ValueError):
        lpp.sector_mesh(64, 64, 90, 2.0 / 64, Q=1)  # one sector spans pi: no shift helps
    with pytest.raises(ValueError):
        lpp.sector_mesh(64, 64, 90, 2.0 / 64, Q=3)  # must divide the angle nodes


def test_step1_against_pointwise_evaluation():
    rng = np.random.default_rng(0)
    n_det, n_theta = 40, 25
    theta = np.sort(rng.uniform(0, np.pi, n_theta))
    g = rng.normal(size=(n_theta, n_det))
    dt = 2.0 / n_det
    m = lpp.sector_mesh(32, n_det, n_theta, dt, Q=4)
    th_ext = np.concatenate([theta - np.pi, theta, theta + np.pi])  # g(t, theta +- pi) = g(-t, theta)
    t_det = (np.arange(n_det) - 0.5 * (n_det - 1)) * dt

    def g_at(t, phi):  # independent: np.interp on the zero-extended rows, bracket by search
        k = np.searchsorted(th_ext, phi, side="right") - 1
        vals = []
        for kk in (k, k + 1):
            row = g[kk % n_theta]
            sgn = -1.0 if (kk < n_theta or kk >= 2 * n_theta) else 1.0
            vals.append(np.interp(sgn * t, t_det, row, left=0.0, right=0.0))
        w = (phi - th_ext[k]) / (th_ext[k + 1] - th_ext[k])
        return (1 - w) * vals[0] + w * vals[1]

    for q in (0, 3):
        G = lpp.sample_sector(g, theta, dt, m, q)
        phic = lpp.sector_centre(m, q)
        for jp in (0, m.K // 2, m.K - 1):
            phi = (q * m.K + jp) * m.dphi
            for i in (0, m.n_rho // 3, m.n_rho - 1):
                t = math.exp(m.rho0 + i * m.drho) - m.d * math.cos(phi - phic)
                assert abs(G[jp, i] - g_at(t, phi)) <= 1e-12


def test_step2_kernel_mass_and_centre():
    m = lpp.sector_mesh(48, 48, 60, 2.0 / 48, Q=8)
    Kk = lpp.sector_kernel(m)
    idx = np.arange(Kk.shape[1])
    for bi in range(Kk.shape[0]):
        b = bi + m.b_lo
        assert abs(Kk[bi].sum() - 1.0) <= 1e-14
        assert abs((Kk[bi] * idx).sum() + math.log(math.cos(b * m.dphi)) / m.drho) <= 1e-9


def test_step3_against_direct_double_sum():
    rng = np.random.default_rng(1)
    m = lpp.sector_mesh(16, 16, 12, 2.0 / 16, Q=8)
    G = rng.normal(size=(m.K, m.n_rho))
    Kk = lpp.sector_kernel(m)
    B = lpp.convolve_sector(G, Kk, m)
    ref = np.zeros_like(B)
    for ai in range(m.n_aout):
        a = m.a_lo + ai
        for ci in range(m.n_out):
            c = m.c_lo + ci
            s = 0.0
            for jp in range(m.K):
                b = a - jp
                for i in range(m.n_rho):
                    dc = c - i
                    if 0 <= dc < Kk.shape[1]:
                        s += Kk[b - m.b_lo, dc] * G[jp, i]
            ref[ai, ci] = m.dphi * s
    assert np.abs(B - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("N,a_r,Q", [(24, 0.25, 8), (33, 0.2, 4), (48, 0.3, 16)])
def test_constant_sinogram_is_exact_everywhere(N, a_r, Q):
    # R* of a constant sinogram on a detector covering every line through the image is pi at
    # every pixel, the centre included: each output node takes dphi times the unit mass of
    # every lag, K dphi per sector, pi over the sectors (exact up to rounding); the adaptive-
    # rho_0 form loses the lines near the origin there
    n_det, n_theta = 2 * N, 2 * N
    theta = synth.uniform_theta(n_theta)
    dt = 3.2 / n_det  # detector [-1.6, 1.6] covers |t| <= sqrt(2)
    g = np.ones((n_theta, n_det))
    b = oracle.bp_logpolar_partial(g, N, theta, dt, Q=Q, a_r=a_r)
    assert np.abs(b - math.pi).max() <= 1e-12
    c = N // 2
    assert abs(oracle.bp_logpolar(g, N, theta, dt)[c, c] - math.pi) > 1e-2


def test_converges_to_the_direct_backprojection_and_fixes_the_origin():
    # smooth phantom (ellipse sinogram, no filter): distance to the C oracle's R* falls with N;
    # near the image centre it is far below the adaptive-rho_0 form's (Section 5.2)
    prev = None
    for N in (32, 64):
        theta = synth.uniform_theta(2 * N)
        e = synth.random_ellipses(5, seed=11)
        g = synth.ellipse_sinogram(e, theta, N)
        dt = 2.0 / N
        ref = oracle.bp_linear(g, N, theta, dt)
        b = oracle.bp_logpolar_partial(g, N, theta, dt)
        err = oracle.rel_l2(b, ref)
        if prev is not None:
            assert err < 0.75 * prev
        prev = err
        c = slice(N // 2 - 3, N // 2 + 3)
        e_part = np.abs(b[c, c] - ref[c, c]).max()
        e_adapt = np.abs(oracle.bp_logpolar(g, N, theta, dt)[c, c] - ref[c, c]).max()
        assert e_part < 0.25 * e_adapt
    assert prev < 0.02


def test_sector_counts_agree():
    N = 40
    theta = synth.uniform_theta(64)
    g = synth.ellipse_sinogram(synth.random_ellipses(4, seed=2), theta, N)
    b4 = oracle.bp_logpolar_partial(g, N, theta, 2.0 / N, Q=4)
    b8 = oracle.bp_logpolar_partial(g, N, theta, 2.0 / N, Q=8)
    ref = oracle.bp_linear(g, N, theta, 2.0 / N)
    assert oracle.rel_l2(b4, b8) < 0.5 * max(oracle.rel_l2(b4, ref), oracle.rel_l2(b8, ref)) + 1e-3
