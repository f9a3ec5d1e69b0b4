"""Pins of the FP64 oracle of Andersson's log-polar backprojection (Section 5.1 Steps 1-4,
Section 5.2 adaptive rho_0; eqs "andersson", "and_kernel", "calc_and_kernel", "N_rho"):
brute force of each step on tiny meshes, the point-mass property of the kernel, a
quarter-turn symmetry, and first-order convergence to closed forms and to the independent
C oracle of R*.  CPU only."""
import math
import os

import numpy as np
import pytest
from scipy.special import ellipe

import oracle
from oracle import logpolar as lp
from paper_1608_03589_gb300 import synth


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "logpolar_mesh_example.txt")


def test_mesh_matches_the_paper_size_rule():
    # the paper's worked example (tests/golden): 1024 bins on [-1, 1] (ds = 2/1024) and a
    # 1024^2 image give N_rho = ln(1/1024) / ln(1 - ds) = 3546 nodes; our mesh adds the
    # half-pixel below rho_0 and the last half bin of the detector (a few nodes more)
    n_s, n_x, n_y, n_rho = [int(v) for v in open(GOLDEN).read().split("\n")[-2].split()]
    ds = 2.0 / n_s
    assert math.ceil(math.log(min(1.0 / n_x, 1.0 / n_y)) / math.log(1.0 - ds)) == n_rho
    m = lp.mesh(n_x, n_s, 720, ds)
    assert n_rho <= m.n_rho <= n_rho + 10
    s_max = 0.5 * 1023 * (2.0 / 1024) + 2.0 / 1024
    assert s_max * (1.0 - math.exp(-m.drho)) <= 2.0 / 1024 + 1e-15  # outer step <= pitch
    assert m.L >= m.n_rho + m.n_out and m.n_phi == 2048


def test_step1_against_pointwise_evaluation():
    rng = np.random.default_rng(1)
    n_theta, n_det, N = 9, 14, 12
    th = rng.uniform(0, np.pi, n_theta)  # unsorted, random
    g = rng.normal(size=(n_theta, n_det))
    dt = 0.9 * 2.0 / n_det
    m = lp.mesh(N, n_det, n_theta, dt)
    gL = lp.sample_logpolar(g, th, dt, m)
    order = np.argsort(th)

    def sino(t, theta):  # g(t, theta) for theta in [0, pi): lerp in t, then in angle (cyclic, flipped)
        def row(k, tt):
            u = tt / dt + 0.5 * (n_det - 1)
            j = math.floor(u)
            f = u - j
            v = lambda jj: g[k, jj] if 0 <= jj < n_det else 0.0
            return (1 - f) * v(j) + f * v(j + 1)
        angs = [(th[k], k, 1.0) for k in order] + [(th[order[0]] + np.pi, order[0], -1.0)]
        angs = [(th[order[-1]] - np.pi, order[-1], -1.0)] + angs
        for (a0, k0, s0), (a1, k1, s1) in zip(angs[:-1], angs[1:]):
            if a0 <= theta < a1:
                w = (theta - a0) / (a1 - a0)
                return (1 - w) * row(k0, s0 * t) + w * row(k1, s1 * t)
        raise AssertionError

    for q in [0, 3, m.n_phi // 2, m.n_phi - 1]:
        phi = 2 * np.pi * q / m.n_phi
        for i in [0, m.n_rho // 3, m.n_rho - 2, m.n_rho - 1]:
            s = math.exp(m.rho0 + i * m.drho)
            want = sino(s, phi) if phi < np.pi else sino(-s, phi - np.pi)
            assert abs(gL[q, i] - want) <= 1e-12 * max(1.0, abs(want))


def test_step2_kernel_is_a_unit_point_mass():
    m = lp.mesh(64, 64, 90, 2.0 / 64)
    K = lp.kernel_weights(m)
    for b in range(m.n_phi):
        c = math.cos(2 * math.pi * b / m.n_phi)
        r = -math.log(c) / m.drho if c > 0 else math.inf
        if r < m.n_out - 1:
            assert abs(K[b].sum() - 1.0) <= 1e-12
            idx = np.nonzero(K[b])[0]
            assert abs((idx * K[b, idx]).sum() - r) <= 1e-9  # centre of mass at -ln cos
        elif c <= 0:
            assert not K[b].any()


def test_step3_against_direct_sum():
    rng = np.random.default_rng(2)
    m = lp.LogPolarMesh(rho0=-2.0, drho=0.3, n_rho=7, n_phi=8, n_out=9, L=16)
    gL = rng.normal(size=(m.n_phi, m.n_rho))
    K = rng.normal(size=(m.n_phi, m.n_out))
    B = lp.convolve(gL, K, m)
    want = np.zeros((m.n_phi, m.n_out))
    for b in range(m.n_phi):
        for c in range(m.n_out):
            for j in range(m.n_phi):
                for i in range(m.n_rho):
                    a = c - i
                    if 0 <= a < m.n_out:
                        want[b, c] += K[(b - j) % m.n_phi, a] * gL[j, i]
    assert np.abs(B - (2 * math.pi / m.n_phi) * want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("N", [64, 65])
def test_quarter_turn(N):
    n = 90
    th = synth.uniform_theta(n)
    e = synth.random_ellipses(6, 5)
    g = synth.ellipse_sinogram(e, th, N)
    h = n // 2
    gr = np.empty_like(g)
    gr[h:] = g[:n - h]
    gr[:h] = g[h:][:, ::-1]
    b = lp.bp_logpolar(g, N, th, 2.0 / N)
    br = lp.bp_logpolar(gr, N, th, 2.0 / N)
    assert np.abs(br - np.rot90(b, -1)).max() <= 1e-10 * np.abs(b).max()


def test_first_order_convergence_away_from_the_origin():
    # the lines through x that pass closer than e^{rho_0} to the origin are missing from the
    # mesh (the origin problem of Section 5.2); away from the origin the method converges
    # at first order to R* of a constant (pi, eq "bp_app"), to Example II (4 E(r)) and to
    # the C oracle's R* of an ellipse phantom
    errs = []
    for N, n in [(64, 90), (128, 180), (256, 360)]:
        th = synth.uniform_theta(n)
        x = -1 + (np.arange(N) + 0.5) * 2.0 / N
        X, Y = np.meshgrid(x, x)
        r = np.hypot(X, Y)
        ring = (r > 0.1) & (r < 0.9)
        const = np.abs(lp.bp_logpolar(np.ones((n, N)), N, th, 2.0 / N) - np.pi)[ring].max()
        circ = lp.bp_logpolar(synth.circ_sinogram(th, N), N, th, 2.0 / N)
        ec = np.abs(circ - 4 * ellipe(np.minimum(r, 1) ** 2))[ring].max() / 4.0
        e = synth.random_ellipses(8, 3)
        g = synth.ellipse_sinogram(e, th, N)
        el = oracle.rel_l2(lp.bp_logpolar(g, N, th, 2.0 / N)[ring], oracle.bp_linear(g, N, th, 2.0 / N)[ring])
        errs.append((const, ec, el))
    for k in range(3):
        assert errs[1][k] < 0.65 * errs[0][k] and errs[2][k] < 0.65 * errs[1][k]
    assert errs[2][0] < 0.1 and errs[2][2] < 0.01
