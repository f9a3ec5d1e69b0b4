"""Pins of the FP64 oracle of the BST algorithm on Kaiser-Bessel-windowed semi-polar half-lines
(Section 5.3 Steps 1-4 with Step 2.1 and eq "w"): the window's closed-form values, the exact
reduction to the full-line algorithm (itself pinned in test_oracle_bst.py) without a window
and with the window moved onto the full lines, and the resampling of Step 1.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import bst_semipolar as sp
from paper_1608_03589_gb300 import synth

I0_OF_1 = 1.2660658777520082  # modified Bessel function I_0(1) (sum_k (1/4)^k / (k!)^2)


def _data(N, n_det, n_theta, seed):
    th = synth.uniform_theta(n_theta)
    e = synth.random_ellipses(6, seed)
    g = synth.ellipse_sinogram(e, th, n_det)
    return th, oracle.filter_rows(g, 2.0 / n_det, oracle.SHEPP_LOGAN)


def test_window_values():
    # eq "w": identity at beta = 0; symmetric; 1 at the middle sample and 1 / I0(beta) at both ends
    assert np.array_equal(sp.kb_window(9, 0.0), np.ones(9))
    w = sp.kb_window(9, 1.0)
    assert np.allclose(w, w[::-1], rtol=0, atol=1e-15)
    assert abs(w[4] - 1.0) <= 1e-15
    assert abs(w[0] - 1.0 / I0_OF_1) <= 1e-14 and abs(w[-1] - 1.0 / I0_OF_1) <= 1e-14
    # interior sample: x = (2 i - N_s + 1) / (N_s - 1) = -1/2 at i = 2, I0 by its power series
    z = 1.0 * math.sqrt(0.75)
    i0z = sum((z * z / 4.0) ** k / math.factorial(k) ** 2 for k in range(30))
    assert abs(w[2] - i0z / I0_OF_1) <= 1e-14
    assert np.all(np.diff(sp.kb_window(11, 6.0)[:6]) > 0)  # rises towards the middle


def test_halfline_mesh_reaches_the_detector_end():
    for n_det in (7, 8, 64, 65):
        n_s = sp.halfline_count(n_det)
        assert (n_s - 1) >= 0.5 * (n_det - 1)  # s_max covers the last detector centre
        assert (n_s - 2) < 0.5 * (n_det - 1)   # and no sample lies wholly beyond it


def test_step1_resampling():
    # odd n_det: the half-line samples are detector centres; even n_det: the mean of the two
    # centres around each s_i
    rng = np.random.default_rng(0)
    g = rng.normal(size=(3, 7))
    hp, hm = sp.semipolar_rows(g, 2.0 / 7)
    assert np.array_equal(hp, g[:, 3:])
    assert np.array_equal(hm, g[:, 3::-1])
    g = rng.normal(size=(3, 8))
    hp, hm = sp.semipolar_rows(g, 2.0 / 8)
    assert np.allclose(hp[:, :4], 0.5 * (g[:, 3:7] + g[:, 4:8]), rtol=0, atol=1e-15)
    assert np.allclose(hp[:, 4], 0.5 * g[:, 7], rtol=0, atol=1e-15)  # half a bin off the detector
    assert np.allclose(hm[:, :4], 0.5 * (g[:, 4:0:-1] + g[:, 3::-1]), rtol=0, atol=1e-15)


@pytest.mark.parametrize("N,n_det", [(48, 49), (33, 41)])
def test_no_window_is_the_full_line_algorithm(N, n_det):
    # beta = 0, odd n_det: the two half-lines with the shared centre sample halved are the full
    # line; 2 Re of the one-sided grid equals the full-line algorithm exactly
    th, q = _data(N, n_det, 30, seed=N)
    b = sp.bp_bst_semipolar(q, N, th, 2.0 / n_det, 0.0)
    ref = oracle.bp_bst_interp(q, N, th, 2.0 / n_det)
    assert np.abs(b - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("beta", [2.0, 7.5])
def test_window_is_the_full_line_algorithm_on_windowed_lines(beta):
    # the window on each half-line is the window w(|t|) on the full line
    N, n_det = 40, 45
    th, q = _data(N, n_det, 24, seed=5)
    w = sp.kb_window(sp.halfline_count(n_det), beta)
    j = np.abs(np.arange(n_det) - (n_det - 1) // 2)
    b = sp.bp_bst_semipolar(q, N, th, 2.0 / n_det, beta)
    ref = oracle.bp_bst_interp(q * w[j][None, :], N, th, 2.0 / n_det)
    assert np.abs(b - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(b - oracle.bp_bst_interp(q, N, th, 2.0 / n_det)).max() > 1e-3 * np.abs(ref).max()


def test_even_detector_is_the_full_line_algorithm_on_resampled_lines():
    # even n_det: Step 1 moves the samples to s_i = i ds; the result is the full-line
    # algorithm on the resampled odd line t = i dt, |i| < N_s, with the same transform length
    N, n_det = 36, 40
    th, q = _data(N, n_det, 20, seed=8)
    n_s = sp.halfline_count(n_det)
    hp, hm = sp.semipolar_rows(q, 2.0 / n_det)
    line = np.concatenate([hm[:, :0:-1], hp], axis=1)  # t = -(N_s-1) .. (N_s-1) times dt
    assert line.shape[1] == 2 * n_s - 1
    P = oracle.fourier_pad(n_det)
    for beta in (0.0, 3.0):
        b = sp.bp_bst_semipolar(q, N, th, 2.0 / n_det, beta)
        w = sp.kb_window(n_s, beta)
        j = np.abs(np.arange(2 * n_s - 1) - (n_s - 1))
        ref = oracle.bp_bst_interp(line * w[j][None, :], N, th, 2.0 / n_det, P=P)
        assert np.abs(b - ref).max() <= 1e-11 * np.abs(ref).max()
