"""GPU parity of the paper's own BST algorithm (bp_backproject_bst: polar-to-Cartesian
interpolation in frequency with K^sigma, Section 5.3 Steps 1-4) against its FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_DIRECT, bp, dev, random_theta, rounded, sample_pixels, synth, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,os,seed", [
    (64, 64, 90, 1.0, 1, 0), (64, 64, 90, 1.0, 4, 1), (37, 41, 7, 1.3, 2, 2), (50, 30, 33, 0.8, 8, 3),
    (96, 128, 64, 1.0, 4, 4), (1, 1, 1, 1.0, 1, 5)])
def test_bst_vs_oracle(N, n_det, n_theta, dt_scale, os, seed):
    rng = np.random.default_rng(seed)
    theta = random_theta(rng, n_theta) if seed % 2 else synth.uniform_theta(n_theta)
    dt = dt_scale * 2.0 / n_det
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    plan = bp.Plan(N, n_det, theta, dt)
    img = plan.backproject_bst(g, os)
    ref = oracle.bp_bst_interp(rounded(g), N, theta, dt, P=oracle.fourier_pad(n_det) * os)
    err = oracle.rel_l2(img.cpu().numpy(), ref)
    print(f"N={N} n_det={n_det} n_theta={n_theta} os={os}: BST vs its oracle rel-L2 {err:.2e}")
    assert err <= TOL_DIRECT


def test_bst_batch_low_precision_and_filtered_accuracy():
    rng = np.random.default_rng(6)
    N, n_det, n_theta = 96, 96, 120
    theta = synth.uniform_theta(n_theta)
    plan = bp.Plan(N, n_det, theta)
    for dtype in (torch.bfloat16, torch.float16):
        g = to_dev(rng.normal(size=(2, n_theta, n_det)), dtype)
        img = plan.backproject_bst(g, 4)
        for i in range(2):
            ref = oracle.bp_bst_interp(rounded(g[i]), N, theta, plan.det_spacing, P=4 * oracle.fourier_pad(n_det))
            assert oracle.rel_l2(img[i].cpu().numpy(), ref) <= TOL_DIRECT
    # accuracy of the algorithm itself on FBP data: distance to the band-limited R* (printed)
    e = synth.random_ellipses(8, 3)
    q = plan.filter(to_dev(synth.ellipse_sinogram(e, theta, n_det)), "shepp-logan")
    exact = oracle.bp_trig_dirichlet(rounded(q), N, theta, plan.det_spacing)
    for os in (1, 2, 4, 8):
        d = oracle.rel_l2(plan.backproject_bst(q, os).cpu().numpy(), exact)
        print(f"FBP 96^2 x 120: BST (oversampling {os}) vs band-limited R* rel-L2 {d:.3e}")
        if os == 4:
            assert d < 0.03


def test_bst_full_size_sampled():
    # 2048^2, 2048 bins, 1800 angles, Shepp-Logan-filtered noisy sinogram, oversampling 4
    wl = synth.LARGE
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    q = plan.filter(to_dev(wl.sinogram()), "shepp-logan")
    img = plan.backproject_bst(q, 4)
    full = oracle.bp_bst_interp(rounded(q), wl.N, wl.theta, wl.det_spacing, P=4 * oracle.fourier_pad(wl.n_det))
    pix = sample_pixels(wl.N, 2000, seed=8)
    got = img.reshape(-1)[torch.from_numpy(pix).to(dev())].cpu().numpy()
    assert oracle.rel_l2(got, full.reshape(-1)[pix]) <= TOL_DIRECT
    assert oracle.rel_l2(img.cpu().numpy(), full) <= TOL_DIRECT


def test_bst_rejects_bad_oversampling():
    plan = bp.Plan(32, 32, synth.uniform_theta(8))
    g = to_dev(np.ones((8, 32)))
    with pytest.raises(bp.BPError, match="radial_oversampling"):
        plan.backproject_bst(g, 3)
    big = bp.Plan(8192, 8192, synth.uniform_theta(4))  # rejected before any workspace is allocated
    with pytest.raises(bp.BPError, match="too large"):
        big.backproject_bst(to_dev(np.ones((4, 8192))), 2)


# ------------------------------------------------- windowed semi-polar form (Step 2.1, eq "w")
@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,os,beta,seed", [
    (64, 64, 90, 1.0, 1, 4.0, 0), (64, 65, 90, 1.0, 4, 8.0, 1), (37, 41, 7, 1.3, 2, 0.0, 2),
    (50, 30, 33, 0.8, 8, 2.5, 3), (96, 128, 64, 1.0, 1, 12.0, 4), (1, 1, 1, 1.0, 1, 3.0, 5), (9, 2, 5, 1.0, 2, 1.0, 6)])
def test_bst_windowed_vs_oracle(N, n_det, n_theta, dt_scale, os, beta, seed):
    rng = np.random.default_rng(seed)
    theta = random_theta(rng, n_theta) if seed % 2 else synth.uniform_theta(n_theta)
    dt = dt_scale * 2.0 / n_det
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    plan = bp.Plan(N, n_det, theta, dt)
    img = plan.backproject_bst_windowed(g, beta, os)
    ref = oracle.bp_bst_semipolar(rounded(g), N, theta, dt, beta, P=oracle.fourier_pad(n_det) * os)
    err = oracle.rel_l2(img.cpu().numpy(), ref)
    print(f"N={N} n_det={n_det} os={os} beta={beta}: windowed BST vs its oracle rel-L2 {err:.2e}")
    assert err <= TOL_DIRECT


def test_bst_windowed_without_window_is_the_full_line_form():
    # beta = 0 and odd n_det: the joined half-lines are the detector rows themselves
    rng = np.random.default_rng(7)
    N, n_det, n_theta = 80, 81, 60
    plan = bp.Plan(N, n_det, synth.uniform_theta(n_theta))
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    a = plan.backproject_bst_windowed(g, 0.0, 2)
    b = plan.backproject_bst(g, 2)
    assert torch.equal(a, b)
    # a new beta, then another oversampling (workspace rebuilt), then back
    c = plan.backproject_bst_windowed(g, 5.0, 2)
    assert oracle.rel_l2(c.cpu().numpy(), a.cpu().numpy()) > 1e-3
    plan.backproject_bst_windowed(g, 5.0, 4)
    assert torch.equal(plan.backproject_bst_windowed(g, 5.0, 2), c)


def test_bst_windowed_batch_low_precision_and_accuracy():
    rng = np.random.default_rng(8)
    N, n_det, n_theta = 96, 96, 120
    theta = synth.uniform_theta(n_theta)
    plan = bp.Plan(N, n_det, theta)
    for dtype in (torch.bfloat16, torch.float16):
        g = to_dev(rng.normal(size=(2, n_theta, n_det)), dtype)
        img = plan.backproject_bst_windowed(g, 6.0, 4)
        for i in range(2):
            ref = oracle.bp_bst_semipolar(rounded(g[i]), N, theta, plan.det_spacing, 6.0,
                                          P=4 * oracle.fourier_pad(n_det))
            assert oracle.rel_l2(img[i].cpu().numpy(), ref) <= TOL_DIRECT
    # the variant's own accuracy on FBP data: distance to the band-limited R* (printed)
    e = synth.random_ellipses(8, 3)
    q = plan.filter(to_dev(synth.ellipse_sinogram(e, theta, n_det)), "shepp-logan")
    exact = oracle.bp_trig_dirichlet(rounded(q), N, theta, plan.det_spacing)
    for beta in (0.0, 1.0, 2.0, 4.0, 8.0):
        d = oracle.rel_l2(plan.backproject_bst_windowed(q, beta, 4).cpu().numpy(), exact)
        print(f"FBP 96^2 x 120: windowed BST (beta {beta}, oversampling 4) vs band-limited R* rel-L2 {d:.3e}")


def test_bst_windowed_full_size_sampled():
    wl = synth.LARGE
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    q = plan.filter(to_dev(wl.sinogram()), "shepp-logan")
    img = plan.backproject_bst_windowed(q, 6.0, 4)
    full = oracle.bp_bst_semipolar(rounded(q), wl.N, wl.theta, wl.det_spacing, 6.0,
                                   P=4 * oracle.fourier_pad(wl.n_det))
    assert oracle.rel_l2(img.cpu().numpy(), full) <= TOL_DIRECT


def test_bst_windowed_rejects_bad_beta():
    plan = bp.Plan(32, 32, synth.uniform_theta(8))
    g = to_dev(np.ones((8, 32)))
    for beta in (-1.0, float("nan"), float("inf")):
        with pytest.raises(bp.BPError, match="beta"):
            plan.backproject_bst_windowed(g, beta)
