"""GPU parity of Andersson's log-polar backprojection (bp_backproject_logpolar, Sections
5.1-5.2) against its FP64 oracle (the same discretisation)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_DIRECT, bp, dev, random_theta, rounded, sample_pixels, synth, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,seed", [
    (64, 64, 90, 1.0, 0), (65, 64, 90, 1.0, 2), (37, 41, 7, 1.3, 1), (100, 80, 50, 0.8, 3), (48, 2, 3, 1.0, 5)])
def test_logpolar_vs_oracle(N, n_det, n_theta, dt_scale, seed):
    rng = np.random.default_rng(seed)
    theta = random_theta(rng, n_theta) if seed % 2 else synth.uniform_theta(n_theta)
    dt = dt_scale * 2.0 / n_det
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    plan = bp.Plan(N, n_det, theta, dt)
    img = plan.backproject_logpolar(g)
    ref = oracle.bp_logpolar(rounded(g), N, theta, dt)
    err = oracle.rel_l2(img.cpu().numpy(), ref)
    print(f"N={N} n_det={n_det} n_theta={n_theta}: log-polar vs its oracle rel-L2 {err:.2e}")
    assert err <= TOL_DIRECT


def test_logpolar_batch_low_precision_and_accuracy():
    rng = np.random.default_rng(6)
    N, n_theta = 128, 180
    theta = synth.uniform_theta(n_theta)
    plan = bp.Plan(N, N, theta)
    for dtype in (torch.bfloat16, torch.float16):
        g = to_dev(rng.normal(size=(2, n_theta, N)), dtype)
        img = plan.backproject_logpolar(g)
        for i in range(2):
            ref = oracle.bp_logpolar(rounded(g[i]), N, theta, plan.det_spacing)
            assert oracle.rel_l2(img[i].cpu().numpy(), ref) <= TOL_DIRECT
    # accuracy of the method itself: distance to the direct R* (printed), away from the origin
    e = synth.random_ellipses(8, 3)
    q = to_dev(synth.ellipse_sinogram(e, theta, N))
    lp = plan.backproject_logpolar(q).cpu().numpy()
    direct = oracle.bp_linear(rounded(q), N, theta, plan.det_spacing)
    x = -1 + (np.arange(N) + 0.5) * 2.0 / N
    r = np.hypot(*np.meshgrid(x, x))
    ring = (r > 0.1) & (r < 0.9)
    print(f"128^2 x 180: log-polar vs linear R* rel-L2 {oracle.rel_l2(lp, direct):.3e} (0.1 < r < 0.9: "
          f"{oracle.rel_l2(lp[ring], direct[ring]):.3e})")
    assert oracle.rel_l2(lp[ring], direct[ring]) < 0.03


@pytest.mark.parametrize("wl_name", ["LARGE"])
def test_logpolar_full_size(wl_name):
    wl = getattr(synth, wl_name)
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    g = to_dev(wl.sinogram())
    img = plan.backproject_logpolar(g)
    ref = oracle.bp_logpolar(rounded(g), wl.N, wl.theta, wl.det_spacing)
    assert oracle.rel_l2(img.cpu().numpy(), ref) <= TOL_DIRECT


def test_logpolar_unsupported_sizes():
    with pytest.raises(bp.BPError, match="log-polar"):
        bp.Plan(32, 1, synth.uniform_theta(4)).backproject_logpolar(to_dev(np.ones((4, 1))))
    big = bp.Plan(4096, 4096, synth.uniform_theta(8))
    with pytest.raises(bp.BPError, match="too fine"):
        big.backproject_logpolar(to_dev(np.ones((8, 4096))))


# ----------------------------------------------- partial backprojections (sectors, Section 5.2)
@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,Q,a_r,seed", [
    (64, 64, 90, 1.0, 8, 0.25, 0), (65, 64, 90, 1.0, 16, 0.25, 2), (37, 41, 20, 1.3, 4, 0.2, 1),
    (100, 80, 50, 0.8, 8, 0.3, 3), (48, 2, 16, 1.0, 4, 0.25, 5), (1, 1, 16, 1.0, 8, 0.25, 7)])
def test_logpolar_partial_vs_oracle(N, n_det, n_theta, dt_scale, Q, a_r, seed):
    rng = np.random.default_rng(seed)
    theta = random_theta(rng, n_theta) if seed % 2 else synth.uniform_theta(n_theta)
    dt = dt_scale * 2.0 / n_det
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    plan = bp.Plan(N, n_det, theta, dt)
    img = plan.backproject_logpolar_partial(g, Q, a_r)
    ref = oracle.bp_logpolar_partial(rounded(g), N, theta, dt, Q=Q, a_r=a_r)
    err = oracle.rel_l2(img.cpu().numpy(), ref)
    print(f"N={N} n_det={n_det} n_theta={n_theta} Q={Q} a_r={a_r}: partial log-polar vs its oracle rel-L2 {err:.2e}")
    assert err <= TOL_DIRECT


def test_logpolar_partial_batch_low_precision_and_accuracy():
    rng = np.random.default_rng(9)
    N, n_theta = 128, 180
    theta = synth.uniform_theta(n_theta)
    plan = bp.Plan(N, N, theta)
    for dtype in (torch.bfloat16, torch.float16):
        g = to_dev(rng.normal(size=(2, n_theta, N)), dtype)
        img = plan.backproject_logpolar_partial(g)
        for i in range(2):
            ref = oracle.bp_logpolar_partial(rounded(g[i]), N, theta, plan.det_spacing)
            assert oracle.rel_l2(img[i].cpu().numpy(), ref) <= TOL_DIRECT
    # the method's own accuracy: distance to the direct R*, everywhere and at the centre, where
    # the adaptive-rho_0 form loses the lines near its origin (printed; the centre is gated)
    e = synth.random_ellipses(8, 3)
    q = to_dev(synth.ellipse_sinogram(e, theta, N))
    direct = oracle.bp_linear(rounded(q), N, theta, plan.det_spacing)
    part = plan.backproject_logpolar_partial(q).cpu().numpy()
    adapt = plan.backproject_logpolar(q).cpu().numpy()
    c = slice(N // 2 - 4, N // 2 + 4)
    ep, ea = oracle.rel_l2(part[c, c], direct[c, c]), oracle.rel_l2(adapt[c, c], direct[c, c])
    print(f"128^2 x 180: partial log-polar vs linear R* rel-L2 {oracle.rel_l2(part, direct):.3e} "
          f"(centre 8x8: {ep:.3e}; adaptive rho_0: {oracle.rel_l2(adapt, direct):.3e}, centre {ea:.3e})")
    assert ep < 0.5 * ea and oracle.rel_l2(part, direct) < 0.03
    # another sector count rebuilds the workspace; back again reproduces the first result
    plan.backproject_logpolar_partial(q, 16)
    assert torch.equal(plan.backproject_logpolar_partial(q), torch.from_numpy(part).to(dev()))


def test_logpolar_partial_full_size():
    wl = synth.LARGE
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    g = to_dev(wl.sinogram())
    img = plan.backproject_logpolar_partial(g)
    ref = oracle.bp_logpolar_partial(rounded(g), wl.N, wl.theta, wl.det_spacing)
    assert oracle.rel_l2(img.cpu().numpy(), ref) <= TOL_DIRECT


def test_logpolar_partial_rejects_bad_arguments():
    plan = bp.Plan(32, 32, synth.uniform_theta(64))
    g = to_dev(np.ones((64, 32)))
    with pytest.raises(bp.BPError, match="power of two"):
        plan.backproject_logpolar_partial(g, 3)
    with pytest.raises(bp.BPError, match="a_r"):
        plan.backproject_logpolar_partial(g, 8, 0.6)
    with pytest.raises(bp.BPError, match="too wide"):
        plan.backproject_logpolar_partial(g, 1)
