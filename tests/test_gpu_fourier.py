"""GPU parity of the Fourier (BST / gridding) backprojection against the FP64 band-limited oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_FOURIER, bp, dev, random_theta, rounded, sample_pixels, synth, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,seed", [
    (64, 64, 90, 1.0, 0), (37, 41, 7, 1.0, 1), (50, 30, 33, 1.3, 2), (33, 64, 20, 0.6, 3), (1, 1, 1, 1.0, 4),
    (96, 128, 64, 1.0, 5)])
def test_fourier_small_vs_dirichlet_oracle(N, n_det, n_theta, dt_scale, seed):
    rng = np.random.default_rng(seed)
    theta = random_theta(rng, n_theta) if seed % 2 else synth.uniform_theta(n_theta)
    dt = dt_scale * 2.0 / n_det
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    plan = bp.Plan(N, n_det, theta, dt)
    img = plan.backproject_fourier(g)
    ref = oracle.bp_trig_dirichlet(rounded(g), N, theta, dt)
    err = oracle.rel_l2(img.cpu().numpy(), ref)
    print(f"N={N} n_det={n_det} n_theta={n_theta}: Fourier vs band-limited oracle rel-L2 {err:.2e}")
    assert err <= TOL_FOURIER


def test_fourier_small_workload_sampled():
    wl = synth.SMALL
    q = oracle.filter_rows(wl.sinogram(), wl.det_spacing, oracle.RAMLAK)
    qd = to_dev(q)
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    img = plan.backproject_fourier(qd)
    pix = sample_pixels(wl.N, 600, seed=3)
    ref = oracle.bp_trig_points(rounded(qd), wl.N, wl.theta, wl.det_spacing, pix)
    got = img.reshape(-1)[torch.from_numpy(pix).to(dev())].cpu().numpy()
    err = oracle.rel_l2(got, ref)
    lin = oracle.bp_linear_points(rounded(qd), wl.N, wl.theta, wl.det_spacing, pix)
    print(f"256^2: Fourier vs band-limited oracle {err:.2e}; vs linear-interpolation oracle "
          f"{oracle.rel_l2(got, lin):.2e} (different discretisation, not gated)")
    assert err <= TOL_FOURIER


def test_fourier_full_size_sampled():
    # 2048^2, 2048 bins, 1800 angles, Shepp-Logan-filtered noisy sinogram: full launch, sampled pixels.
    wl = synth.LARGE
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    q = plan.filter(to_dev(wl.sinogram()), "shepp-logan")
    img = plan.backproject_fourier(q)
    pix = sample_pixels(wl.N, 150, seed=4)
    ref = oracle.bp_trig_points(rounded(q), wl.N, wl.theta, wl.det_spacing, pix)
    got = img.reshape(-1)[torch.from_numpy(pix).to(dev())].cpu().numpy()
    err = oracle.rel_l2(got, ref)
    print(f"2048^2 x 1800: Fourier vs band-limited oracle rel-L2 {err:.2e}")
    assert err <= TOL_FOURIER


def test_fourier_batch_and_low_precision():
    rng = np.random.default_rng(7)
    N, n_det, n_theta = 48, 48, 40
    theta = synth.uniform_theta(n_theta)
    plan = bp.Plan(N, n_det, theta)
    g = to_dev(rng.normal(size=(2, n_theta, n_det)))
    out = plan.backproject_fourier(g)
    for i in range(2):
        # gridding accumulates with shared-memory atomics: equal up to summation order
        single = plan.backproject_fourier(g[i].contiguous())
        assert oracle.rel_l2(single.cpu().numpy(), out[i].cpu().numpy()) <= 1e-6
    g16 = g.to(torch.bfloat16)
    img16 = plan.backproject_fourier(g16)
    ref = oracle.bp_trig_dirichlet(rounded(g16[0]), N, theta, 2.0 / n_det)
    assert oracle.rel_l2(img16[0].cpu().numpy(), ref) <= TOL_FOURIER


@pytest.mark.parametrize("N,n_det,n_theta,fused", [(300, 300, 50, False), (600, 700, 40, True), (2100, 1000, 24, False),
                                                    (256, 256, 40, False), (512, 400, 30, True)])
def test_fourier_pair_at_every_persistent_transform_length(N, n_det, n_theta, fused):
    # grid sides M = 512 ... 8192 and projection lengths P = 512 ... 2048 (the persistent row
    # transforms are compiled per length; N = M/2 takes the paired column pass of R_F): R*_F
    # (or the fused FBP) and R_F on sampled outputs against the band-limited oracle
    rng = np.random.default_rng(N)
    theta = synth.uniform_theta(n_theta)
    plan = bp.Plan(N, n_det, theta)
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    pix = sample_pixels(N, 200, seed=N)
    if fused:
        img = plan.fbp_fourier(g, "ramlak")
        ref = oracle.bp_trig_points(oracle.filter_rows(rounded(g), plan.det_spacing, oracle.RAMLAK), N, theta,
                                    plan.det_spacing, pix)
    else:
        img = plan.backproject_fourier(g)
        ref = oracle.bp_trig_points(rounded(g), N, theta, plan.det_spacing, pix)
    got = img.reshape(-1)[torch.from_numpy(pix).to(dev())].cpu().numpy()
    assert oracle.rel_l2(got, ref) <= TOL_FOURIER
    f = to_dev(rng.normal(size=(N, N)))
    sino = plan.radon(f, fourier=True)
    ks = rng.choice(n_theta, 4, replace=False)
    js = rng.choice(n_det, 4, replace=False)
    kj = np.array([k * n_det + j for k in ks for j in js])
    ref = oracle.radon_trig_points(rounded(f), n_det, theta, plan.det_spacing, kj)
    got = sino.reshape(-1)[torch.from_numpy(kj).to(dev())].cpu().numpy()
    assert oracle.rel_l2(got, ref) <= TOL_FOURIER


# ----------------------------------------------------------------------------------- adjoint R_F
@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,seed", [
    (32, 32, 24, 1.0, 0), (37, 41, 7, 1.0, 1), (20, 30, 11, 1.3, 2), (33, 24, 9, 0.6, 3), (1, 1, 1, 1.0, 4)])
def test_fourier_adjoint_vs_oracle(N, n_det, n_theta, dt_scale, seed):
    rng = np.random.default_rng(seed)
    theta = random_theta(rng, n_theta)
    dt = dt_scale * 2.0 / n_det
    f = to_dev(rng.normal(size=(N, N)))
    plan = bp.Plan(N, n_det, theta, dt)
    g = plan.radon(f, fourier=True)
    kj = np.arange(n_theta * n_det)
    ref = oracle.radon_trig_points(rounded(f), n_det, theta, dt, kj).reshape(n_theta, n_det)
    err = oracle.rel_l2(g.cpu().numpy(), ref)
    print(f"R_F N={N}: rel-L2 {err:.2e}")
    assert err <= TOL_FOURIER


def test_fourier_adjoint_identity_on_device():
    # eq "adjoint", discrete, for the Fourier pair: sum_k w_k dt <R_F f, g>_k = dx^2 <f, B_F g>
    rng = np.random.default_rng(31)
    N, n_det, n_theta = 200, 181, 97
    theta = random_theta(rng, n_theta)
    dt = 1.1 * 2.0 / n_det
    plan = bp.Plan(N, n_det, theta, dt)
    f = to_dev(rng.normal(size=(N, N)))
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    Rf = rounded(plan.radon(f, fourier=True))
    Bg = rounded(plan.backproject_fourier(g))
    w = oracle.weights(theta)
    lhs = float(np.sum(w[:, None] * dt * Rf * rounded(g)))
    rhs = float((2.0 / N) ** 2 * np.sum(rounded(f) * Bg))
    scale = float(np.linalg.norm(w[:, None] * dt * Rf) * np.linalg.norm(rounded(g)))
    print(f"Fourier adjoint identity: |lhs - rhs| / scale = {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_fourier_adjoint_full_size_sampled():
    wl = synth.LARGE
    e = synth.random_ellipses(wl.n_ellipses, wl.seed)
    f = to_dev(synth.ellipse_image(e, wl.N))
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    g = plan.radon(f, fourier=True)
    rng = np.random.default_rng(5)
    ks = rng.choice(wl.n_theta, 6, replace=False)
    js = rng.choice(wl.n_det, 4, replace=False)
    kj = np.array([k * wl.n_det + j for k in ks for j in js])
    ref = oracle.radon_trig_points(rounded(f), wl.n_det, wl.theta, wl.det_spacing, kj)
    got = g.reshape(-1)[torch.from_numpy(kj).to(dev())].cpu().numpy()
    err = oracle.rel_l2(got, ref)
    print(f"R_F 2048^2 x 1800 sampled rel-L2 {err:.2e}")
    assert err <= TOL_FOURIER


# ----------------------------------------------------------------------------------- FBP fused into the Fourier path
@pytest.mark.parametrize("kind,okind,param", [("ramlak", oracle.RAMLAK, 0.0), ("shepp-logan", oracle.SHEPP_LOGAN, 0.0),
                                              ("tikhonov", oracle.TIKHONOV, 0.05)])
@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,seed", [(64, 64, 90, 1.0, 10), (37, 41, 7, 1.3, 11),
                                                            (96, 128, 64, 0.8, 12)])
def test_fbp_fourier_vs_oracle(kind, okind, param, N, n_det, n_theta, dt_scale, seed):
    rng = np.random.default_rng(seed)
    theta = random_theta(rng, n_theta) if seed % 2 else synth.uniform_theta(n_theta)
    dt = dt_scale * 2.0 / n_det
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    plan = bp.Plan(N, n_det, theta, dt)
    fused = plan.fbp_fourier(g, kind, param)
    # oracle: the filter's linear convolution, then the band-limited R*
    ref = oracle.bp_trig_dirichlet(oracle.filter_rows(rounded(g), dt, okind, param), N, theta, dt)
    assert oracle.rel_l2(fused.cpu().numpy(), ref) <= TOL_FOURIER
    # the same floating-point steps as bp_filter followed by bp_backproject_fourier
    two_step = plan.backproject_fourier(plan.filter(g, kind, param))
    assert torch.equal(fused, two_step)


def test_fbp_fourier_batch_low_precision_and_full_size():
    rng = np.random.default_rng(13)
    N, n_det, n_theta = 48, 48, 41  # odd angle count: batch slices pair rows differently
    plan = bp.Plan(N, n_det, synth.uniform_theta(n_theta))
    g = to_dev(rng.normal(size=(3, n_theta, n_det)), torch.bfloat16)
    fused = plan.fbp_fourier(g, "shepp-logan")
    for i in range(3):
        ref = oracle.bp_trig_dirichlet(oracle.filter_rows(rounded(g[i]), plan.det_spacing, oracle.SHEPP_LOGAN),
                                       N, plan.theta, plan.det_spacing)
        assert oracle.rel_l2(fused[i].cpu().numpy(), ref) <= TOL_FOURIER
    two_step = plan.backproject_fourier(plan.filter(g, "shepp-logan"))
    assert oracle.rel_l2(fused.cpu().numpy(), two_step.cpu().numpy()) <= 1e-6
    # 2048^2, 2048 bins, 1800 angles, sampled pixels against the oracle
    wl = synth.LARGE
    big = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    gd = to_dev(wl.sinogram())
    img = big.fbp_fourier(gd, "shepp-logan")
    pix = sample_pixels(wl.N, 100, seed=14)
    q = oracle.filter_rows(rounded(gd), wl.det_spacing, oracle.SHEPP_LOGAN)
    ref = oracle.bp_trig_points(q, wl.N, wl.theta, wl.det_spacing, pix)
    got = img.reshape(-1)[torch.from_numpy(pix).to(dev())].cpu().numpy()
    assert oracle.rel_l2(got, ref) <= TOL_FOURIER


# ----------------------------------------------------------------------------------- gridding kernel width 4
@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,seed", [(64, 64, 90, 1.0, 20), (37, 41, 7, 1.3, 21),
                                                            (96, 128, 64, 0.8, 22)])
def test_fourier_width4_vs_oracle(N, n_det, n_theta, dt_scale, seed):
    rng = np.random.default_rng(seed)
    theta = random_theta(rng, n_theta) if seed % 2 else synth.uniform_theta(n_theta)
    dt = dt_scale * 2.0 / n_det
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    plan = bp.Plan(N, n_det, theta, dt)
    ref = oracle.bp_trig_dirichlet(rounded(g), N, theta, dt)
    e6 = oracle.rel_l2(plan.backproject_fourier(g).cpu().numpy(), ref)
    plan.set_fourier_width(4)
    e4 = oracle.rel_l2(plan.backproject_fourier(g).cpu().numpy(), ref)
    plan.set_fourier_width(6)
    e6b = oracle.rel_l2(plan.backproject_fourier(g).cpu().numpy(), ref)
    print(f"N={N}: gridding error W=6 {e6:.2e}, W=4 {e4:.2e}")
    assert e4 <= TOL_FOURIER and e6 < e4 and abs(e6b - e6) <= 1e-3 * e6 + 1e-9
    with pytest.raises(bp.BPError, match="width"):
        plan.set_fourier_width(5)


def test_fourier_width4_adjoint_and_full_size():
    # the Fourier R stays the exact transpose of the Fourier R* at W = 4
    rng = np.random.default_rng(33)
    N, n_det, n_theta = 200, 181, 97
    theta = random_theta(rng, n_theta)
    dt = 1.1 * 2.0 / n_det
    plan = bp.Plan(N, n_det, theta, dt)
    plan.set_fourier_width(4)
    f = to_dev(rng.normal(size=(N, N)))
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    Rf = rounded(plan.radon(f, fourier=True))
    Bg = rounded(plan.backproject_fourier(g))
    w = oracle.weights(theta)
    lhs = float(np.sum(w[:, None] * dt * Rf * rounded(g)))
    rhs = float((2.0 / N) ** 2 * np.sum(rounded(f) * Bg))
    scale = float(np.linalg.norm(w[:, None] * dt * Rf) * np.linalg.norm(rounded(g)))
    assert abs(lhs - rhs) <= 1e-5 * scale
    # 2048^2 x 1800, sampled pixels against the band-limited oracle
    wl = synth.LARGE
    big = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    big.set_fourier_width(4)
    q = big.filter(to_dev(wl.sinogram()), "shepp-logan")
    img = big.backproject_fourier(q)
    pix = sample_pixels(wl.N, 150, seed=34)
    ref = oracle.bp_trig_points(rounded(q), wl.N, wl.theta, wl.det_spacing, pix)
    got = img.reshape(-1)[torch.from_numpy(pix).to(dev())].cpu().numpy()
    err = oracle.rel_l2(got, ref)
    print(f"2048^2 x 1800 at W=4: Fourier vs band-limited oracle rel-L2 {err:.2e}")
    assert err <= TOL_FOURIER


def test_transform_paths_replay_from_cuda_graph():
    # after one call (which builds the plan's workspaces) the Fourier FBP, the BST interpolation
    # and the log-polar R* are recorded in a CUDA graph and replay to the same bits
    rng = np.random.default_rng(40)
    N, n_det, n_theta = 96, 96, 60
    plan = bp.Plan(N, n_det, synth.uniform_theta(n_theta))
    g = to_dev(rng.normal(size=(2, n_theta, n_det)))
    outs = [torch.empty((2, N, N), device=dev()) for _ in range(3)]
    calls = [lambda: plan.fbp_fourier(g, "shepp-logan", out=outs[0]),
             lambda: plan.backproject_bst(g, 4, out=outs[1]),
             lambda: plan.backproject_logpolar(g, out=outs[2])]
    for c in calls:
        c()
    eager = [o.clone() for o in outs]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        for c in calls:
            c()
    for o in outs:
        o.fill_(-1.0)
    graph.replay()
    torch.cuda.synchronize()
    for o, e in zip(outs, eager):
        assert torch.equal(o, e)
