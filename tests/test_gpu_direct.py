"""GPU parity of the direct path (filter, R*, R) against the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import oracle
from gpu_util import (TOL_DIRECT, bp, dev, random_theta, rounded, sample_pixels, synth, to_dev)

pytestmark = pytest.mark.gpu


# ----------------------------------------------------------------------------------- R* (direct)
def test_direct_small_workload():
    wl = synth.SMALL
    q = oracle.filter_rows(wl.sinogram(), wl.det_spacing, oracle.RAMLAK)
    qd = to_dev(q)
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    img = plan.backproject(qd)
    ref = oracle.bp_linear(rounded(qd), wl.N, wl.theta, wl.det_spacing)
    assert oracle.rel_l2(img.cpu().numpy(), ref) <= TOL_DIRECT


@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,seed", [
    (1, 1, 1, 1.0, 0), (2, 3, 2, 1.0, 1), (37, 41, 7, 1.0, 2), (65, 64, 33, 1.3, 3),
    (130, 90, 50, 0.7, 4), (64, 100, 17, 0.5, 5), (200, 257, 181, 1.0, 6), (129, 129, 16, 1.0, 7)])
def test_direct_ragged(N, n_det, n_theta, dt_scale, seed):
    rng = np.random.default_rng(seed)
    theta = random_theta(rng, n_theta) if seed % 2 else synth.uniform_theta(n_theta)
    dt = dt_scale * 2.0 / n_det
    g = rng.normal(size=(n_theta, n_det))
    gd = to_dev(g)
    plan = bp.Plan(N, n_det, theta, dt)
    img = plan.backproject(gd)
    ref = oracle.bp_linear(rounded(gd), N, theta, dt)
    assert oracle.rel_l2(img.cpu().numpy(), ref) <= TOL_DIRECT


@pytest.mark.parametrize("N,n_det,dt_scale,seed", [(96, 96, 1.0, 11), (150, 100, 1.0, 12), (127, 131, 1.0, 13)])
def test_direct_block_kernel_all_quadrants(N, n_det, dt_scale, seed):
    # |c|, |s| <= 1 (n_det / N <= 1 / dt_scale): the 2 x 2-block kernel, whose corner roles follow
    # the signs of (cos, sin).  Angles over the whole circle in shuffled order exchange the roles
    # between most consecutive angles; exact axis angles and diagonals put corners on bin edges.
    rng = np.random.default_rng(seed)
    special = np.array([0.0, 1.25, 0.5, 1.75]) * np.pi  # axis and diagonal angles, distinct mod pi
    theta = rng.permutation(np.concatenate([rng.uniform(-np.pi, 2 * np.pi, 40), special]))
    dt = dt_scale * 2.0 / n_det
    for dtype in (torch.float32, torch.bfloat16):
        gd = to_dev(rng.normal(size=(theta.size, n_det)), dtype)
        plan = bp.Plan(N, n_det, theta, dt)
        img = plan.backproject(gd)
        ref = oracle.bp_linear(rounded(gd), N, theta, dt)
        assert oracle.rel_l2(img.cpu().numpy(), ref) <= TOL_DIRECT


def test_direct_status_word_clean_after_calls():
    # bp_check synchronises and reports device-side wait failures; none after normal calls.
    wl = synth.SMALL
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    for dtype in (torch.float32, torch.bfloat16):
        plan.backproject(to_dev(np.ones((wl.n_theta, wl.n_det)), dtype))
    plan.check()


def test_direct_unsupported_geometry_is_an_error():
    with pytest.raises(bp.BPError, match="window"):
        bp.Plan(64, 1000, synth.uniform_theta(8), 0.0005)


def test_direct_accumulate_and_batch():
    rng = np.random.default_rng(9)
    N, n_det, n_theta = 96, 80, 45
    theta = synth.uniform_theta(n_theta)
    plan = bp.Plan(N, n_det, theta)
    g = to_dev(rng.normal(size=(3, n_theta, n_det)))
    out = plan.backproject(g)
    for i in range(3):
        # small images split the angles over several CTAs per tile whose partial sums are
        # added atomically: equal up to the summation order
        single = plan.backproject(g[i].contiguous())
        assert oracle.rel_l2(single.cpu().numpy(), out[i].cpu().numpy()) <= 1e-6
    base = to_dev(rng.normal(size=(3, N, N)))
    acc = base.clone()
    plan.backproject(g, out=acc, accumulate=True)
    assert torch.allclose(acc, base + out, rtol=0, atol=1e-5)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_direct_low_precision_storage(dtype):
    # 16-bit sinogram storage, float32 interpolation and accumulation: parity against the
    # oracle on the same rounded values; the error of the rounding itself is only reported.
    wl = synth.SMALL
    q = oracle.filter_rows(wl.sinogram(), wl.det_spacing, oracle.SHEPP_LOGAN)
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    q16 = to_dev(q, dtype)
    img = plan.backproject(q16)
    ref = oracle.bp_linear(rounded(q16), wl.N, wl.theta, wl.det_spacing)
    assert oracle.rel_l2(img.cpu().numpy(), ref) <= TOL_DIRECT
    full = oracle.bp_linear(q, wl.N, wl.theta, wl.det_spacing)
    print(f"{dtype}: storage-rounding error vs FP64 input {oracle.rel_l2(img.cpu().numpy(), full):.2e}")


@pytest.mark.parametrize("shape", ["default", "autotuned"])
def test_direct_full_size_sampled(shape):
    # 2048^2 image, 2048 bins, 1800 angles, Shepp-Logan-filtered noisy 50-ellipse sinogram:
    # the full launch, in the default launch shape and in the one the autotuner picks (the
    # benchmark's), checked on sampled pixels that the oracle evaluates one by one.
    wl = synth.LARGE
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    if shape == "autotuned":
        plan.autotune("direct", torch.float32, 1)
    g = to_dev(wl.sinogram())
    q = plan.filter(g, "shepp-logan")
    img = plan.backproject(q)
    pix = sample_pixels(wl.N, 400, seed=1)
    ref = oracle.bp_linear_points(rounded(q), wl.N, wl.theta, wl.det_spacing, pix)
    got = img.reshape(-1)[torch.from_numpy(pix).to(dev())].cpu().numpy()
    assert oracle.rel_l2(got, ref) <= TOL_DIRECT
    # the benchmark's step: the filter writing the row tables (its filtered values are bp_filter's)
    fused = plan.fbp_direct(g, "shepp-logan")
    got = fused.reshape(-1)[torch.from_numpy(pix).to(dev())].cpu().numpy()
    assert oracle.rel_l2(got, ref) <= TOL_DIRECT
    assert oracle.rel_l2(fused.cpu().numpy(), img.cpu().numpy()) <= 1e-6


def test_direct_full_size_shuffled_angles():
    # 2048^2, 2048 bins, 1800 angles over the whole circle in random order: nearly every
    # 16-angle stage mixes the signs of (cos, sin), so the 2x2-block kernel runs its checked
    # loop with role exchanges between angles (sorted angle sets take the stage-uniform loop)
    wl = synth.LARGE
    rng = np.random.default_rng(17)
    theta = rng.permutation(rng.uniform(0.0, 2.0 * np.pi, wl.n_theta))
    plan = bp.Plan(wl.N, wl.n_det, theta, wl.det_spacing)
    plan.set_shape((16, 4), "direct", torch.float32, 1)  # the benchmark's launch shape
    q = to_dev(rng.normal(size=(wl.n_theta, wl.n_det)))
    img = plan.backproject(q)
    pix = sample_pixels(wl.N, 3000, seed=2)
    ref = oracle.bp_linear_points(rounded(q), wl.N, theta, wl.det_spacing, pix)
    got = img.reshape(-1)[torch.from_numpy(pix).to(dev())].cpu().numpy()
    assert oracle.rel_l2(got, ref) <= TOL_DIRECT


# ----------------------------------------------------------------------------------- filter
@pytest.mark.parametrize("kind,param", [("ramlak", 0.0), ("shepp-logan", 0.0), ("tikhonov", 0.02)])
@pytest.mark.parametrize("n_det,rows", [(256, 180), (41, 7), (1, 3), (2048, 64)])
def test_filter_parity(kind, param, n_det, rows):
    okind = {"ramlak": oracle.RAMLAK, "shepp-logan": oracle.SHEPP_LOGAN, "tikhonov": oracle.TIKHONOV}[kind]
    e = synth.random_ellipses(10, seed=n_det)
    th = synth.uniform_theta(rows)
    g = synth.add_gaussian_noise(synth.ellipse_sinogram(e, th, n_det), 0.01, seed=3)
    gd = to_dev(g)
    plan = bp.Plan(n_det, n_det, th)
    q = plan.filter(gd, kind, param)
    ref = oracle.filter_rows(rounded(gd), 2.0 / n_det, okind, param)
    assert oracle.rel_l2(q.cpu().numpy(), ref) <= TOL_DIRECT


def test_filter_in_place_and_low_precision():
    wl = synth.SMALL
    g = wl.sinogram()
    plan = bp.Plan(wl.N, wl.n_det, wl.theta)
    gd = to_dev(g)
    ref = plan.filter(gd, "ramlak")
    inplace = gd.clone()
    plan.filter(inplace, "ramlak", out=inplace)
    assert torch.equal(inplace, ref)
    g16 = to_dev(g, torch.bfloat16)
    q16 = plan.filter(g16, "ramlak")
    ref16 = oracle.filter_rows(rounded(g16), wl.det_spacing, oracle.RAMLAK)
    assert oracle.rel_l2(q16.cpu().numpy(), ref16) <= TOL_DIRECT


# ----------------------------------------------------------------------------------- R (direct transpose)
def test_radon_small_workload():
    wl = synth.SMALL
    e = synth.random_ellipses(wl.n_ellipses, wl.seed)
    f = to_dev(synth.ellipse_image(e, wl.N, supersample=2))
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    g = plan.radon(f)
    ref = oracle.radon(rounded(f), wl.n_det, wl.theta, wl.det_spacing)
    assert oracle.rel_l2(g.cpu().numpy(), ref) <= TOL_DIRECT


@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,seed", [
    (1, 1, 1, 1.0, 0), (37, 41, 7, 1.0, 2), (65, 64, 33, 1.3, 3), (130, 90, 50, 0.7, 4), (64, 100, 17, 0.5, 5)])
def test_radon_ragged(N, n_det, n_theta, dt_scale, seed):
    rng = np.random.default_rng(seed)
    theta = random_theta(rng, n_theta)
    dt = dt_scale * 2.0 / n_det
    fd = to_dev(rng.normal(size=(2, N, N)))
    plan = bp.Plan(N, n_det, theta, dt)
    g = plan.radon(fd)
    for i in range(2):
        ref = oracle.radon(rounded(fd[i]), n_det, theta, dt)
        assert oracle.rel_l2(g[i].cpu().numpy(), ref) <= TOL_DIRECT


@pytest.mark.parametrize("N,n_det,dt_scale,seed", [
    (96, 96, 1.0, 6), (129, 140, 1.0, 7), (70, 30, 1.0, 8), (130, 20, 1.0, 9), (64, 45, 1.0, 10),
    (80, 100, 0.5, 11)])
def test_radon_shuffled_whole_circle(N, n_det, dt_scale, seed):
    # Angles over the whole circle in shuffled order: all four corner roles and both dominant
    # axes, mixed within one CTA's angles in any pattern; exact axis angles and diagonals put
    # corners on bin edges.  Steps |c|, |s| <= 1 run the 2 x 2-block R (pixels down to a sixth of
    # a bin: lanes several blocks apart), larger steps (129 / 140, 80 / 100 at half pitch) the
    # pair form.  Every angles-per-CTA count, one and several bands, a batch of two and the
    # per-angle-weight variant (the transpose of R*).
    rng = np.random.default_rng(seed)
    special = np.array([0.0, 1.25, 0.5, 1.75]) * np.pi
    theta = rng.permutation(np.concatenate([rng.uniform(-np.pi, 2 * np.pi, 29), special]))
    dt = dt_scale * 2.0 / n_det
    plan = bp.Plan(N, n_det, theta, dt)
    fd = to_dev(rng.normal(size=(2, N, N)))
    refs = [oracle.radon(rounded(fd[i]), n_det, theta, dt) for i in range(2)]
    for kang, bands in ((1, 1), (2, 3), (4, 1), (4, 4)):
        plan.set_shape((kang, bands), "radon", batch=2)
        g = plan.radon(fd)
        for i in range(2):
            assert oracle.rel_l2(g[i].cpu().numpy(), refs[i]) <= TOL_DIRECT, (kang, bands)
    w = oracle.weights(theta)
    at = plan.backproject_transpose(fd[0])
    ref = w[:, None] * dt / (2.0 / N) ** 2 * refs[0]
    assert oracle.rel_l2(at.cpu().numpy(), ref) <= TOL_DIRECT


def test_radon_full_size_sampled_angles():
    wl = synth.LARGE
    e = synth.random_ellipses(wl.n_ellipses, wl.seed)
    f = to_dev(synth.ellipse_image(e, wl.N))
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    g = plan.radon(f)
    ks = np.array([0, 1, 449, 450, 451, 899, 900, 1234, 1799])
    ref = oracle.radon(rounded(f), wl.n_det, wl.theta[ks], wl.det_spacing)
    assert oracle.rel_l2(g[ks].cpu().numpy(), ref) <= TOL_DIRECT
    # the launch shape the benchmark times (autotuned)
    plan.autotune("radon", batch=1)
    g = plan.radon(f)
    assert oracle.rel_l2(g[ks].cpu().numpy(), ref) <= TOL_DIRECT


def test_adjoint_identity_on_device():
    # Section 1, eq "adjoint", discrete and weighted: sum_k w_k dt <R f, g>_k = dx^2 <f, R* g>.
    rng = np.random.default_rng(17)
    N, n_det, n_theta = 300, 311, 97
    theta = random_theta(rng, n_theta)
    dt = 1.1 * 2.0 / n_det
    plan = bp.Plan(N, n_det, theta, dt)
    f = to_dev(rng.normal(size=(N, N)))
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    Rf = rounded(plan.radon(f))
    Bg = rounded(plan.backproject(g))
    w = oracle.weights(theta)
    lhs = float(np.sum(w[:, None] * dt * Rf * rounded(g)))
    rhs = float((2.0 / N) ** 2 * np.sum(rounded(f) * Bg))
    scale = float(np.linalg.norm(w[:, None] * dt * Rf) * np.linalg.norm(rounded(g)))
    assert abs(lhs - rhs) <= TOL_DIRECT * scale


# ----------------------------------------------------------------------------------- host entry point
def test_fbp_host_matches_device_calls():
    wl = synth.SMALL
    g = torch.from_numpy(wl.sinogram().astype(np.float32))
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    out = plan.fbp_host(g.pin_memory(), "shepp-logan")
    dev_img = plan.backproject(plan.filter(g.to(dev()), "shepp-logan"))
    assert oracle.rel_l2(out.numpy(), dev_img.cpu().numpy()) <= 1e-6  # atomic summation order
    out2 = plan.fbp_host(torch.stack([g, 2 * g]), "shepp-logan")
    assert torch.allclose(out2[1], 2 * out2[0], rtol=1e-6, atol=1e-6)
    # five slices through the three-slot ring (copies of neighbouring slices overlap the
    # kernels), pinned and pageable, each slice distinct
    gs = torch.stack([g * (i + 1) + i for i in range(5)])
    refs = [plan.backproject(plan.filter(gs[i].to(dev()), "shepp-logan")).cpu() for i in range(5)]
    for src in (gs.pin_memory(), gs):
        out5 = plan.fbp_host(src, "shepp-logan")
        for i in range(5):
            assert oracle.rel_l2(out5[i].numpy(), refs[i].numpy()) <= 1e-6, i
    with pytest.raises(bp.BPError, match="lambda"):
        plan.fbp_host(gs.pin_memory(), "tikhonov", -1.0)


# ----------------------------------------------------------------------------------- persistent batched launch
def test_batched_mixed_geometries_match_single_calls():
    rng = np.random.default_rng(21)
    specs = [(64, 64, 45, 1.0, torch.float32), (100, 90, 33, 0.8, torch.bfloat16), (37, 41, 7, 1.0, torch.float16),
             (256, 256, 180, 1.0, torch.float32), (130, 200, 60, 1.3, torch.float32), (1, 1, 1, 1.0, torch.float32)]
    plans, sinos = [], []
    for N, nd, nt, sc, dt in specs:
        theta = random_theta(rng, nt)
        plans.append(bp.Plan(N, nd, theta, sc * 2.0 / nd))
        sinos.append(to_dev(rng.normal(size=(nt, nd)), dt))
    imgs = bp.backproject_batched(plans, sinos)
    for p, s, img, (N, nd, nt, sc, dt) in zip(plans, sinos, imgs, specs):
        # the persistent batched kernel's synchronous tiles and the single calls' TMA kernels
        # compute the same sum with different FP32 roundings (and, where the stride rules
        # differ, in different forms: 2 x 2-block or pair table)
        single = p.backproject(s)
        assert oracle.rel_l2(img.cpu().numpy(), single.cpu().numpy()) <= TOL_DIRECT
        ref = oracle.bp_linear(rounded(s), N, p.theta, p.det_spacing)
        assert oracle.rel_l2(img.cpu().numpy(), ref) <= TOL_DIRECT


def test_batched_more_than_one_launch():
    rng = np.random.default_rng(22)
    plans = [bp.Plan(8 + (i % 5), 9, synth.uniform_theta(3 + i % 4)) for i in range(300)]
    sinos = [to_dev(rng.normal(size=(p.n_theta, p.n_det))) for p in plans]
    imgs = bp.backproject_batched(plans, sinos)
    for p, s, img in zip(plans[::37], sinos[::37], imgs[::37]):
        assert oracle.rel_l2(img.cpu().numpy(), p.backproject(s).cpu().numpy()) <= TOL_DIRECT  # two kernels


def test_batched_four_image_form():
    # every slice mirror-symmetric (N even, uniform or mirror angle sets, pixels no larger than
    # bins): one launch writes all slices' row tables and clears the images, one persistent
    # four-image launch backprojects them, each slice in its own geometry and element type
    rng = np.random.default_rng(23)
    specs = [(64, 64, 45, "uniform", torch.float32), (100, 90, 30, "uniform", torch.bfloat16),
             (256, 256, 180, "uniform", torch.float16), (130, 150, 20, "whole-circle", torch.float32),
             (66, 41, 7, "uniform", torch.float16), (512, 512, 360, "uniform", torch.bfloat16)]
    plans, sinos = [], []
    for N, nd, nt, angles, dt in specs:
        theta = synth.uniform_theta(nt) if angles == "uniform" else _mirror_set(rng, nt, True)
        plans.append(bp.Plan(N, nd, theta, 2.0 / N))
        sinos.append(to_dev(rng.normal(size=(len(theta), nd)), dt))
    outs = [torch.full((p.N, p.N), 7.0, device=dev()) for p in plans]  # cleared by the table launch
    imgs, names = _kernels(plans[0], lambda: bp.backproject_batched(plans, sinos, outs))
    assert {"klein_tables_mixed_kernel", "bp_direct_klein_mixed_kernel"} <= names, names
    singles = [p.backproject(s) for p, s in zip(plans, sinos)]
    for p, s, img, single in zip(plans, sinos, imgs, singles):
        assert oracle.rel_l2(img.cpu().numpy(), single.cpu().numpy()) <= 1e-6
        ref = oracle.bp_linear(rounded(s), p.N, p.theta, p.det_spacing)
        assert oracle.rel_l2(img.cpu().numpy(), ref) <= TOL_DIRECT
    # a workspace bound of one slice: a launch pair per slice
    plans[0].set_direct_workspace(1)
    imgs1, names1 = _kernels(plans[0], lambda: bp.backproject_batched(plans, sinos))
    assert names1 == names, names1
    for img, single in zip(imgs1, singles):
        assert oracle.rel_l2(img.cpu().numpy(), single.cpu().numpy()) <= 1e-6
    plans[0].set_direct_workspace(0)
    # one slice without the symmetry: the whole batch takes the tiled persistent kernel
    odd = bp.Plan(65, 64, synth.uniform_theta(16))
    godd = to_dev(rng.normal(size=(16, 64)))
    imgs2, names2 = _kernels(plans[0], lambda: bp.backproject_batched(plans[:2] + [odd], sinos[:2] + [godd]))
    assert "bp_batched_kernel" in names2 and "bp_direct_klein_mixed_kernel" not in names2, names2
    for img, single in zip(imgs2, singles[:2] + [odd.backproject(godd)]):
        assert oracle.rel_l2(img.cpu().numpy(), single.cpu().numpy()) <= TOL_DIRECT
    # more slices than one launch's descriptors
    many = [bp.Plan(8 + 2 * (i % 3), 8, synth.uniform_theta(4 + i % 4)) for i in range(300)]
    gm = [to_dev(rng.normal(size=(p.n_theta, p.n_det))) for p in many]
    out, namesm = _kernels(many[0], lambda: bp.backproject_batched(many, gm))
    assert "bp_direct_klein_mixed_kernel" in namesm, namesm
    for p, s, img in zip(many[::29], gm[::29], out[::29]):
        assert oracle.rel_l2(img.cpu().numpy(), p.backproject(s).cpu().numpy()) <= 1e-6


def test_fbp_pipeline_in_cuda_graph():
    # filter + backprojection of a batch recorded once in a CUDA graph and replayed
    wl = synth.SMALL
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    g = to_dev(np.stack([wl.sinogram(slice_id=i) for i in range(3)]))
    q = torch.empty_like(g)
    img = torch.empty((3, wl.N, wl.N), device=dev())
    plan.filter(g, "shepp-logan", out=q)  # first calls allocate plan tables: before capture
    plan.backproject(q, out=img)
    eager = img.clone()
    img.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.filter(g, "shepp-logan", out=q)
        plan.backproject(q, out=img)
    graph.replay()
    torch.cuda.synchronize()
    assert oracle.rel_l2(img.cpu().numpy(), eager.cpu().numpy()) <= 1e-6  # atomic summation order
    plans = [plan, bp.Plan(96, 80, synth.uniform_theta(40))]
    sinos = [q[0].contiguous(), to_dev(np.random.default_rng(1).normal(size=(40, 80)))]
    outs = [torch.empty((p.N, p.N), device=dev()) for p in plans]
    bp.backproject_batched(plans, sinos, outs)
    ref = [o.clone() for o in outs]
    graph2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph2, stream=s):
        bp.backproject_batched(plans, sinos, outs)
    for o in outs:
        o.zero_()
    graph2.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):  # the four-image form adds partial sums atomically
        assert oracle.rel_l2(o.cpu().numpy(), r.cpu().numpy()) <= 1e-6


def test_stage_timer_reports_each_kernel():
    # bp_stage_timing / bp_stage_times: one record per kernel launch, names of the kernels that ran,
    # times that add up to the calls' own CUDA-event time
    wl = synth.SMALL
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    g = to_dev(wl.sinogram())
    q = plan.filter(g, "ramlak")
    plan.backproject(q)
    plan.backproject_fourier(q)
    torch.cuda.synchronize()
    plan.stage_timing(True)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(3):
        plan.filter(g, "ramlak", out=q)
        img = plan.backproject(q)
        plan.backproject_fourier(q)
    e.record()
    times = plan.stage_times()
    plan.stage_timing(False)
    torch.cuda.synchronize()
    assert times["filter_pt_kernel"][1] == 3
    assert any(k.startswith("bp_direct") for k in times)
    assert times["grid_gather_pair_kernel"][1] == 3 and times["fourier_spectra_pt_kernel"][1] == 3
    assert all(ms > 0 for ms, _ in times.values())
    total = sum(ms for ms, _ in times.values())
    assert total <= s.elapsed_time(e) * 1.01 + 0.01
    assert plan.stage_times() == {}  # records dropped after a read
    ref = oracle.bp_linear(rounded(q), wl.N, wl.theta, wl.det_spacing)
    assert oracle.rel_l2(img.cpu().numpy(), ref) <= TOL_DIRECT


# ----------------------------------------------------------------------------------- R*, four-image form
def _mirror_set(rng, n_half, whole_circle):
    """A mirror-symmetric angle set: random angles in (0, pi/2), their mirrors pi - theta, and the
    self-mirrored 0 and pi/2; optionally some angles moved by pi (their rows then pair backwards)."""
    half = rng.uniform(0.0, np.pi / 2, n_half)
    th = np.concatenate([[0.0, np.pi / 2], half, np.pi - half])
    if whole_circle:
        th = th + np.pi * (rng.uniform(size=th.shape) < 0.5)
    return rng.permutation(th)


def _kernels(plan, call):
    plan.stage_timing(True)
    out = call()
    names = set(plan.stage_times())
    plan.stage_timing(False)
    return out, names


@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,seed,angles", [
    (64, 64, 90, 1.0, 30, "uniform"), (66, 41, 7, 1.3, 31, "uniform"),  # N/2 odd: last block column split
    (100, 128, 16, 1.3, 32, "mirror"), (130, 130, 61, 1.0, 33, "whole-circle"),
    (256, 300, 180, 1.2, 34, "uniform"), (192, 150, 40, 1.2, 35, "whole-circle")])
def test_direct_four_image_form(N, n_det, n_theta, dt_scale, seed, angles):
    # even N and a mirror-symmetric angle set take the four-image kernel (global row tables); the
    # whole image against the oracle, also with accumulation, a batch of two and BF16 storage
    rng = np.random.default_rng(seed)
    theta = synth.uniform_theta(n_theta) if angles == "uniform" else _mirror_set(rng, n_theta, angles == "whole-circle")
    dt = dt_scale * 2.0 / n_det
    plan = bp.Plan(N, n_det, theta, dt)
    g = to_dev(rng.normal(size=(2, len(theta), n_det)))
    img, names = _kernels(plan, lambda: plan.backproject(g))
    assert "bp_direct_klein_batch_kernel" in names, names  # a batch: one cooperative launch
    _, names1 = _kernels(plan, lambda: plan.backproject(g[0]))
    assert "bp_direct_klein_kernel" in names1 and "klein_tables_kernel" in names1, names1
    for i in range(2):
        ref = oracle.bp_linear(rounded(g[i]), N, theta, dt)
        assert oracle.rel_l2(img[i].cpu().numpy(), ref) <= TOL_DIRECT
    base = to_dev(rng.normal(size=(2, N, N)))
    acc = base.clone()
    plan.backproject(g, out=acc, accumulate=True)
    assert oracle.rel_l2(acc.cpu().numpy(), img.cpu().numpy() + rounded(base)) <= TOL_DIRECT
    dirty = torch.full_like(img, 7.0)  # cleared inside the table launch
    plan.backproject(g, out=dirty)
    assert oracle.rel_l2(dirty.cpu().numpy(), img.cpu().numpy()) <= 1e-6
    g16 = g.to(torch.bfloat16)  # a batch of 16-bit slices: one persistent launch builds each slice's tables
    img16 = plan.backproject(g16)
    for i in range(2):
        ref16 = oracle.bp_linear(rounded(g16[i]), N, theta, dt)
        assert oracle.rel_l2(img16[i].cpu().numpy(), ref16) <= TOL_DIRECT
    # variants (one block per thread at 3 or 2 CTAs per SM, two blocks per thread) and angle groups
    for shp in ((16, 1), (16, 3), (16, 64), (8, 2), (32, 1), (32, 5)):
        plan.set_shape(shp, "direct", torch.float32, 2)
        assert oracle.rel_l2(plan.backproject(g).cpu().numpy(), img.cpu().numpy()) <= TOL_DIRECT, shp
        plan.set_shape(shp, "direct", torch.float32, 1)
        g1 = g[1].clone()  # own (16-byte aligned) allocation
        assert oracle.rel_l2(plan.backproject(g1).cpu().numpy(), img[1].cpu().numpy()) <= TOL_DIRECT, shp


def test_direct_four_image_form_not_taken_without_symmetry():
    # odd N, or an angle set without mirror partners, keeps the shared-memory kernels
    rng = np.random.default_rng(36)
    for N, theta in ((65, synth.uniform_theta(40)), (64, random_theta(rng, 40))):
        plan = bp.Plan(N, 64, theta)
        g = to_dev(rng.normal(size=(len(theta), 64)))
        img, names = _kernels(plan, lambda: plan.backproject(g))
        assert "bp_direct_klein_kernel" not in names and any(n.startswith("bp_direct") for n in names), names
        assert oracle.rel_l2(img.cpu().numpy(), oracle.bp_linear(rounded(g), N, theta, plan.det_spacing)) <= TOL_DIRECT


# ----------------------------------------------------------------------------------- fused FBP, direct form
@pytest.mark.parametrize("N,n_det,n_theta,angles,kind,param,seed", [
    (256, 256, 180, "uniform", "shepp-logan", 0.0, 40),      # P = 512
    (300, 300, 61, "uniform", "ramlak", 0.0, 41),             # odd n_theta: the last pair holds one row
    (1024, 1100, 40, "whole-circle", "tikhonov", 0.05, 42),   # P = 4096, rows read backwards
    (100, 128, 16, "mirror", "shepp-logan", 0.0, 43),         # P = 256: filtered array path
    (64, 64, 40, "random", "shepp-logan", 0.0, 44),           # no mirror partners: filtered array path
    (130, 300, 61, "uniform", "ramlak", 0.0, 45),             # pixels larger than bins: filtered array path
    (2048, 2100, 20, "uniform", "ramlak", 0.0, 46)])          # P = 8192: filtered array path
def test_fbp_direct_matches_filter_then_backproject(N, n_det, n_theta, angles, kind, param, seed):
    # the fused form (the filter writes the four-image tables and clears the image) where the
    # four-image form runs (N even, mirror-symmetric angles, pixels no larger than bins) and
    # 512 <= P <= 4096, else filter into the plan's array and backproject; either way the image
    # of filter() then backproject(), and the oracle's
    rng = np.random.default_rng(seed)
    if angles == "uniform":
        theta = synth.uniform_theta(n_theta)
    elif angles == "random":
        theta = random_theta(rng, n_theta)
    else:
        theta = _mirror_set(rng, n_theta, angles == "whole-circle")
    plan = bp.Plan(N, n_det, theta, 1.1 * 2.0 / n_det)
    # sinograms shaped like the workloads: seeded ellipse phantoms plus 1 % Gaussian noise
    g = to_dev(np.stack([synth.add_gaussian_noise(synth.ellipse_sinogram(synth.random_ellipses(10, seed + i), theta,
                                                                         n_det, plan.det_spacing), 0.01, seed + i)
                         for i in range(3)]))
    P = 1 << int(np.ceil(np.log2(2 * n_det)))
    fused = 512 <= P <= 4096 and angles != "random" and 2.0 / N <= plan.det_spacing
    img, names = _kernels(plan, lambda: plan.fbp_direct(g[0], kind, param))
    if fused:
        assert "klein_filter_tables_kernel" in names and "bp_direct_klein_kernel" in names, names
        assert not any(n.startswith(("filter", "memset", "klein_tables")) for n in names), names
    else:
        assert "klein_filter_tables_kernel" not in names and any(n.startswith("filter") for n in names), names
    q = plan.filter(g[0], kind, param)
    two = plan.backproject(q)
    assert oracle.rel_l2(img.cpu().numpy(), two.cpu().numpy()) <= 1e-6  # atomic summation order
    # R* of the same filtered rows (the fused filter's values are bp_filter's) against the oracle,
    # and the whole FBP against the oracle's filter and R*: within the sum of the filter's and
    # R*'s float32 tolerances
    assert oracle.rel_l2(img.cpu().numpy(), oracle.bp_linear(rounded(q), N, theta, plan.det_spacing)) <= TOL_DIRECT
    fk = {"ramlak": oracle.RAMLAK, "shepp-logan": oracle.SHEPP_LOGAN, "tikhonov": oracle.TIKHONOV}[kind]
    ref = oracle.bp_linear(oracle.filter_rows(rounded(g[0]), plan.det_spacing, fk, param), N, theta,
                           plan.det_spacing)
    assert oracle.rel_l2(img.cpu().numpy(), ref) <= 2 * TOL_DIRECT
    # into a buffer holding garbage (the clear inside the table launch), a batch (one table launch
    # and one persistent launch for all slices; rows are filtered in pairs across the batch, as
    # bp_filter pairs them) and 16-bit storage
    dirty = torch.full_like(img, 7.0)
    plan.fbp_direct(g[0], kind, param, out=dirty)
    assert oracle.rel_l2(dirty.cpu().numpy(), img.cpu().numpy()) <= 1e-6
    imgs, bnames = _kernels(plan, lambda: plan.fbp_direct(g, kind, param))
    if fused:
        assert "bp_direct_klein_batch_kernel" in bnames and "klein_filter_tables_kernel" in bnames, bnames
    refs = plan.backproject(plan.filter(g, kind, param))
    for i in range(3):
        assert oracle.rel_l2(imgs[i].cpu().numpy(), refs[i].cpu().numpy()) <= 1e-6, i
    g16 = g[:2].to(torch.float16)
    i16 = plan.fbp_direct(g16, kind, param)
    r16 = plan.backproject(plan.filter(g16, kind, param))
    assert oracle.rel_l2(i16.cpu().numpy(), r16.cpu().numpy()) <= 1e-6


def test_fbp_direct_rejects_bad_arguments():
    plan = bp.Plan(64, 64, synth.uniform_theta(16))
    g = torch.zeros((16, 64), device=dev())
    with pytest.raises(bp.BPError, match="lambda"):
        plan.fbp_direct(g, "tikhonov", -1.0)
    with pytest.raises(bp.BPError):
        plan.fbp_direct(g, 7)
    assert plan.fbp_direct(g, "ramlak").abs().max().item() == 0.0


def _table_bytes_per_slice(N, n_det, theta, dt):
    """About the four-image form's row-table bytes per slice: 2 planes x 16 B x (reachable bins + 4
    on each side + 48) per angle (restated from the layout; only used to pick workspace bounds)."""
    r = (2.0 / N) / dt
    E = 32 * ((N // 2 + 31) // 32) - 1
    c, s = np.cos(theta) * r, np.sin(theta) * r
    u00 = (c + s) * (0.5 - 0.5 * N) + 0.5 * (n_det - 1)
    lo = u00 + np.minimum(0, c * E) + np.minimum(0, s * E)
    hi = u00 + np.maximum(0, c * E) + np.maximum(0, s * E)
    L = int(np.floor(hi.max()) + 4 - (np.floor(lo.min()) - 4) + 1)
    return 32 * len(theta) * (L + 48)


def test_direct_batch_in_chunks():
    # a workspace bound smaller than the batch: the slices go through in chunks (one table launch
    # and one persistent launch each), with the result of the single-chunk call
    N, n_det = 256, 256
    theta = synth.uniform_theta(90)
    plan = bp.Plan(N, n_det, theta)
    rng = np.random.default_rng(50)
    g = to_dev(np.stack([synth.add_gaussian_noise(synth.ellipse_sinogram(synth.random_ellipses(10, 50 + i), theta,
                                                                         n_det, plan.det_spacing), 0.01, 50 + i)
                         for i in range(5)]))
    whole, names = _kernels(plan, lambda: plan.backproject(g))
    assert "bp_direct_klein_batch_kernel" in names and "bp_direct_klein_kernel" not in names, names
    fbp_whole = plan.fbp_direct(g, "shepp-logan")
    per = _table_bytes_per_slice(N, n_det, theta, plan.det_spacing)
    for bound, want in ((1, {"bp_direct_klein_kernel"}), (int(2.5 * per), {"bp_direct_klein_batch_kernel",
                                                                         "bp_direct_klein_kernel"})):
        plan.set_direct_workspace(bound)  # chunks of 1, then of 2, 2, 1
        img, names = _kernels(plan, lambda: plan.backproject(g))
        assert want == {n for n in names if n.startswith("bp_direct")}, (bound, names)
        for i in range(5):
            assert oracle.rel_l2(img[i].cpu().numpy(), whole[i].cpu().numpy()) <= 1e-6, (bound, i)
        acc = whole.clone()
        plan.backproject(g, out=acc, accumulate=True)
        assert oracle.rel_l2(acc.cpu().numpy(), 2 * whole.cpu().numpy()) <= 1e-6, bound
        fimg = plan.fbp_direct(g, "shepp-logan")
        for i in range(5):
            assert oracle.rel_l2(fimg[i].cpu().numpy(), fbp_whole[i].cpu().numpy()) <= 1e-6, (bound, i)
    plan.set_direct_workspace(0)
    ref = oracle.bp_linear(rounded(g[4]), N, theta, plan.det_spacing)
    assert oracle.rel_l2(plan.backproject(g)[4].cpu().numpy(), ref) <= TOL_DIRECT
