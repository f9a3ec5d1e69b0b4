"""Launch shapes and the autotuner: every shape the tuner can pick gives the oracle's result."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_DIRECT, bp, dev, random_theta, rounded, synth, to_dev

pytestmark = pytest.mark.gpu


# (N, n_det, n_theta, dt_scale, dtype): TMA path (f32, f16) and the synchronous path (bf16 rows
# of 90 bins are not 16-byte strided), several tiles with ragged edges
GEOMS = [(256, 256, 180, 1.0, torch.float32), (130, 90, 50, 0.8, torch.bfloat16), (100, 64, 75, 1.3, torch.float16)]


@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,dtype", GEOMS)
def test_every_direct_shape_matches_oracle(N, n_det, n_theta, dt_scale, dtype):
    rng = np.random.default_rng(N + n_theta)
    theta = random_theta(rng, n_theta)
    dt = dt_scale * 2.0 / n_det
    plan = bp.Plan(N, n_det, theta, dt)
    g = to_dev(rng.normal(size=(2, n_theta, n_det)), dtype)
    ref = np.stack([oracle.bp_linear(rounded(g[i]), N, theta, dt) for i in range(2)])
    base = to_dev(rng.normal(size=(2, N, N)))
    seen = set()
    for stage in (8, 16, 32):
        for asplit in (1, 2, 3, 7, 1000):
            plan.set_shape((stage, asplit), "direct", dtype, batch=2)
            used = plan.get_shape("direct", dtype, batch=2)
            assert used[0] in (8, 16, 32) and 1 <= used[1] <= asplit
            seen.add(used)
            img = plan.backproject(g)
            assert oracle.rel_l2(img.cpu().numpy(), ref) <= TOL_DIRECT, used
            acc = base.clone()
            plan.backproject(g, out=acc, accumulate=True)
            assert oracle.rel_l2(acc.cpu().numpy(), ref + rounded(base)) <= TOL_DIRECT, used
    assert len(seen) >= 4
    if dtype == torch.bfloat16:
        assert {s[0] for s in seen} == {16}  # the synchronous path always stages 16 angles


def test_radon_shapes_match_oracle():
    rng = np.random.default_rng(3)
    N, n_det, n_theta = 200, 190, 61
    theta = random_theta(rng, n_theta)
    plan = bp.Plan(N, n_det, theta)
    f = to_dev(rng.normal(size=(N, N)))
    ref = oracle.radon(rounded(f), n_det, theta, plan.det_spacing)
    for kang in (1, 2, 4):
        for bands in (1, 2, 5, 1000):
            plan.set_shape((kang, bands), "radon", batch=1)
            used = plan.get_shape("radon", batch=1)
            assert used[0] == kang and 1 <= used[1] <= min(bands, 16)
            assert oracle.rel_l2(plan.radon(f).cpu().numpy(), ref) <= TOL_DIRECT, used


def test_autotune_picks_a_candidate_and_keeps_parity():
    wl = synth.SMALL
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    default = plan.get_shape("direct", torch.float32, 1)
    assert default[0] in (16, 32) and default[1] >= 1
    shape, ms = plan.autotune("direct", torch.float32, 1)
    assert ms > 0 and shape == plan.get_shape("direct", torch.float32, 1)
    q = to_dev(oracle.filter_rows(wl.sinogram(), wl.det_spacing, oracle.RAMLAK))
    ref = oracle.bp_linear(rounded(q), wl.N, wl.theta, wl.det_spacing)
    assert oracle.rel_l2(plan.backproject(q).cpu().numpy(), ref) <= TOL_DIRECT
    # a second plan of the same geometry finds the shape in the process-wide cache
    other = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    assert other.get_shape("direct", torch.float32, 1) == shape
    # radon
    rshape, rms = plan.autotune("radon", batch=1)
    assert rms > 0 and rshape == plan.get_shape("radon", batch=1)
    f = to_dev(synth.ellipse_image(synth.random_ellipses(6, 4), wl.N))
    ref = oracle.radon(rounded(f), wl.n_det, wl.theta, wl.det_spacing)
    assert oracle.rel_l2(plan.radon(f).cpu().numpy(), ref) <= TOL_DIRECT


def test_autotune_rejects_capture():
    plan = bp.Plan(64, 64, synth.uniform_theta(16))
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    x = torch.zeros(1, device=dev())
    with pytest.raises(bp.BPError, match="capture"):
        with torch.cuda.graph(graph, stream=s):
            x += 1
            plan.autotune("direct", torch.float32, 1)


def test_split_angles_in_cuda_graph():
    # the angle-split path (memset + atomic partial sums) replays correctly from a graph
    rng = np.random.default_rng(5)
    N, n_det, n_theta = 128, 128, 100
    plan = bp.Plan(N, n_det, synth.uniform_theta(n_theta))
    plan.set_shape((16, 4), "direct", torch.float32, 1)
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    img = torch.empty((N, N), device=dev())
    plan.backproject(g, out=img)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.backproject(g, out=img)
    img.fill_(123.0)
    graph.replay()
    torch.cuda.synchronize()
    ref = oracle.bp_linear(rounded(g), N, plan.theta, plan.det_spacing)
    assert oracle.rel_l2(img.cpu().numpy(), ref) <= TOL_DIRECT
