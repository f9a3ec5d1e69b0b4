"""GPU parity at the largest single-slice workloads, in the launch configuration the benchmark
times: the 8192^2 slice (8192 bins, 6000 angles; direct R*, Fourier R* with P = 16384 projection
transforms and a 16384^2 grid, and the Fourier R) on sampled outputs, and the 2048^2 x 1800 slice
in BF16 storage against the oracle on the whole image."""
import numpy as np
import torch

import oracle
from gpu_util import TOL_DIRECT, TOL_FOURIER, bp, dev, rounded, sample_pixels, synth, to_dev

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hires():
    wl = synth.HIRES
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    e = synth.random_ellipses(wl.n_ellipses, wl.seed)
    g = synth.ellipse_sinogram_torch(e, wl.theta, wl.n_det, wl.det_spacing, dev()).float()
    q = plan.filter(g, "shepp-logan")
    del g
    qh = rounded(q)
    yield wl, plan, q, qh
    plan.close()
    torch.cuda.empty_cache()


def _pick(img, pix):
    return img.reshape(-1)[torch.from_numpy(pix).to(dev())].cpu().numpy()


def _seam_pixels(N, n, seed):
    """Random pixels, the image corners and centre, and pixels on both sides of tile seams."""
    pix = set(sample_pixels(N, n, seed).tolist())
    rng = np.random.default_rng(seed + 1)
    for _ in range(40):
        x = int(rng.integers(1, N // 64)) * 64 + int(rng.integers(-1, 1))
        y = int(rng.integers(0, N))
        pix.add(y * N + x)
        pix.add(x * N + y)
    return np.array(sorted(pix), dtype=np.int64)


def test_hires_direct_sampled(hires):
    # Section 2 eq "bp_app" at 8192^2 x 6000 with the autotuned launch shape
    wl, plan, q, qh = hires
    plan.autotune("direct", torch.float32, 1)
    img = plan.backproject(q)
    pix = _seam_pixels(wl.N, 300, seed=61)
    ref = oracle.bp_linear_points(qh, wl.N, wl.theta, wl.det_spacing, pix)
    err = oracle.rel_l2(_pick(img, pix), ref)
    print(f"8192^2 x 6000 direct R*: rel-L2 {err:.2e} at {len(pix)} pixels")
    assert err <= TOL_DIRECT


def test_hires_fourier_sampled(hires):
    # Section 5.3 Steps 2-4 at P = 16384 and a 16384^2 grid, against the band-limited oracle
    wl, plan, q, qh = hires
    img = plan.backproject_fourier(q)
    pix = sample_pixels(wl.N, 40, seed=62)
    ref = oracle.bp_trig_points(qh, wl.N, wl.theta, wl.det_spacing, pix)
    err = oracle.rel_l2(_pick(img, pix), ref)
    print(f"8192^2 x 6000 Fourier R*: rel-L2 {err:.2e} at {len(pix)} pixels")
    assert err <= TOL_FOURIER


def test_hires_fourier_adjoint_sampled(hires):
    # the transpose of the Fourier path (forward 16384-point transforms) on sampled (k, j)
    wl, plan, q, qh = hires
    rng = np.random.default_rng(63)
    f = torch.randn((wl.N, wl.N), generator=torch.Generator(device=dev()).manual_seed(63), device=dev())
    g = plan.radon(f, fourier=True)
    ks = rng.choice(wl.n_theta, 4, replace=False)
    js = rng.integers(wl.n_det // 4, 3 * wl.n_det // 4, 4)
    kj = np.array([k * wl.n_det + j for k in ks for j in js])
    ref = oracle.radon_trig_points(rounded(f), wl.n_det, wl.theta, wl.det_spacing, kj)
    err = oracle.rel_l2(_pick(g, kj), ref)
    print(f"8192^2 x 6000 Fourier R: rel-L2 {err:.2e} at {len(kj)} entries")
    assert err <= TOL_FOURIER


def test_bf16_storage_2048_full_image():
    # BF16 sinogram storage, FP32 interpolation and accumulation: the whole 2048^2 image against the
    # oracle on the same BF16-rounded values, in the autotuned shape the benchmark times
    wl = synth.LARGE
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    q = plan.filter(to_dev(wl.sinogram()), "shepp-logan")
    q16 = q.to(torch.bfloat16)
    plan.autotune("direct", torch.bfloat16, 1)
    img = plan.backproject(q16)
    ref = oracle.bp_linear(rounded(q16), wl.N, wl.theta, wl.det_spacing)
    err = oracle.rel_l2(img.cpu().numpy(), ref)
    storage = oracle.rel_l2(ref, oracle.bp_linear(rounded(q), wl.N, wl.theta, wl.det_spacing))
    print(f"2048^2 x 1800 BF16 storage: rel-L2 {err:.2e} vs the oracle on the rounded input "
          f"(storage rounding itself: {storage:.2e}, reported)")
    assert err <= TOL_DIRECT
    plan.close()
