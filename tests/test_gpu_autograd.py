"""Exact transposes, autograd and TV-regularised gradient descent on the device (Section 6)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_DIRECT, TOL_FOURIER, bp, dev, random_theta, rounded, synth, to_dev
from paper_1608_03589_gb300 import autograd as ag

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,n_det,n_theta,dt_scale,seed", [(37, 41, 7, 1.0, 1), (64, 64, 33, 1.3, 2),
                                                            (100, 90, 50, 0.8, 3)])
def test_transposes_vs_oracle(N, n_det, n_theta, dt_scale, seed):
    rng = np.random.default_rng(seed)
    theta = random_theta(rng, n_theta)
    dt = dt_scale * 2.0 / n_det
    dx = 2.0 / N
    plan = bp.Plan(N, n_det, theta, dt)
    w = oracle.weights(theta)
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    f = to_dev(rng.normal(size=(N, N)))
    # R^T g = (dx^2/dt) A diag(1/w) g   and   A^T f = (dt/dx^2) diag(w) R f
    rt = plan.radon_transpose(g)
    ref = dx * dx / dt * oracle.bp_linear(rounded(g) / w[:, None], N, theta, dt)
    assert oracle.rel_l2(rt.cpu().numpy(), ref) <= TOL_DIRECT
    at = plan.backproject_transpose(f)
    ref = w[:, None] * dt / (dx * dx) * oracle.radon(rounded(f), n_det, theta, dt)
    assert oracle.rel_l2(at.cpu().numpy(), ref) <= TOL_DIRECT


@pytest.mark.parametrize("fourier", [False, True])
def test_euclidean_adjoint_identities_full_size(fourier):
    # 1024^2 image, 1024 bins, 720 angles (the differentiable-reconstruction slice size)
    rng = np.random.default_rng(7)
    N, n_det, n_theta = 1024, 1024, 720
    plan = bp.Plan(N, n_det, synth.uniform_theta(n_theta))
    f = to_dev(rng.normal(size=(N, N)))
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    tol = TOL_DIRECT if not fourier else TOL_FOURIER
    Rf, Rtg = rounded(plan.radon(f, fourier=fourier)), rounded(plan.radon_transpose(g, fourier=fourier))
    lhs, rhs = float(np.sum(Rf * rounded(g))), float(np.sum(rounded(f) * Rtg))
    assert abs(lhs - rhs) <= tol * np.linalg.norm(Rf) * np.linalg.norm(rounded(g))
    Bg = rounded(plan.backproject_fourier(g) if fourier else plan.backproject(g))
    Atf = rounded(plan.backproject_transpose(f, fourier=fourier))
    lhs, rhs = float(np.sum(Bg * rounded(f))), float(np.sum(rounded(g) * Atf))
    assert abs(lhs - rhs) <= tol * np.linalg.norm(Bg) * np.linalg.norm(rounded(f))


@pytest.mark.parametrize("fourier", [False, True])
def test_gradients_match_finite_differences(fourier):
    # 64 x 64: directional derivative of ||R f - g||^2 + lam TV(f) and of <B g, h> against
    # central differences along random directions.
    rng = np.random.default_rng(11)
    N, n_det, n_theta = 64, 64, 48
    plan = bp.Plan(N, n_det, synth.uniform_theta(n_theta))
    g = to_dev(rng.normal(size=(n_theta, n_det)))
    f0 = to_dev(rng.normal(size=(N, N)))
    v = to_dev(rng.normal(size=(N, N)))
    lam = 1e-3

    def loss(f):
        r = ag.radon(f, plan, fourier) - g
        return (r * r).sum() + lam * ag.total_variation(f)

    f = f0.clone().requires_grad_(True)
    (grad,) = torch.autograd.grad(loss(f), f)
    analytic = float((grad * v).sum())
    eps = 1e-2
    with torch.no_grad():
        fd = (float(loss(f0 + eps * v)) - float(loss(f0 - eps * v))) / (2 * eps)
    assert abs(fd - analytic) <= 1e-3 * abs(analytic)

    s = to_dev(rng.normal(size=(n_theta, n_det))).requires_grad_(True)
    h = to_dev(rng.normal(size=(N, N)))
    u = to_dev(rng.normal(size=(n_theta, n_det)))
    (gs,) = torch.autograd.grad((ag.backproject(s, plan, fourier) * h).sum(), s)
    with torch.no_grad():
        fd = (float((ag.backproject(s + eps * u, plan, fourier) * h).sum()) -
              float((ag.backproject(s - eps * u, plan, fourier) * h).sum())) / (2 * eps)
    assert abs(fd - float((gs * u).sum())) <= 1e-3 * abs(float((gs * u).sum()))


def test_tv_reconstruction_converges_and_resumes(tmp_path):
    e = synth.random_ellipses(5, seed=3)
    N, n_det, n_theta = 128, 128, 96
    theta = synth.uniform_theta(n_theta)
    plan = bp.Plan(N, n_det, theta)
    truth = synth.ellipse_image(e, N, supersample=2)
    g = to_dev(np.stack([synth.ellipse_sinogram(e, theta, n_det), synth.ellipse_sinogram(e, theta, n_det)]))
    st = ag.tv_reconstruct(g, plan, iters=30, lam=1e-3)
    losses = np.array(st.losses)
    assert np.all(np.diff(losses) < 0)             # monotone decrease at step 1/L
    assert losses[-1] < 0.2 * losses[0]
    err = oracle.rel_l2(st.f[0].cpu().numpy(), truth)
    assert err < 0.8                                # approaching the phantom after 30 steps
    # checkpoint / resume: 15 + (save, load) + 15 equals 30 in one go, up to summation order
    step = 1.0 / (2.0 * ag.lipschitz_estimate(plan, (2, N, N), dev()) + 1e-3 * 8.0 / 1e-3)
    a = ag.tv_reconstruct(g, plan, iters=15, step=step)
    torch.save({"f": a.f, "iteration": a.iteration}, tmp_path / "ckpt.pt")
    ck = torch.load(tmp_path / "ckpt.pt")
    b = ag.tv_reconstruct(g, plan, iters=15, step=step, state=ag.TVState(f=ck["f"], iteration=ck["iteration"]))
    c = ag.tv_reconstruct(g, plan, iters=30, step=step)
    assert b.iteration == 30
    assert oracle.rel_l2(b.f.cpu().numpy(), c.f.cpu().numpy()) < 1e-5
