"""bp_fbp_static: the filtered backprojection for callers that cannot allocate device memory
when they reconstruct (a framework that owns every device allocation through a fixed pool or
budget; real-time loops where cudaMalloc's device synchronisation and unbounded latency are
not allowed).  Checked through the C ABI against the ordinary entry points (bp_filter +
bp_backproject_direct) on two calls in a row, the second with different data and another
filter, so a stale static scratch would show.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_DIRECT, bp, dev, synth, to_dev

pytestmark = pytest.mark.gpu


def _call_static(plan, sino, kind, img):
    L = bp.lib()
    st = L.bp_fbp_static(plan.handle, ctypes.c_void_p(sino.data_ptr()), bp._DTYPES[sino.dtype],
                         ctypes.c_void_p(img.data_ptr()), bp.FILTERS[kind], 1 if sino.dim() == 2 else sino.shape[0],
                         ctypes.c_void_p(torch.cuda.current_stream(dev()).cuda_stream))
    return st, L.bp_last_error().decode()


def test_static_fbp_matches_regular_entry_points_twice():
    wl = synth.SMALL
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    rng = np.random.default_rng(3)
    inputs = [(to_dev(wl.sinogram()), "ramlak"),
              (to_dev(wl.sinogram(slice_id=1) + rng.normal(0, 0.01, (wl.n_theta, wl.n_det))), "shepp-logan")]
    for sino, kind in inputs:  # two calls in a row through the same static scratch
        img = torch.empty((wl.N, wl.N), dtype=torch.float32, device=dev())
        st, msg = _call_static(plan, sino, kind, img)
        assert st == 0, msg
        ref = plan.backproject(plan.filter(sino, kind))
        torch.cuda.synchronize()
        assert oracle.rel_l2(img.cpu().numpy(), ref.cpu().numpy()) <= TOL_DIRECT


def test_static_fbp_batch_and_size_limit():
    rng = np.random.default_rng(4)
    N, n_det, n_theta = 96, 100, 60
    plan = bp.Plan(N, n_det, synth.uniform_theta(n_theta))
    sino = to_dev(rng.normal(size=(2, n_theta, n_det)), torch.float16)
    img = torch.empty((2, N, N), dtype=torch.float32, device=dev())
    st, msg = _call_static(plan, sino, "shepp-logan", img)
    assert st == 0, msg
    ref = plan.backproject(plan.filter(sino, "shepp-logan"))
    torch.cuda.synchronize()
    assert oracle.rel_l2(img.cpu().numpy(), ref.cpu().numpy()) <= TOL_DIRECT
    # the limit is n_theta * n_det <= 4 Mi floats: 1024 x 4096 fits exactly, 1025 x 4096 does not
    fits = bp.Plan(64, 4096, synth.uniform_theta(1024), 2.0 / 64)
    g = to_dev(rng.normal(size=(1024, 4096)))
    out = torch.empty((64, 64), device=dev())
    st, msg = _call_static(fits, g, "ramlak", out)
    assert st == 0, msg
    ref = fits.backproject(fits.filter(g, "ramlak"))
    torch.cuda.synchronize()
    assert oracle.rel_l2(out.cpu().numpy(), ref.cpu().numpy()) <= TOL_DIRECT
    big = bp.Plan(64, 4096, synth.uniform_theta(1025), 2.0 / 64)
    small_in = torch.zeros((1025, 4096), dtype=torch.float32, device=dev())
    st, msg = _call_static(big, small_in, "ramlak", torch.empty((64, 64), device=dev()))
    assert st == 4 and "exceeds the static scratch" in msg
