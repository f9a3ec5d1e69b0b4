"""Helpers shared by the GPU parity tests (inputs only; no operator arithmetic)."""
import numpy as np
import torch

import __graft_entry__
from paper_1608_03589_gb300 import bp, synth

_built = False

TOL_DIRECT = 1e-5   # relative L2, float32 direct path vs FP64 oracle of the same discretisation
TOL_FOURIER = 1e-3  # relative L2, Fourier path vs FP64 band-limited oracle


def dev():
    global _built
    if not _built:
        __graft_entry__.build()
        _built = True
    return torch.device("cuda", 0)


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev()).to(dtype)


def rounded(t: torch.Tensor) -> np.ndarray:
    """Exact float64 values of a (possibly 16-bit) device tensor, as the kernels read them."""
    return t.float().cpu().numpy().astype(np.float64)


def random_theta(rng, n):
    return np.sort(rng.uniform(0.0, np.pi, n))


def sample_pixels(N, n, seed):
    """Random pixels plus corners, centre and tile seams (flat indices)."""
    rng = np.random.default_rng(seed)
    pts = set(rng.choice(N * N, size=min(n, N * N), replace=False).tolist())
    for y in (0, N // 2, N - 1, min(63, N - 1), min(64, N - 1)):
        for x in (0, N // 2, N - 1, min(63, N - 1), min(64, N - 1)):
            pts.add(y * N + x)
    return np.array(sorted(pts), dtype=np.int64)


__all__ = ["bp", "synth", "dev", "to_dev", "rounded", "random_theta", "sample_pixels", "TOL_DIRECT",
           "TOL_FOURIER"]
