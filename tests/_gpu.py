"""Helpers for the GPU tests: availability, library build, parity metric."""
import os

import numpy as np
import pytest


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def pimd():
    if not gpu_available():
        pytest.skip("no CUDA GPU")
    from paper_2602_13553_gb300 import build, binding
    build.build()
    binding.lib()
    return binding


def coord_err(g, c):
    """max over elements of |g - c| / max(|c|, RMS(c)) (per-coordinate relative
    error, with the array's RMS as the floor for coordinates near zero)."""
    g = np.asarray(g)
    c = np.asarray(c)
    rms = np.sqrt(np.mean(c * c))
    scale = np.maximum(np.abs(c), rms)
    diff = np.abs(g - c)
    if not np.all(np.isfinite(g)):
        return float("inf")
    return float(np.max(np.where(scale > 0, diff / np.where(scale > 0, scale, 1.0), diff * 1e300)))


def scalar_err(g, c):
    return abs(g - c) / max(abs(c), 1e-300)
