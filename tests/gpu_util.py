"""Helpers shared by the GPU parity tests (inputs only; no solver arithmetic)."""
import numpy as np

from paper_2203_11025_gb300 import synth


def medium(ny, nx, seed=1000, sigma=8.0):
    return synth.grf_kappa2(ny, nx, seed, sigma=sigma)


def crandn(seed, shape):
    return synth.complex_normal(seed, shape)


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
