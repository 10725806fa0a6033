"""Shared helpers for the GPU parity tests: seeded inputs (drawn by the generator module,
combined by the FP64 oracle) and error measures."""
from __future__ import annotations

import numpy as np

from oracle import tproduct as O
from paper_1806_07247_gb300 import synth

# Relative Frobenius error bound of the plain FP32 path against the FP64 oracle.
TOL_FP32 = 1e-5


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def randn(shape, seed, std=1.0):
    return synth.normal(np.random.Generator(np.random.PCG64(seed)), shape, std)


def low_rank(factors: dict) -> np.ndarray:
    """X = P * Q + E in FP64 by the oracle's t-product, rounded once to FP32."""
    X = O.tprod_fourier(factors["P"], factors["Q"]) + factors["E"].astype(np.float64)
    return np.asfortranarray(X.astype(np.float32))


def small_inputs(seed: int = 0):
    f = synth.small(seed)
    return f, low_rank(f)


def batched_inputs(count: int, seed: int = 0):
    specs = synth.batched_specs(512, seed)[:count]
    out = []
    for i, s in enumerate(specs):
        f = synth.batched_tensor(s, i, seed)
        out.append((s, low_rank(f)))
    return out


def median_sigma(Y) -> float:
    """A threshold inside the singular spectrum: the median Fourier-slice singular value."""
    return float(np.median(O.slice_singular_values(Y)))
