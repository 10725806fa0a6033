"""Seeded synthetic inputs for the t-product workloads.

This module only draws random numbers and sizes.  It holds none of the method's
arithmetic (no DFT, no t-product, no SVD), so both the CUDA path and the FP64
oracle can use it: a low-tubal-rank tensor is returned as its factors P, Q and a
noise tensor, and each side forms X = P * Q + noise with its own t-product.

Every array is float32 with shape (n1, n2, n3) in Fortran (column-major) order,
so entry (i, j, k) sits at offset i + n1*j + n1*n2*k, the layout of the C API.

Generators: numpy PCG64 streams.  A multi-tensor workload derives one child
stream per tensor with SeedSequence.spawn, so tensor t of a workload is the same
whether 1 or all tensors are drawn.

Workloads (the paper's method has no public dataset; these stand in for the
low-rank-plus-noise tensors of its use case):

* small(): P 64x4x16, Q 4x64x16 iid N(0,1), noise 64x64x16 iid N(0, 0.01^2),
  tau = 0.5.
* batched(): 512 tensors, n1, n2 uniform in {16..160}, n3 uniform in {4..64},
  tubal rank r uniform in {2..12}, factors iid N(0,1), noise N(0, 0.05^2),
  tau = 2 * 0.05 * sqrt(n3) * (sqrt(n1) + sqrt(n2)) (twice the expected top
  singular value of one Fourier slice of the noise).
* gemm(): A 2048x1024x64 and B 1024x1024x64 iid N(0,1).
* shifted_square(): n x n x n3 with frontal slice 0 = I + G_0 and slices k > 0 = G_k,
  G iid N(0, 1/(16 n n3)), so every Fourier slice is I plus a matrix of spectral norm
  about 1/2 (condition number about 3): the inverse and QR workloads.
* gaussian(): n1 x n2 x n3 iid N(0, 1) (tall shapes give well-conditioned QR slices).
* stream_specs(): the mixed call stream: each call is prox_tnn or tprod by a fair coin,
  n1, n2 uniform in {16..512}, n3 uniform in {4..256}, tprod's third size l uniform in
  {16..512}, tubal rank r uniform in {4..40}, noise N(0, 0.02^2), tau = 2 nu as for
  batched() (every operand is a rank-r t-product of N(0,1) factors plus noise).
* trpca(): 240x320x100, tubal rank 10 factors iid N(0,1), 10% of positions
  (without replacement) corrupted by values uniform in [-5, 5],
  tau = 1 / sqrt(max(n1, n2) * n3).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["normal", "small", "batched_specs", "batched_tensor", "gemm", "trpca",
           "LowRankSpec", "shifted_square", "gaussian", "StreamCall", "stream_specs"]


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def normal(rng: np.random.Generator, shape, std: float = 1.0) -> np.ndarray:
    """iid N(0, std^2) float32 array of the given (n1, n2, n3) shape, Fortran order.

    Drawn in float64 in Fortran element order and rounded once to float32.
    """
    n = int(np.prod(shape))
    x = rng.standard_normal(n) * std
    return np.asarray(x, dtype=np.float32).reshape(shape, order="F")


def small(seed: int = 0) -> dict:
    """64x64x16 tubal-rank-4 factors plus noise; tau = 0.5."""
    rng = _rng(seed)
    P = normal(rng, (64, 4, 16))
    Q = normal(rng, (4, 64, 16))
    E = normal(rng, (64, 64, 16), 0.01)
    return {"P": P, "Q": Q, "E": E, "tau": 0.5, "rank": 4}


@dataclass(frozen=True)
class LowRankSpec:
    n1: int
    n2: int
    n3: int
    r: int
    noise: float
    tau: float


def batched_specs(count: int = 512, seed: int = 0, n_lo: int = 16, n_hi: int = 160,
                  n3_lo: int = 4, n3_hi: int = 64, r_lo: int = 2, r_hi: int = 12,
                  noise: float = 0.05) -> list[LowRankSpec]:
    """Sizes, ranks and thresholds of the batched workload (no tensor data)."""
    rng = _rng(seed)
    n1 = rng.integers(n_lo, n_hi + 1, size=count)
    n2 = rng.integers(n_lo, n_hi + 1, size=count)
    n3 = rng.integers(n3_lo, n3_hi + 1, size=count)
    r = rng.integers(r_lo, r_hi + 1, size=count)
    out = []
    for t in range(count):
        nu = noise * np.sqrt(n3[t]) * (np.sqrt(n1[t]) + np.sqrt(n2[t]))
        out.append(LowRankSpec(int(n1[t]), int(n2[t]), int(n3[t]), int(r[t]), noise,
                               float(2.0 * nu)))
    return out


def batched_tensor(spec: LowRankSpec, index: int, seed: int = 0) -> dict:
    """Factors P (n1 x r x n3), Q (r x n2 x n3) and noise E of tensor `index`."""
    child = np.random.SeedSequence(seed).spawn(index + 1)[index]
    rng = _rng(child)
    P = normal(rng, (spec.n1, spec.r, spec.n3))
    Q = normal(rng, (spec.r, spec.n2, spec.n3))
    E = normal(rng, (spec.n1, spec.n2, spec.n3), spec.noise)
    return {"P": P, "Q": Q, "E": E, "tau": spec.tau, "rank": spec.r}


@dataclass(frozen=True)
class StreamCall:
    op: str          # "prox" (prox_tnn of a) or "tprod" (a * b)
    a: LowRankSpec   # n1 x n2 x n3
    b: LowRankSpec | None  # tprod: n2 x l x n3


def stream_specs(count: int = 2000, seed: int = 0, n_lo: int = 16, n_hi: int = 512,
                 n3_lo: int = 4, n3_hi: int = 256, r_lo: int = 4, r_hi: int = 40,
                 noise: float = 0.02) -> list[StreamCall]:
    """Sizes, ranks and thresholds of the mixed call stream (no tensor data)."""
    rng = _rng(seed)
    out = []
    for _ in range(count):
        op = "prox" if rng.integers(0, 2) == 0 else "tprod"
        n1, n2, l = (int(v) for v in rng.integers(n_lo, n_hi + 1, size=3))
        n3 = int(rng.integers(n3_lo, n3_hi + 1))
        ra, rb = (int(v) for v in rng.integers(r_lo, r_hi + 1, size=2))

        def spec(p, q, r):
            nu = noise * np.sqrt(n3) * (np.sqrt(p) + np.sqrt(q))
            return LowRankSpec(p, q, n3, r, noise, float(2.0 * nu))

        out.append(StreamCall(op, spec(n1, n2, ra), spec(n2, l, rb) if op == "tprod" else None))
    return out


def gemm(seed: int = 0, n1: int = 2048, n2: int = 1024, l: int = 1024, n3: int = 64) -> dict:
    """A (n1 x n2 x n3) and B (n2 x l x n3), iid N(0,1)."""
    rng = _rng(seed)
    return {"A": normal(rng, (n1, n2, n3)), "B": normal(rng, (n2, l, n3))}


def trpca(seed: int = 0, n1: int = 240, n2: int = 320, n3: int = 100, r: int = 10,
          frac: float = 0.1, amp: float = 5.0) -> dict:
    """Factors of the low-rank part, plus sparse corruption positions and values.

    The low-rank part is meant to be scaled to unit RMS after the t-product.
    """
    rng = _rng(seed)
    P = normal(rng, (n1, r, n3))
    Q = normal(rng, (r, n2, n3))
    n = n1 * n2 * n3
    pos = rng.choice(n, size=int(round(frac * n)), replace=False)
    val = rng.uniform(-amp, amp, size=pos.size).astype(np.float32)
    tau = 1.0 / np.sqrt(max(n1, n2) * n3)
    return {"P": P, "Q": Q, "pos": pos, "val": val, "tau": float(tau), "rank": r}


def shifted_square(n: int, n3: int, seed: int = 0) -> np.ndarray:
    """n x n x n3: iid N(0, 1/(16 n n3)) entries plus 1 on the diagonal of frontal slice 0."""
    X = normal(_rng(seed), (n, n, n3), 1.0 / (4.0 * np.sqrt(n * max(n3, 1))))
    if n > 0 and n3 > 0:
        X[np.arange(n), np.arange(n), 0] += np.float32(1.0)
    return X


def gaussian(n1: int, n2: int, n3: int, seed: int = 0) -> np.ndarray:
    """n1 x n2 x n3 iid N(0, 1)."""
    return normal(_rng(seed), (n1, n2, n3))
