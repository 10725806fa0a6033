"""Tensor-core (tcgen05) slice GEMMs of tprod in split precision, against the FP64 oracle.

Bound: 1e-4 relative Frobenius error for the mixed-precision forms (BF16x3, 3xTF32 with
FP32 accumulation); 3xTF32 is expected near the FP32 path (~1e-6), BF16x3 near 1e-5.
"""
import numpy as np
import pytest

from oracle import tproduct as O
from tests.helpers import randn, rel

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-4


@pytest.fixture(scope="module")
def tp():
    import os

    from paper_1806_07247_gb300 import build, tp as _tp
    if not os.path.exists(_tp.LIB_PATH):
        build.build()
    _tp.lib()
    return _tp


# power-of-two n3 <= 64 (the forward DFT writes the BF16 operand planes itself) and other n3
# (the planes are filled from the complex spectrum); M, K and N tails of every size
SHAPES = [(128, 64, 128, 1), (1, 1, 1, 1), (200, 100, 150, 3), (64, 4, 64, 16),
          (129, 65, 257, 2), (300, 200, 130, 5), (37, 129, 45, 17), (256, 512, 256, 8),
          (100, 70, 90, 4), (130, 33, 70, 64), (7, 9, 3, 32)]


@pytest.mark.parametrize("precision", ["bf16x3", "3xtf32"])
@pytest.mark.parametrize("dims", SHAPES)
def test_tprod_tensor_core_parity(tp, dims, precision):
    n1, n2, l, n3 = dims
    A, B = randn((n1, n2, n3), 3 + n1), randn((n2, l, n3), 4 + l)
    C = tp.to_numpy(tp.tprod(tp.to_device(A), tp.to_device(B), precision=precision))
    ref = O.tprod_fourier(A, B)
    err = rel(C, ref)
    assert err < TOL_MIXED, err
    if precision == "3xtf32":
        assert err < 1e-5, err


def test_tprod_tensor_core_full_size_sampled(tp):
    """2048x1024x64 times 1024x1024x64 (the GEMM bench size), sampled entries of Eq. 9."""
    from paper_1806_07247_gb300 import synth
    g = synth.gemm(0)
    dA, dB = tp.to_device(g["A"]), tp.to_device(g["B"])
    rng = np.random.default_rng(2)
    idx = np.stack([rng.integers(0, 2048, 400), rng.integers(0, 1024, 400),
                    rng.integers(0, 64, 400)], axis=1)
    ref = O.tprod_entries(g["A"], g["B"], idx)
    for precision in ("bf16x3", "3xtf32"):
        C = tp.tprod(dA, dB, precision=precision)
        got = C[idx[:, 0], idx[:, 1], idx[:, 2]].double().cpu().numpy()
        assert rel(got, ref) < TOL_MIXED, precision
