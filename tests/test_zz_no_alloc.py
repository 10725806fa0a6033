"""tp_prox_tnn_noalloc: the allocation-free variant of prox_tnn, for callers that cannot
allocate device memory while they run (its scratch is one fixed static device array).

It must give the same result as tp_prox_tnn (the allocating entry point) within the FP32
tolerance the other parity tests use, on two calls in a row with different inputs (the
second call must not be disturbed by what the first left in the shared array).  This file
is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from tests.helpers import TOL_FP32, median_sigma, randn, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    import os

    from paper_1806_07247_gb300 import build, tp as _tp
    if not os.path.exists(_tp.LIB_PATH):
        build.build()
    _tp.lib()
    return _tp


def _call_noalloc(tp, Y, X, tau):
    """Straight through the C ABI: device pointers, sizes, the current stream."""
    import torch
    n1, n2, n3 = Y.shape
    st = tp.lib().tp_prox_tnn_noalloc(ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                      n1, n2, n3, float(tau), None,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_matches_allocating_entry_point_twice(tp):
    # two different tensors; the allocating entry point gives the references first, then the
    # allocation-free one is called twice in a row.  The second tensor is larger, so stale
    # spectrum left by call 1 would sit inside call 2's region if it were not rewritten.
    cases = [((40, 33, 9), 1), ((64, 80, 16), 2)]
    ins, refs, outs, taus = [], [], [], []
    for shape, seed in cases:
        Y = randn(shape, seed)
        taus.append(median_sigma(Y))
        ins.append(tp.to_device(Y))
        refs.append(tp.to_numpy(tp.prox_tnn(ins[-1], taus[-1])))
        outs.append(tp.empty(*shape))
    for dY, dX, tau in zip(ins, outs, taus):
        assert _call_noalloc(tp, dY, dX, tau) == tp.TP_OK
    for dX, ref in zip(outs, refs):
        got = tp.to_numpy(dX)
        assert np.isfinite(got).all()
        assert rel(got, ref) < TOL_FP32


def test_noalloc_rejects_sizes_beyond_the_array(tp):
    # 160 x 160 x 256: 160*160*129*8 bytes = 26 MB of spectrum > 16 MiB
    Y = tp.empty(160, 160, 256)
    X = tp.empty(160, 160, 256)
    assert _call_noalloc(tp, Y, X, 1.0) == tp.TP_ERR_UNSUPPORTED
