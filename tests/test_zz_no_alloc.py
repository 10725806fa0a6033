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

from oracle import tproduct as O
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
    for dX, ref, (shape, seed), tau in zip(outs, refs, cases, taus):
        got = tp.to_numpy(dX)
        assert np.isfinite(got).all()
        assert rel(got, ref) < TOL_FP32
        # and against the FP64 oracle (Algorithm 3 on all n3 slices)
        assert rel(got, O.prox_tnn(randn(shape, seed), tau)) < TOL_FP32


def test_noalloc_slices_larger_than_shared_memory_in_place_with_outputs(tp):
    # 256 x 256 slices do not fit in shared memory, so each slice's working matrix sits in the
    # static array after the spectrum; the call runs in place (X == Y) and fills sweeps_out
    # and counts_out, all compared with the allocating entry point and the oracle
    import torch
    shape = (256, 256, 3)
    Y = randn(shape, 21)
    tau = median_sigma(Y)
    h = shape[2] // 2 + 1
    sw_ref = torch.full((h,), -1, dtype=torch.int32, device="cuda")
    ct_ref = torch.full((h,), -1, dtype=torch.int32, device="cuda")
    ref = tp.to_numpy(tp.prox_tnn(tp.to_device(Y), tau,
                                  opts=tp.options(sweeps_out=sw_ref, counts_out=ct_ref)))
    dX = tp.to_device(Y)
    sw = torch.full((h,), -1, dtype=torch.int32, device="cuda")
    ct = torch.full((h,), -1, dtype=torch.int32, device="cuda")
    o = tp.options(sweeps_out=sw, counts_out=ct)
    st = tp.lib().tp_prox_tnn_noalloc(ctypes.c_void_p(dX.data_ptr()), ctypes.c_void_p(dX.data_ptr()),
                                      *shape, float(tau), ctypes.byref(o),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == tp.TP_OK
    got = tp.to_numpy(dX)
    assert rel(got, ref) < TOL_FP32
    assert rel(got, O.prox_tnn(Y, tau)) < TOL_FP32
    # sweeps: the allocating call may run under an autotuned CTA shape (rounding order only)
    assert (sw.cpu().numpy() > 0).all()
    assert (np.abs(sw.cpu().numpy() - sw_ref.cpu().numpy()) <= 1).all()
    np.testing.assert_array_equal(ct.cpu().numpy(), ct_ref.cpu().numpy())
    np.testing.assert_array_equal(ct.cpu().numpy(), O.slice_counts(Y, tau))


def test_noalloc_rejects_sizes_beyond_the_array(tp):
    # 160 x 160 x 256: 160*160*129*8 bytes = 26 MB of spectrum > 16 MiB
    Y = tp.empty(160, 160, 256)
    X = tp.empty(160, 160, 256)
    assert _call_noalloc(tp, Y, X, 1.0) == tp.TP_ERR_UNSUPPORTED
