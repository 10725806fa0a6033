"""GPU checks of the Jacobi CTA-shape autotuner (tp_autotune_jacobi) and of the shapes it
chooses between: every candidate shape must give the prox of Algorithm 3 (and the singular
values behind tnn, Def. 2.9) within the plain path's TOL_FP32 of the FP64 oracle, the
autotuner must leave the device on one of its candidates, and the default must come back.
"""
import numpy as np
import pytest

from oracle import tproduct as O
from tests.helpers import TOL_FP32, batched_inputs, median_sigma, randn, rel

pytestmark = pytest.mark.gpu

DEFAULT = {"target_lane_pairs": 5, "max_warps": 32, "split_launches": 0}


@pytest.fixture(scope="module")
def tp():
    import os

    from paper_1806_07247_gb300 import build, tp as _tp
    if not os.path.exists(_tp.LIB_PATH):
        build.build()
    _tp.lib()
    yield _tp
    _tp.jacobi_shape_set(None)


def _mixed_batch():
    """Low-rank batched tensors plus two shapes that reach the other kernel variants: a wide
    slice (Jacobi on the conjugate transpose) and one too large for shared memory."""
    items = [(Y, float(s.tau)) for s, Y in batched_inputs(6, seed=3)]
    for shape, seed in [((24, 150, 5), 11), ((260, 230, 3), 12)]:
        Y = randn(shape, seed)
        items.append((Y, median_sigma(Y)))
    return items


@pytest.mark.parametrize("shape", [(3, 8, 1), (7, 16, 0), (5, 8, 1), (3, 32, 1), (7, 32, 0)])
def test_prox_parity_under_each_shape(tp, shape):
    items = _mixed_batch()
    tp.jacobi_shape_set(dict(zip(DEFAULT, shape)))
    try:
        outs = tp.prox_tnn_batched([tp.to_device(Y) for Y, _ in items], [t for _, t in items])
        for (Y, tau), X in zip(items, outs):
            assert rel(tp.to_numpy(X), O.prox_tnn(Y, tau)) < TOL_FP32
    finally:
        tp.jacobi_shape_set(None)


def test_tnn_under_a_split_shape(tp):
    Y = randn((90, 70, 9), 5)
    tp.jacobi_shape_set({"target_lane_pairs": 3, "max_warps": 8, "split_launches": 1})
    try:
        got = float(tp.tnn(tp.to_device(Y)).item())
    finally:
        tp.jacobi_shape_set(None)
    ref = O.tnn(Y)
    assert abs(got - ref) / ref < TOL_FP32


def test_autotune_chooses_a_candidate_and_results_hold(tp):
    items = _mixed_batch()
    Ys = [tp.to_device(Y) for Y, _ in items]
    taus = [t for _, t in items]
    before = [tp.to_numpy(Y).copy() for Y in Ys]
    shape, default_ms, chosen_ms = tp.autotune_jacobi(Ys, taus, reps=1)
    assert shape["target_lane_pairs"] in (3, 5, 7)
    assert shape["max_warps"] in (8, 16, 32)
    assert shape["split_launches"] in (0, 1)
    assert 0 < chosen_ms <= default_ms
    assert tp.jacobi_shape_get() == shape
    # the tuned tensors are read only
    for Y, b in zip(Ys, before):
        assert np.array_equal(tp.to_numpy(Y), b)
    try:
        outs = tp.prox_tnn_batched(Ys, taus)
        for (Y, tau), X in zip(items, outs):
            assert rel(tp.to_numpy(X), O.prox_tnn(Y, tau)) < TOL_FP32
        # a plan recorded under the tuned shape replays to the same result
        plan = tp.ProxPlan(Ys, taus)
        try:
            for X, ref in zip(plan.run(), outs):
                assert rel(tp.to_numpy(X), tp.to_numpy(ref)) < TOL_FP32
        finally:
            plan.close()
    finally:
        tp.jacobi_shape_set(None)
    assert tp.jacobi_shape_get() == DEFAULT
