"""prox_tnn with the learned rank proposer and randomized SVT (TP_METHOD_LEARNED).

The plain Jacobi path is the fallback and the accuracy reference: every slice the sketch
path does not certify is recomputed by it.  Bound for this mixed form: 1e-4 relative
Frobenius error against the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import tproduct as O
from tests.helpers import TOL_FP32, batched_inputs, low_rank, median_sigma, randn, rel

pytestmark = pytest.mark.gpu
TOL_LEARNED = 1e-4


@pytest.fixture(scope="module")
def tp():
    import os

    from paper_1806_07247_gb300 import build, tp as _tp
    if not os.path.exists(_tp.LIB_PATH):
        build.build()
    _tp.lib()
    return _tp


def _train(tp, count=96, seed=1000):
    items = batched_inputs(count, seed=seed)
    return tp.proposer_train([tp.to_device(X) for _, X in items], [s.tau for s, _ in items],
                             steps=300, seed=7)


def test_learned_requires_a_trained_proposer(tp):
    Y = tp.to_device(randn((20, 16, 4), 1))
    try:
        tp.proposer_get()
        trained = True
    except tp.TpError:
        trained = False
    if trained:
        pytest.skip("a proposer is already loaded in this process")
    with pytest.raises(tp.TpError) as e:
        tp.prox_tnn_batched([Y], [1.0], opts=tp.options(method="learned"))
    assert e.value.status == tp.TP_ERR_INVALID_ARG


def test_train_and_roundtrip(tp):
    mse = _train(tp)
    assert np.isfinite(mse) and mse < 4.0, mse      # counts are within ~2 of the labels
    w = tp.proposer_get()
    assert w.shape == (tp.PROPOSER_FLOATS,) and np.isfinite(w).all()
    tp.proposer_set(w)
    np.testing.assert_array_equal(tp.proposer_get(), w)


def test_learned_prox_matches_oracle_on_low_rank_batch(tp):
    import torch
    _train(tp)
    items = batched_inputs(32, seed=0)
    Ys = [tp.to_device(X) for _, X in items]
    nsl = sum(s.n3 // 2 + 1 for s, _ in items)
    flags = torch.full((nsl,), -1, dtype=torch.int32, device="cuda")
    outs = tp.prox_tnn_batched(Ys, [s.tau for s, _ in items],
                               opts=tp.options(method="learned", slice_flags_out=flags))
    for (s, X), out in zip(items, outs):
        assert rel(tp.to_numpy(out), O.prox_tnn(X, s.tau)) < TOL_LEARNED, s
    f = flags.cpu().numpy()
    assert set(np.unique(f)) <= {0, 1}
    # low rank plus noise with tau at twice the noise level: most slices certify
    assert (f == 0).mean() > 0.5, (f == 0).mean()


def test_learned_prox_falls_back_on_full_rank_inputs(tp):
    import torch
    _train(tp)
    shapes = [(40, 33, 6), (64, 64, 4), (20, 90, 5)]
    Ys = [randn(sh, i) for i, sh in enumerate(shapes)]
    taus = [median_sigma(Y) for Y in Ys]
    nsl = sum(sh[2] // 2 + 1 for sh in shapes)
    flags = torch.full((nsl,), -1, dtype=torch.int32, device="cuda")
    outs = tp.prox_tnn_batched([tp.to_device(Y) for Y in Ys], taus,
                               opts=tp.options(method="learned", slice_flags_out=flags))
    for Y, tau, out in zip(Ys, taus, outs):
        assert rel(tp.to_numpy(out), O.prox_tnn(Y, tau)) < TOL_FP32
    assert (flags.cpu().numpy() == 1).all()


def test_learned_prox_on_large_slices(tp):
    # slices of the mixed call stream's sizes (up to 512, ranks up to 40): the sketch path
    # takes those whose width fits a size class, the rest fall back to the global-memory
    # Jacobi; every output must still be the prox of Algorithm 3 within the mixed-form bound
    import torch

    from paper_1806_07247_gb300 import synth
    _train(tp)
    specs = []
    for (n1, n2, n3), r in zip([(512, 300, 3), (300, 512, 4), (480, 440, 2), (512, 512, 1),
                                (350, 260, 5)], [8, 20, 36, 6, 12]):
        nu = 0.02 * np.sqrt(n3) * (np.sqrt(n1) + np.sqrt(n2))
        specs.append(synth.LowRankSpec(n1, n2, n3, r, 0.02, float(2.0 * nu)))
    Xs = [low_rank(synth.batched_tensor(s, i, seed=5)) for i, s in enumerate(specs)]
    nsl = sum(s.n3 // 2 + 1 for s in specs)
    flags = torch.full((nsl,), -1, dtype=torch.int32, device="cuda")
    outs = tp.prox_tnn_batched([tp.to_device(X) for X in Xs], [s.tau for s in specs],
                               opts=tp.options(method="learned", slice_flags_out=flags))
    for s, X, out in zip(specs, Xs, outs):
        assert rel(tp.to_numpy(out), O.prox_tnn(X, s.tau)) < TOL_LEARNED, s
    assert set(np.unique(flags.cpu().numpy())) <= {0, 1}
