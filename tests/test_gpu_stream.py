"""Sampled calls of the mixed call stream (prox_tnn or tprod; n1, n2 up to 512, n3 up to 256,
tubal rank 4..40 plus noise) through the combined path the bench times -- learned prox from a
replayed CUDA-graph plan, BF16x3 tensor-core tprod -- against the FP64 oracle (Algorithm 3 on
all n3 slices; the t-product of Eq. 10).  Bound: 1e-4 relative Frobenius error, the bound of
the mixed-precision forms.  The calls are the stream's own, taken in stream order among those
small enough for the oracle to finish in seconds.
"""
import numpy as np
import pytest

from oracle import tproduct as O
from paper_1806_07247_gb300 import synth
from tests.helpers import low_rank, rel

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-4
MAX_ENTRIES = 2_500_000   # n1 n2 n3 of every operand of a sampled call


@pytest.fixture(scope="module")
def tp():
    import os

    from paper_1806_07247_gb300 import build, tp as _tp
    if not os.path.exists(_tp.LIB_PATH):
        build.build()
    _tp.lib()
    return _tp


def _small(spec):
    return spec is None or spec.n1 * spec.n2 * spec.n3 <= MAX_ENTRIES


def _sample(op, count, seed):
    calls = [c for c in synth.stream_specs(400, seed=seed)
             if c.op == op and _small(c.a) and _small(c.b)]
    return calls[:count]


def test_stream_prox_calls_learned_plan_against_oracle(tp):
    # proposer trained on prox calls of another draw of the stream (as the bench does)
    train = _sample("prox", 24, seed=1)
    tY = [tp.to_device(low_rank(synth.batched_tensor(c.a, i, 1))) for i, c in enumerate(train)]
    tp.proposer_train(tY, [c.a.tau for c in train], steps=300, seed=3)
    calls = _sample("prox", 5, seed=0)
    Ys = [low_rank(synth.batched_tensor(c.a, i, 0)) for i, c in enumerate(calls)]
    plan = tp.ProxPlan([tp.to_device(Y) for Y in Ys], [c.a.tau for c in calls],
                       opts=tp.options(method="learned"))
    try:
        outs = plan.run()
        import torch
        torch.cuda.synchronize()
        for Y, c, X in zip(Ys, calls, outs):
            err = rel(tp.to_numpy(X), O.prox_tnn(Y, c.a.tau))
            assert err < TOL_MIXED, (c.a, err)
    finally:
        plan.close()


def test_stream_tprod_calls_bf16x3_against_oracle(tp):
    for i, c in enumerate(_sample("tprod", 3, seed=0)):
        A = low_rank(synth.batched_tensor(c.a, 2 * i, 0))
        B = low_rank(synth.batched_tensor(c.b, 2 * i + 1, 0))
        C = tp.to_numpy(tp.tprod(tp.to_device(A), tp.to_device(B), precision="bf16x3"))
        err = rel(C, O.tprod_fourier(A, B))
        assert err < TOL_MIXED, (c.a, c.b, err)
