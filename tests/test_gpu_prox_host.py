"""GPU tests of tp_prox_tnn_batched_host: tensors in host memory, copied in and out by the
library in overlapped chunks.  The results must match the device-memory batched call on the
same tensors (the same kernels run on every slice) and the FP64 oracle within TOL_FP32."""
import numpy as np
import pytest
import torch

from oracle import tproduct as O
from tests.helpers import TOL_FP32, batched_inputs, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    import os

    from paper_1806_07247_gb300 import build, tp as _tp
    if not os.path.exists(_tp.LIB_PATH):
        build.build()
    _tp.lib()
    return _tp


@pytest.fixture(scope="module")
def batch():
    # about 60 MB of tensors: several 16 MiB chunks
    items = batched_inputs(60, seed=4)
    return [Y for _, Y in items], [s.tau for s, _ in items]


def _host_slab(tp, Ys):
    slab, views = tp.pinned_tensors([Y.shape for Y in Ys])
    for v, Y in zip(views, Ys):
        v.copy_(torch.from_numpy(np.ascontiguousarray(Y.transpose(2, 1, 0))).permute(2, 1, 0))
    return slab, views


def _np(t):
    return t.permute(2, 1, 0).contiguous().numpy().transpose(2, 1, 0)


@pytest.mark.parametrize("method,parts", [("jacobi", 2), ("learned", 2), ("jacobi", 1),
                                          ("learned", 1)])
def test_host_matches_device(tp, batch, method, parts):
    Ys, taus = batch
    if method == "learned":
        tp.proposer_train([tp.to_device(Y) for Y in Ys[:24]], taus[:24], steps=200, seed=1)
    _, hin = _host_slab(tp, Ys)
    houts = tp.prox_tnn_batched_host(hin, taus, opts=tp.options(method=method, host_parts=parts))
    douts = tp.prox_tnn_batched([tp.to_device(Y) for Y in Ys], taus, opts=tp.options(method=method))
    worst = max(rel(_np(h), tp.to_numpy(d)) for h, d in zip(houts, douts))
    assert worst < 1e-6, worst
    for i in (0, 17, 59):
        assert rel(_np(houts[i]), O.prox_tnn(Ys[i].astype(np.float64), taus[i])) < \
            (TOL_FP32 if method == "jacobi" else 1e-4)


def test_host_layouts_and_aliasing(tp, batch):
    """Separate (non-contiguous) pinned buffers, a pageable buffer, in == out, and an empty
    tensor in the middle of the list."""
    Ys, taus = batch
    sel = [Y for Y in Ys[:5]]
    ins = []
    for i, Y in enumerate(sel):
        t = torch.from_numpy(np.ascontiguousarray(Y.transpose(2, 1, 0))).permute(2, 1, 0)
        ins.append(t.pin_memory() if i % 2 == 0 else t.clone())
    empty = torch.zeros((0, 4, 3), dtype=torch.float32)
    ins.insert(2, empty)
    tau = [taus[0], taus[1], 0.1, taus[2], taus[3], taus[4]]
    outs = [x for x in ins]          # fully in place
    tp.prox_tnn_batched_host(ins, tau, outs=outs)
    for k, Y in zip([0, 1, 3, 4, 5], sel):
        i = k if k < 2 else k - 1
        assert rel(_np(outs[k]), O.prox_tnn(Y.astype(np.float64), taus[i])) < TOL_FP32


def test_host_sweeps_indexing(tp, batch):
    """sweeps_out is indexed over the whole batch although the call runs in chunks."""
    Ys, taus = batch
    _, hin = _host_slab(tp, Ys)
    slices = sum(Y.shape[2] // 2 + 1 for Y in Ys)
    sw_h = torch.full((slices,), -1, dtype=torch.int32, device="cuda")
    sw_d = torch.full((slices,), -1, dtype=torch.int32, device="cuda")
    tp.prox_tnn_batched_host(hin, taus, opts=tp.options(sweeps_out=sw_h))
    tp.prox_tnn_batched([tp.to_device(Y) for Y in Ys], taus, opts=tp.options(sweeps_out=sw_d))
    assert torch.equal(sw_h, sw_d)
    assert int(sw_h.min()) >= 1


def test_host_rejects_bad_args(tp):
    d = (tp.TensorDesc * 1)()
    d[0].n1, d[0].n2, d[0].n3, d[0].tau = 4, 4, 4, 0.5
    o = tp.options()
    assert tp.lib().tp_prox_tnn_batched_host(d, 1, tp.ctypes.byref(o), None) == tp.TP_ERR_INVALID_ARG
    d[0].n1 = -1
    assert tp.lib().tp_prox_tnn_batched_host(d, 1, tp.ctypes.byref(o), None) == tp.TP_ERR_INVALID_ARG
    assert tp.lib().tp_prox_tnn_batched_host(d, 0, tp.ctypes.byref(o), None) == tp.TP_OK


# ----------------------------------------------------------------------------- replayable plans
@pytest.mark.parametrize("method", ["jacobi", "learned"])
def test_plan_replays_the_batched_call(tp, batch, method):
    """A recorded plan gives the batched call's result, follows new input contents, and
    reports through the same status path."""
    Ys, taus = batch
    Ys, taus = Ys[:24], taus[:24]
    if method == "learned":
        tp.proposer_train([tp.to_device(Y) for Y in Ys], taus, steps=200, seed=1)
    dY = [tp.to_device(Y) for Y in Ys]
    plan = tp.ProxPlan(dY, taus, opts=tp.options(method=method))
    ref = tp.prox_tnn_batched(dY, taus, opts=tp.options(method=method))
    for _ in range(2):
        out = plan.run()
        worst = max(rel(tp.to_numpy(a), tp.to_numpy(b)) for a, b in zip(out, ref))
        assert worst < 1e-6, worst
    # new contents in the same tensors
    for Y in dY:
        Y.mul_(0.5)
    out = plan.run()
    for i in (0, 11, 23):
        assert rel(tp.to_numpy(out[i]), O.prox_tnn(0.5 * Ys[i].astype(np.float64), taus[i])) < \
            (TOL_FP32 if method == "jacobi" else 1e-4)
    plan.close()


def test_plan_rejects_stage_events(tp):
    Y = tp.to_device(np.ones((4, 4, 3), dtype=np.float32, order="F"))
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(tp.STAGE_EVENTS)]
    for e in evs:
        e.record()
    with pytest.raises(tp.TpError) as e:
        tp.ProxPlan([Y], [0.1], opts=tp.options(stage_events=evs))
    assert e.value.status == tp.TP_ERR_INVALID_ARG
