"""Per-slice counts #{sigma > tau} (Algorithm 3's kept singular values) against the FP64
oracle, exactly.

Two kinds of input:
* planted spectra: every independent Fourier slice is U diag(s) with orthonormal U and
  singular values s that include tau (1 + 5e-7) and tau (1 - 5e-7); the GPU decides those
  two from column norms accumulated in FP64 (a sigma within 1e-6 relative of tau is
  re-decided), so its counts must equal the oracle's on every slice;
* the gapped low-rank-plus-noise tensors of the batched workload (tau at twice the noise
  level), plain and learned methods.
"""
import numpy as np
import pytest

from oracle import tproduct as O
from paper_1806_07247_gb300 import synth
from tests.helpers import batched_inputs, randn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    import os

    from paper_1806_07247_gb300 import build, tp as _tp
    if not os.path.exists(_tp.LIB_PATH):
        build.build()
    _tp.lib()
    return _tp


def planted(n1, n2, n3, tau, seed):
    """Real n1 x n2 x n3 tensor (FP32) whose free Fourier slices are U_k diag(s_k), U_k with
    orthonormal columns (real on the real slices of Eq. 8), s_k holding tau (1 +- 5e-7) and
    values well away from tau; the mirrored slices are the conjugates (Lemma 2.1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = O.n_free_slices(n3)
    Ab = np.zeros((n1, n2, n3), dtype=np.complex128)
    for k in range(h):
        real = k == 0 or 2 * k == n3
        m, r = max(n1, n2), min(n1, n2)
        g = synth.normal(rng, (m, r, 1))[:, :, 0].astype(np.float64)
        if not real:
            g = g + 1j * synth.normal(rng, (m, r, 1))[:, :, 0].astype(np.float64)
        u, _ = np.linalg.qr(g)  # m x r, orthonormal columns
        base = np.array([tau * (1 + 5e-7), tau * (1 - 5e-7), 3 * tau, 0.3 * tau, 1.7 * tau,
                         0.6 * tau, 2.4 * tau, 0.1 * tau])
        s = base[(np.arange(r) + k) % len(base)]
        Ab[:, :, k] = u * s if n1 >= n2 else (u * s).conj().T
        if 0 < k and 2 * k != n3:
            Ab[:, :, n3 - k] = np.conj(Ab[:, :, k])
    A = O.ifft3(Ab)
    assert np.abs(A.imag).max() < 1e-12 * np.abs(A.real).max()
    return np.asfortranarray(A.real.astype(np.float32))


@pytest.mark.parametrize("shape", [(48, 6, 4), (40, 8, 2), (33, 5, 3), (6, 48, 4)])
def test_counts_exact_with_sigma_at_tau_plus_minus_5e7(tp, shape):
    import torch
    n1, n2, n3 = shape
    tau = 2.0
    A = planted(n1, n2, n3, tau, seed=n1 + 7 * n2 + n3)
    ref = O.slice_counts(A, tau)
    # the construction: each slice holds exactly one of the two near-tau values above tau
    # among its min(n1, n2) planted values (the oracle sees them on the FP32-rounded input)
    r = min(n1, n2)
    for k in range(O.n_free_slices(n3)):
        base = np.array([1 + 5e-7, 1 - 5e-7, 3, 0.3, 1.7, 0.6, 2.4, 0.1])
        assert ref[k] == int(np.sum(base[(np.arange(r) + k) % 8] > 1)), (k, ref)
    h = O.n_free_slices(n3)
    counts = torch.full((h,), -1, dtype=torch.int32, device="cuda")
    tp.prox_tnn(tp.to_device(A), tau, opts=tp.options(counts_out=counts))
    np.testing.assert_array_equal(counts.cpu().numpy(), ref)
    # the allocation-free entry point writes the same counts
    counts.fill_(-1)
    tp.prox_tnn_noalloc(tp.to_device(A), tau, opts=tp.options(counts_out=counts))
    np.testing.assert_array_equal(counts.cpu().numpy(), ref)


def test_counts_exact_with_fp64_rotations(tp):
    import torch
    A = planted(48, 6, 4, 2.0, seed=3)
    counts = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    tp.prox_tnn(tp.to_device(A), 2.0, opts=tp.options(counts_out=counts, jacobi_fp64=True))
    np.testing.assert_array_equal(counts.cpu().numpy(), O.slice_counts(A, 2.0))


def _batch_counts(tp, items, method):
    import torch
    nsl = sum(s.n3 // 2 + 1 for s, _ in items)
    counts = torch.full((nsl,), -1, dtype=torch.int32, device="cuda")
    tp.prox_tnn_batched([tp.to_device(X) for _, X in items], [s.tau for s, _ in items],
                        opts=tp.options(method=method, counts_out=counts))
    return counts.cpu().numpy()


def test_counts_exact_on_gapped_batch_plain(tp):
    items = batched_inputs(40, seed=0)
    got = _batch_counts(tp, items, "jacobi")
    ref = np.concatenate([O.slice_counts(X, s.tau) for s, X in items])
    np.testing.assert_array_equal(got, ref)
    # gapped inputs: the count of every slice is the planted tubal rank
    assert (ref == np.concatenate([[s.r] * (s.n3 // 2 + 1) for s, _ in items])).all()


def test_counts_exact_on_gapped_batch_learned(tp):
    items = batched_inputs(96, seed=1000)
    tp.proposer_train([tp.to_device(X) for _, X in items], [s.tau for s, _ in items],
                      steps=300, seed=7)
    items = batched_inputs(40, seed=0)
    got = _batch_counts(tp, items, "learned")
    ref = np.concatenate([O.slice_counts(X, s.tau) for s, X in items])
    np.testing.assert_array_equal(got, ref)


def test_counts_on_full_rank_input_match_away_from_tau(tp):
    # no gap: a count may differ from the oracle's only through a sigma within 1e-6 of tau
    Y = randn((30, 20, 5), 11)
    sv = O.slice_singular_values(Y)[:3]
    tau = float(np.median(sv))
    import torch
    counts = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    tp.prox_tnn(tp.to_device(Y), tau, opts=tp.options(counts_out=counts))
    got = counts.cpu().numpy()
    ref = O.slice_counts(Y, tau)
    near = np.sum(np.abs(sv - tau) <= 1e-6 * tau, axis=1)
    assert (np.abs(got - ref) <= near).all(), (got, ref)
