"""GPU parity: every C-ABI operation against the FP64 oracle on the same seeded inputs.

Bars: tran is a permutation and must be bit-exact; the floating-point operations must be
within TOL_FP32 = 1e-5 relative Frobenius error of the oracle (plain FP32 path); integer
results (tubal rank on gapped inputs) must match exactly.  U and V of the t-SVD are not
unique, so they are checked through the paper's invariants (Eq. 12, Def. 2.5, Eq. 13)
and S elementwise.
"""
import ctypes

import numpy as np
import pytest

from oracle import tproduct as O
from tests.helpers import TOL_FP32, batched_inputs, low_rank, median_sigma, randn, rel, \
    small_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    import os

    from paper_1806_07247_gb300 import build, tp as _tp
    if not os.path.exists(_tp.LIB_PATH):
        build.build()
    _tp.lib()
    return _tp


def dev(tp, a):
    return tp.to_device(a)


def host(tp, t):
    return tp.to_numpy(t)


# ----------------------------------------------------------------------------- tprod
TPROD_SHAPES = [(1, 1, 1, 1), (3, 5, 7, 1), (17, 33, 9, 2), (65, 31, 70, 3), (64, 4, 64, 16),
                (128, 64, 96, 5), (37, 129, 45, 17), (100, 50, 80, 61), (8, 8, 8, 64),
                (33, 17, 5, 128), (16, 16, 16, 256), (5, 6, 7, 1024), (130, 70, 66, 4)]


@pytest.mark.parametrize("dims", TPROD_SHAPES)
def test_tprod_parity(tp, dims):
    n1, n2, l, n3 = dims
    A, B = randn((n1, n2, n3), 1 + n1), randn((n2, l, n3), 2 + l)
    C = host(tp, tp.tprod(dev(tp, A), dev(tp, B)))
    ref = O.tprod_fourier(A, B) if n1 * n2 * n3 > 4096 else O.tprod(A, B)
    assert C.shape == (n1, l, n3)
    assert rel(C, ref) < TOL_FP32


@pytest.mark.parametrize("n3", list(range(1, 65)) + [127, 251, 256])
def test_tprod_parity_every_tube_length(tp, n3):
    # every per-length DFT kernel (even lengths, two-tube odd lengths, direct odd primes) and
    # the direct kernel above 64, forward and inverse
    A, B = randn((13, 7, n3), 100 + n3), randn((7, 5, n3), 200 + n3)
    C = host(tp, tp.tprod(dev(tp, A), dev(tp, B)))
    assert rel(C, O.tprod_fourier(A, B)) < TOL_FP32


def test_batched_prox_mixed_tube_lengths_all_classes(tp):
    # one batched call over every n3 in 1..64: the DFT launches group the tensors by register
    # class; 20 x 31 = 620 tubes spans three CTAs of 256 tubes with a ragged tail
    Ys = [randn((20, 31, n3), 300 + n3) for n3 in range(1, 65)]
    taus = [median_sigma(Y) for Y in Ys]
    outs = tp.prox_tnn_batched([dev(tp, Y) for Y in Ys], taus)
    for Y, tau, out in zip(Ys, taus, outs):
        assert rel(host(tp, out), O.prox_tnn(Y, tau)) < TOL_FP32, Y.shape


@pytest.mark.parametrize("n3", [1, 2, 3, 4, 8, 9, 16, 32, 64, 65, 128])
def test_tprod_identity_tensor(tp, n3):
    # Def. 2.3: A * I = I * A = A; covers the register FFT sizes (powers of two <= 64) and the
    # direct DFT beside them
    A = randn((40, 24, n3), 3)
    Ct = host(tp, tp.tprod(dev(tp, A), dev(tp, O.teye(24, n3).astype(np.float32))))
    assert rel(Ct, A) < 1e-6
    Ct = host(tp, tp.tprod(dev(tp, O.teye(40, n3).astype(np.float32)), dev(tp, A)))
    assert rel(Ct, A) < 1e-6


def test_tprod_shape_mismatch(tp):
    with pytest.raises(ValueError):
        tp.tprod(tp.empty(3, 4, 5), tp.empty(5, 2, 5))


def test_tprod_empty_dims(tp):
    C = tp.empty(0, 3, 4)
    tp.tprod(tp.empty(0, 2, 4), tp.empty(2, 3, 4), out=C)
    # n2 = 0: the product is all zeros
    C = tp.empty(3, 4, 5)
    C.fill_(7.0)
    tp.tprod(tp.empty(3, 0, 5), tp.empty(0, 4, 5), out=C)
    assert float(C.abs().max()) == 0.0


# ----------------------------------------------------------------------------- tran
# multiples of 4 take the float4 64 x 64 tile path (with ragged tiles: 132, 68, 200), the rest
# the scalar 32 x 32 path
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 4), (33, 65, 7), (64, 64, 16), (100, 3, 1),
                                   (31, 97, 2), (4, 4, 3), (132, 68, 5), (200, 132, 1),
                                   (64, 200, 64), (8, 12, 256)])
def test_tran_bit_exact(tp, shape):
    A = randn(shape, 5)
    T = host(tp, tp.tran(dev(tp, A)))
    np.testing.assert_array_equal(T, O.tran(A))


def test_tran_reverse_order_law(tp):
    A, B = randn((20, 12, 6), 6), randn((12, 9, 6), 7)
    dA, dB = dev(tp, A), dev(tp, B)
    lhs = host(tp, tp.tran(tp.tprod(dA, dB)))
    rhs = host(tp, tp.tprod(tp.tran(dB), tp.tran(dA)))
    assert rel(lhs, rhs) < 1e-6


# ----------------------------------------------------------------------------- prox
PROX_SHAPES = [(1, 1, 1), (5, 3, 1), (3, 5, 2), (16, 16, 3), (24, 40, 4), (40, 24, 7),
               (64, 64, 16), (33, 97, 5), (97, 33, 6), (160, 160, 8), (160, 17, 33),
               (20, 150, 64), (129, 128, 2), (48, 48, 61)]


@pytest.mark.parametrize("shape", PROX_SHAPES)
def test_prox_parity(tp, shape):
    Y = randn(shape, sum(shape))
    tau = median_sigma(Y)
    X = host(tp, tp.prox_tnn(dev(tp, Y), tau))
    ref = O.prox_tnn(Y, tau)
    assert rel(X, ref) < TOL_FP32


@pytest.mark.parametrize("shape", [(200, 64, 4), (64, 300, 3), (260, 250, 2), (512, 40, 3)])
def test_prox_parity_large_slices(tp, shape):
    # slices too large for shared memory run with the working matrix in global memory
    Y = randn(shape, 11)
    tau = median_sigma(Y)
    X = host(tp, tp.prox_tnn(dev(tp, Y), tau))
    assert rel(X, O.prox_tnn(Y, tau)) < TOL_FP32


def test_prox_special_cases(tp):
    Y = randn((30, 20, 6), 12)
    dY = dev(tp, Y)
    assert rel(host(tp, tp.prox_tnn(dY, 0.0)), Y) < 1e-6
    big = O.tsn(Y) * 1.001
    assert float(tp.prox_tnn(dY, big).abs().max()) == 0.0
    Y1 = randn((25, 14, 1), 13)
    assert rel(host(tp, tp.prox_tnn(dev(tp, Y1), 1.5)), O.prox_tnn(Y1, 1.5)) < TOL_FP32


def test_prox_in_place(tp):
    Y = randn((45, 38, 9), 14)
    tau = median_sigma(Y)
    dY = dev(tp, Y)
    tp.prox_tnn(dY, tau, out=dY)
    assert rel(host(tp, dY), O.prox_tnn(Y, tau)) < TOL_FP32


def test_prox_small_workload(tp):
    f, X = small_inputs(0)
    Xp = host(tp, tp.prox_tnn(dev(tp, X), f["tau"]))
    assert rel(Xp, O.prox_tnn(X, f["tau"])) < TOL_FP32


def test_prox_rejects_bad_tau(tp):
    with pytest.raises(tp.TpError):
        tp.prox_tnn(dev(tp, randn((4, 4, 2), 1)), -1.0)


def test_prox_not_converged_status(tp):
    Y = randn((64, 64, 4), 15)
    with pytest.raises(tp.TpError) as e:
        tp.prox_tnn(dev(tp, Y), 1.0, opts=tp.options(max_sweeps=1))
    assert e.value.status == tp.TP_ERR_NOT_CONVERGED


def test_prox_batched_subset(tp):
    items = batched_inputs(24)
    Ys = [dev(tp, X) for _, X in items]
    taus = [s.tau for s, _ in items]
    outs = tp.prox_tnn_batched(Ys, taus)
    for (s, X), out in zip(items, outs):
        assert rel(host(tp, out), O.prox_tnn(X, s.tau)) < TOL_FP32, s


def test_prox_batched_ranks_on_gapped_inputs(tp):
    # tau = 2x the noise level puts a clear gap around tau: the output's tubal rank is r
    items = batched_inputs(8, seed=3)
    outs = tp.prox_tnn_batched([dev(tp, X) for _, X in items], [s.tau for s, _ in items])
    for (s, X), out in zip(items, outs):
        counts = O.slice_counts(X, s.tau)
        assert counts.max() == s.r
        rk, _ = tp.tubalrank(out, tol=1e-3 * s.tau)
        assert int(rk.item()) == s.r


def test_prox_batched_sweeps_out(tp):
    import torch
    items = batched_inputs(4, seed=5)
    nsl = sum(s.n3 // 2 + 1 for s, _ in items)
    sw = torch.full((nsl,), -1, dtype=torch.int32, device="cuda")
    tp.prox_tnn_batched([dev(tp, X) for _, X in items], [s.tau for s, _ in items],
                        opts=tp.options(sweeps_out=sw))
    sw = sw.cpu().numpy()
    assert np.all(sw >= 1) and np.all(sw <= 30)


def test_prox_batched_with_empty_and_in_place(tp):
    Y1, Y2 = randn((12, 9, 5), 1), randn((7, 15, 4), 2)
    d1, d2 = dev(tp, Y1), dev(tp, Y2)
    e = tp.empty(0, 5, 3)
    t1, t2 = median_sigma(Y1), median_sigma(Y2)
    tp.prox_tnn_batched([d1, e, d2], [t1, 0.5, t2], outs=[d1, e, d2])
    assert rel(host(tp, d1), O.prox_tnn(Y1, t1)) < TOL_FP32
    assert rel(host(tp, d2), O.prox_tnn(Y2, t2)) < TOL_FP32


# ----------------------------------------------------------------------------- tnn / tsn / rank
NORM_SHAPES = [(1, 1, 1), (6, 4, 1), (4, 6, 2), (64, 64, 16), (31, 77, 9), (120, 33, 64),
               (160, 160, 5), (300, 20, 3)]


@pytest.mark.parametrize("shape", NORM_SHAPES)
def test_tnn_tsn_parity(tp, shape):
    A = randn(shape, 21)
    dA = dev(tp, A)
    assert abs(float(tp.tnn(dA).item()) - O.tnn(A)) <= TOL_FP32 * O.tnn(A)
    assert abs(float(tp.tsn(dA).item()) - O.tsn(A)) <= TOL_FP32 * O.tsn(A)


def test_tubalrank_and_singular_values(tp):
    f, X = small_inputs(0)
    dX = dev(tp, X)
    s_ref = O.tubal_singular_values(X)
    rk, s = tp.tubalrank(dX, tol=5.0)
    assert int(rk.item()) == O.tubalrank(X, 5.0) == 4
    assert rel(s.cpu().numpy(), s_ref) < TOL_FP32
    # default tolerance (matrix-rank convention): ranks may differ only by tensor singular
    # values within the FP32 error of the tolerance itself
    rk, _ = tp.tubalrank(dX)
    tol = 64 * 2.0 ** -23 * s_ref[0]
    near = int(np.sum(np.abs(s_ref - tol) <= TOL_FP32 * s_ref[0]))
    assert abs(int(rk.item()) - O.tubalrank(X)) <= near


def test_scalars_empty_tensor(tp):
    import torch
    out = torch.full((1,), 3.0, dtype=torch.float64, device="cuda")
    tp.tnn(tp.empty(0, 4, 3), out=out)
    assert float(out.item()) == 0.0


# ----------------------------------------------------------------------------- tsvd
def _check_tsvd(tp, A, econ):
    n1, n2, n3 = A.shape
    r = min(n1, n2)
    U, S, V = tp.tsvd(dev(tp, A), econ=econ)
    U, S, V = host(tp, U), host(tp, S), host(tp, V)
    assert U.shape == ((n1, r, n3) if econ else (n1, n1, n3))
    assert V.shape == ((n2, r, n3) if econ else (n2, n2, n3))
    Ud, Sd, Vd = (x.astype(np.float64) for x in (U, S, V))
    # Eq. 12
    rec = O.tprod_fourier(O.tprod_fourier(Ud, Sd), O.tran(Vd))
    assert rel(rec, A) < TOL_FP32
    # Def. 2.5 (orthogonality), largest entry of Q^T * Q - I: the Jacobi convergence test
    # leaves normalised column products below max(8, sqrt(m)) * 2^-23 ~ 1e-6
    for Q in (Ud, Vd):
        k = Q.shape[1]
        G = O.tprod_fourier(O.tran(Q), Q)
        assert np.max(np.abs(G - O.teye(k, n3))) < TOL_FP32
    # S: f-diagonal, elementwise equal to the oracle's (unique)
    _, S_ref, _ = O.tsvd(A, econ=econ)
    off = S.copy()
    for i in range(r):
        off[i, i, :] = 0
    assert np.all(off == 0)
    assert rel(S, S_ref) < TOL_FP32
    d = np.array([S[i, i, 0] for i in range(r)])
    assert np.all(np.diff(d) <= 1e-6 * max(d[0], 1e-30))


@pytest.mark.parametrize("shape", [(1, 1, 1), (8, 5, 1), (5, 8, 2), (16, 16, 3), (40, 24, 4),
                                   (24, 40, 5), (64, 64, 16), (100, 37, 7), (37, 100, 6)])
@pytest.mark.parametrize("econ", [False, True])
def test_tsvd_invariants_and_S(tp, shape, econ):
    _check_tsvd(tp, randn(shape, 31), econ)


def test_tsvd_rank_deficient_small_workload(tp):
    f = {"P": randn((30, 3, 6), 1), "Q": randn((3, 20, 6), 2), "E": np.zeros((30, 20, 6), np.float32)}
    _check_tsvd(tp, low_rank(f), econ=False)


def test_small_workload_all_ops(tp):
    f, X = small_inputs(0)
    P, Q = dev(tp, f["P"]), dev(tp, f["Q"])
    assert rel(host(tp, tp.tprod(P, Q)), O.tprod(f["P"], f["Q"])) < TOL_FP32
    _check_tsvd(tp, X, econ=False)
    dX = dev(tp, X)
    assert abs(float(tp.tnn(dX).item()) - O.tnn(X)) <= TOL_FP32 * O.tnn(X)
    assert abs(float(tp.tsn(dX).item()) - O.tsn(X)) <= TOL_FP32 * O.tsn(X)


# ----------------------------------------------------------------------------- full-size samples
def test_tprod_full_size_sampled(tp):
    """2048x1024x64 times 1024x1024x64: the size the GEMM bench uses, checked on 600
    sampled entries of the literal bcirc product (Eq. 9)."""
    from paper_1806_07247_gb300 import synth
    g = synth.gemm(0)
    C = tp.tprod(dev(tp, g["A"]), dev(tp, g["B"]))
    rng = np.random.default_rng(1)
    idx = np.stack([rng.integers(0, 2048, 600), rng.integers(0, 1024, 600),
                    rng.integers(0, 64, 600)], axis=1)
    got = C[idx[:, 0], idx[:, 1], idx[:, 2]].double().cpu().numpy()
    ref = O.tprod_entries(g["A"], g["B"], idx)
    assert rel(got, ref) < TOL_FP32


def test_prox_batched_full_size_sampled(tp):
    """The full 512-tensor batch in one call, as timed by the bench; 6 tensors checked."""
    items = batched_inputs(512)
    Ys = [dev(tp, X) for _, X in items]
    outs = tp.prox_tnn_batched(Ys, [s.tau for s, _ in items])
    for t in (0, 101, 202, 303, 404, 511):
        s, X = items[t]
        assert rel(host(tp, outs[t]), O.prox_tnn(X, s.tau)) < TOL_FP32, (t, s)
