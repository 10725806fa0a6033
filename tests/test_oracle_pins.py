"""Pins for the FP64 oracle: each check ties an oracle function to something other
than itself -- the paper's printed examples, closed forms, library routines,
brute force on tiny tensors, or invariants the paper states -- so that a dropped
term, a wrong sign or index, or a transposed operand fails at least one test.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import tproduct as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def _crand(shape, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def _read_golden(name):
    """Parse the small text fixtures: 'input n1= n2= n3=' + slices, then 'expected ...'."""
    blocks, cur, meta = {}, None, {}
    slices, rows = [], []
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("input") or line.startswith("expected"):
                if cur is not None:
                    if rows:
                        slices.append(rows)
                    blocks[cur] = (meta, slices)
                head, *kv = line.split()
                cur, meta, slices, rows = head, dict(x.split("=") for x in kv), [], []
            elif line.startswith("slice"):
                if rows:
                    slices.append(rows)
                rows = []
            else:
                rows.append([float(v) for v in line.split()])
    if rows:
        slices.append(rows)
    blocks[cur] = (meta, slices)
    return blocks


def _tensor(slices):
    return np.stack([np.array(s) for s in slices], axis=2)


# ----------------------------------------------------------------------------- DFT
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 16, 17, 61, 64])
def test_dft_matrix_unitarity_eq1(n):
    F = O.dft_matrix(n)
    np.testing.assert_allclose(np.conj(F).T @ F, n * np.eye(n), atol=1e-11 * n)
    np.testing.assert_allclose(F @ np.conj(F).T, n * np.eye(n), atol=1e-11 * n)
    # first row and column all ones, entry (1,1) is omega = exp(-2 pi i / n)
    np.testing.assert_allclose(F[0], 1.0)
    np.testing.assert_allclose(F[:, 0], 1.0)
    if n > 1:
        np.testing.assert_allclose(F[1, 1], np.exp(-2j * np.pi / n), atol=1e-15)


@pytest.mark.parametrize("n3", [1, 2, 3, 4, 5, 7, 16, 17, 61])
def test_fft3_matches_library_fft(n3):
    A = _rand((3, 4, n3), n3)
    np.testing.assert_allclose(O.fft3(A), np.fft.fft(A, axis=2), atol=1e-12 * n3)
    Ab = _crand((3, 4, n3), n3 + 100)
    np.testing.assert_allclose(O.ifft3(Ab), np.fft.ifft(Ab, axis=2), atol=1e-12)
    np.testing.assert_allclose(O.ifft3(O.fft3(A)).real, A, atol=1e-12)


def test_fft3_unit_impulses():
    # DFT of a unit impulse at t0 is omega^(k t0) along the tube (Eq. 2).
    n3 = 6
    for t0 in range(n3):
        A = np.zeros((1, 1, n3))
        A[0, 0, t0] = 1.0
        expect = np.exp(-2j * np.pi * np.arange(n3) * t0 / n3)
        np.testing.assert_allclose(O.fft3(A)[0, 0], expect, atol=1e-14)


@pytest.mark.parametrize("n3", [1, 2, 3, 4, 5, 8, 9])
def test_lemma21_conjugate_symmetry_eq4_eq8(n3):
    A = _rand((4, 3, n3), 7 * n3)
    Ab = O.fft3(A)
    assert np.max(np.abs(Ab[:, :, 0].imag)) < 1e-12
    for i in range(1, n3):
        np.testing.assert_allclose(np.conj(Ab[:, :, i]), Ab[:, :, n3 - i], atol=1e-12)
    if n3 % 2 == 0:
        assert np.max(np.abs(Ab[:, :, n3 // 2].imag)) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_circ_diagonalised_eq3(n):
    v = _rand(n, n)
    F = O.dft_matrix(n)
    D = F @ O.circ(v) @ (np.conj(F).T / n)
    np.testing.assert_allclose(D, np.diag(np.fft.fft(v)), atol=1e-12)
    # printed layout: first column v_1..v_n, first row v_1, v_n, ..., v_2
    C = O.circ(v)
    np.testing.assert_allclose(C[:, 0], v)
    np.testing.assert_allclose(C[0], np.concatenate([[v[0]], v[1:][::-1]]))


# ----------------------------------------------------------------------------- bcirc / bdiag
def test_bcirc_golden_eq6():
    g = _read_golden("bcirc_eq6_n3_3.txt")
    A = _tensor(g["input"][1])
    expect = np.array(g["expected"][1][0])
    np.testing.assert_array_equal(O.bcirc(A), expect)


@pytest.mark.parametrize("shape", [(2, 3, 1), (2, 3, 4), (3, 2, 5), (1, 1, 6)])
def test_block_diagonalisation_eq7(shape):
    n1, n2, n3 = shape
    A = _rand(shape, sum(shape))
    F = O.dft_matrix(n3)
    L = np.kron(F, np.eye(n1))
    R = np.kron(np.conj(F).T / n3, np.eye(n2))
    np.testing.assert_allclose(L @ O.bcirc(A) @ R, O.bdiag(O.fft3(A)), atol=1e-11)


def test_unfold_fold_roundtrip():
    A = _rand((3, 4, 5), 1)
    M = O.unfold(A)
    assert M.shape == (15, 4)
    np.testing.assert_array_equal(M[3:6], A[:, :, 1])
    np.testing.assert_array_equal(O.fold(M, 3, 4, 5), A)


# ----------------------------------------------------------------------------- tprod
def _tprod_bruteforce(A, B):
    """Circular convolution of tubes, written with Python loops on tiny inputs."""
    n1, n2, n3 = A.shape
    l = B.shape[1]
    C = np.zeros((n1, l, n3))
    for i, ll, k in itertools.product(range(n1), range(l), range(n3)):
        s = 0.0
        for j in range(n2):
            for t in range(n3):
                s += A[i, j, t] * B[j, ll, (k - t) % n3]
        C[i, ll, k] = s
    return C


@pytest.mark.parametrize("dims", [(2, 3, 2, 1), (2, 3, 4, 3), (3, 2, 2, 4), (1, 1, 1, 5), (2, 2, 3, 6)])
def test_tprod_bruteforce(dims):
    n1, n2, l, n3 = dims
    A = _rand((n1, n2, n3), 11)
    B = _rand((n2, l, n3), 12)
    ref = _tprod_bruteforce(A, B)
    np.testing.assert_allclose(O.tprod(A, B), ref, atol=1e-12)
    np.testing.assert_allclose(O.tprod_fourier(A, B), ref, atol=1e-12)


def test_tprod_n3_1_is_matmul():
    A = _rand((5, 4, 1), 1)
    B = _rand((4, 3, 1), 2)
    np.testing.assert_allclose(O.tprod(A, B)[:, :, 0], A[:, :, 0] @ B[:, :, 0], atol=1e-13)


@pytest.mark.parametrize("n3", [1, 2, 5, 6])
def test_tprod_identity_def23(n3):
    A = _rand((3, 4, n3), n3)
    np.testing.assert_allclose(O.tprod(A, O.teye(4, n3)), A, atol=1e-13)
    np.testing.assert_allclose(O.tprod(O.teye(3, n3), A), A, atol=1e-13)
    Ib = O.fft3(O.teye(3, n3))
    for k in range(n3):
        np.testing.assert_allclose(Ib[:, :, k], np.eye(3), atol=1e-14)


def test_tprod_associative():
    A, B, C = _rand((3, 4, 5), 1), _rand((4, 2, 5), 2), _rand((2, 3, 5), 3)
    np.testing.assert_allclose(O.tprod(O.tprod(A, B), C), O.tprod(A, O.tprod(B, C)), atol=1e-11)


def test_tprod_entries_sampled():
    A, B = _rand((6, 5, 7), 4), _rand((5, 3, 7), 5)
    C = _tprod_bruteforce(A, B)
    idx = np.array([(i, l, k) for i in range(6) for l in range(3) for k in range(7)][::5])
    np.testing.assert_allclose(O.tprod_entries(A, B, idx), C[idx[:, 0], idx[:, 1], idx[:, 2]], atol=1e-12)


def test_tprod_shape_errors():
    with pytest.raises(ValueError):
        O.tprod(np.zeros((2, 3, 4)), np.zeros((4, 2, 4)))
    with pytest.raises(ValueError):
        O.tprod(np.zeros((2, 3, 4)), np.zeros((3, 2, 5)))


# ----------------------------------------------------------------------------- tran
def test_tran_golden_def22():
    g = _read_golden("tran_def22_n3_4.txt")
    A = _tensor(g["input"][1])
    expect = _tensor(g["expected"][1])
    np.testing.assert_array_equal(O.tran(A), expect)


@pytest.mark.parametrize("n3", [1, 2, 3, 4, 7])
def test_tran_reverse_order_law(n3):
    A, B = _rand((3, 4, n3), 1), _rand((4, 2, n3), 2)
    np.testing.assert_allclose(O.tran(O.tprod(A, B)), O.tprod(O.tran(B), O.tran(A)), atol=1e-12)
    np.testing.assert_array_equal(O.tran(O.tran(A)), A)
    # bcirc(A^T) = bcirc(A)^T for a real tensor (Def. 2.2 + Eq. 6)
    np.testing.assert_array_equal(O.bcirc(O.tran(A)), O.bcirc(A).T)


def test_tran_complex_conjugates():
    A = _crand((2, 3, 4), 9)
    T = O.tran(A)
    np.testing.assert_array_equal(T[:, :, 0], np.conj(A[:, :, 0]).T)
    np.testing.assert_array_equal(T[:, :, 1], np.conj(A[:, :, 3]).T)


# ----------------------------------------------------------------------------- t-SVD and norms
@pytest.mark.parametrize("shape", [(4, 3, 1), (4, 3, 4), (3, 5, 5), (4, 4, 6), (5, 2, 7), (1, 3, 4)])
@pytest.mark.parametrize("econ", [False, True])
def test_tsvd_invariants_thm22(shape, econ):
    n1, n2, n3 = shape
    A = _rand(shape, n1 * 100 + n2 * 10 + n3)
    U, S, V = O.tsvd(A, econ=econ)
    r = min(n1, n2)
    assert U.shape == ((n1, r, n3) if econ else (n1, n1, n3))
    assert V.shape == ((n2, r, n3) if econ else (n2, n2, n3))
    # Eq. 12: A = U * S * V^*
    np.testing.assert_allclose(O.tprod(O.tprod(U, S), O.tran(V)), A, atol=1e-11)
    # Def. 2.5: U^* * U = I (and V), with U * U^* = I too in the full shapes
    np.testing.assert_allclose(O.tprod(O.tran(U), U), O.teye(U.shape[1], n3), atol=1e-11)
    np.testing.assert_allclose(O.tprod(O.tran(V), V), O.teye(V.shape[1], n3), atol=1e-11)
    if not econ:
        np.testing.assert_allclose(O.tprod(U, O.tran(U)), O.teye(n1, n3), atol=1e-11)
        np.testing.assert_allclose(O.tprod(V, O.tran(V)), O.teye(n2, n3), atol=1e-11)
    # Def. 2.6: f-diagonal; Eq. 13: S(:,:,1) diagonal decreasing and >= 0
    off = S.copy()
    for i in range(min(S.shape[0], S.shape[1])):
        off[i, i, :] = 0
    assert np.max(np.abs(off)) < 1e-12
    d = np.array([S[i, i, 0] for i in range(r)])
    assert np.all(np.diff(d) <= 1e-12) and np.all(d >= -1e-12)


@pytest.mark.parametrize("shape", [(4, 3, 4), (3, 5, 5), (2, 2, 1)])
def test_tsvd_singular_values_are_bcirc_spectrum(shape):
    # bcirc(A) is unitarily equivalent to bdiag(Abar) (Eq. 7), so the multiset of
    # Fourier-slice singular values equals the singular values of bcirc(A).
    A = _rand(shape, 3)
    sv = np.sort(O.slice_singular_values(A).ravel())
    ref = np.sort(np.linalg.svd(O.bcirc(A), compute_uv=False))
    np.testing.assert_allclose(sv, ref, atol=1e-11)


@pytest.mark.parametrize("shape", [(4, 3, 4), (3, 5, 5), (6, 6, 1), (5, 4, 8)])
def test_tnn_is_scaled_bcirc_nuclear_norm_def29(shape):
    A = _rand(shape, 17)
    n3 = shape[2]
    ref = np.linalg.svd(O.bcirc(A), compute_uv=False).sum() / n3
    assert abs(O.tnn(A) - ref) < 1e-11 * ref
    # Def. 2.9 literally: sum of the diagonal of S(:,:,1) from the t-SVD
    U, S, V = O.tsvd(A)
    assert abs(O.tnn(A) - sum(S[i, i, 0] for i in range(min(shape[:2])))) < 1e-11 * ref


def test_tnn_n3_1_is_matrix_nuclear_norm():
    A = _rand((5, 7, 1), 2)
    assert abs(O.tnn(A) - np.linalg.norm(A[:, :, 0], "nuc")) < 1e-12


@pytest.mark.parametrize("shape", [(4, 3, 4), (3, 5, 5), (6, 6, 1), (5, 4, 8)])
def test_tsn_is_bcirc_spectral_norm_def28(shape):
    A = _rand(shape, 19)
    ref = np.linalg.norm(O.bcirc(A), 2)
    assert abs(O.tsn(A) - ref) < 1e-12 * ref


def test_tubalrank_low_rank_product():
    P, Q = _rand((8, 3, 6), 1), _rand((3, 7, 6), 2)
    X = O.tprod(P, Q)
    assert O.tubalrank(X) == 3
    assert O.tubalrank(_rand((8, 7, 6), 3)) == 7
    s = O.tubal_singular_values(X)
    U, S, V = O.tsvd(X)
    np.testing.assert_allclose(s, [S[i, i, 0] for i in range(7)], atol=1e-11)


# ----------------------------------------------------------------------------- prox
def _matrix_svt(M, tau):
    u, s, vh = np.linalg.svd(M, full_matrices=False)
    return (u * np.maximum(s - tau, 0)) @ vh


@pytest.mark.parametrize("shape,tau", [((4, 3, 4), 0.7), ((3, 5, 5), 1.3), ((4, 4, 6), 0.2),
                                       ((5, 2, 3), 2.5), ((3, 3, 1), 0.9)])
def test_prox_is_svt_of_bcirc_eq19(shape, tau):
    # Eq. 19 with ||X||_* = ||bcirc X||_* / n3 and ||X||_F^2 = ||bcirc X||_F^2 / n3:
    # the minimiser over all matrices, SVT_tau(bcirc(Y)), is block circulant, so
    # its first block column is the prox (matrix SVT is the textbook closed form).
    n1, n2, n3 = shape
    Y = _rand(shape, int(tau * 10) + n3)
    M = _matrix_svt(O.bcirc(Y), tau)
    ref = np.stack([M[k * n1:(k + 1) * n1, 0:n2] for k in range(n3)], axis=2)
    np.testing.assert_allclose(O.prox_tnn(Y, tau), ref, atol=1e-11)


def test_prox_optimality_eq19():
    Y = _rand((5, 4, 6), 23)
    tau = 0.8
    X = O.prox_tnn(Y, tau)

    def obj(Z):
        return tau * O.tnn(Z) + 0.5 * np.sum((Z - Y) ** 2)

    f0 = obj(X)
    g = np.random.default_rng(5)
    for _ in range(20):
        D = g.standard_normal(Y.shape)
        for eps in (1e-3, 1e-2, 1e-1):
            assert obj(X + eps * D) >= f0 - 1e-10


def test_prox_special_cases():
    Y = _rand((4, 5, 6), 29)
    np.testing.assert_allclose(O.prox_tnn(Y, 0.0), Y, atol=1e-12)
    assert np.max(np.abs(O.prox_tnn(Y, O.tsn(Y) * 1.0001))) < 1e-12
    Y1 = _rand((6, 4, 1), 30)
    np.testing.assert_allclose(O.prox_tnn(Y1, 0.5)[:, :, 0], _matrix_svt(Y1[:, :, 0], 0.5), atol=1e-12)


def test_prox_counts_on_gapped_input():
    P, Q = _rand((10, 3, 5), 1), _rand((3, 9, 5), 2)
    Y = O.tprod(P, Q) + 1e-3 * _rand((10, 9, 5), 3)
    c = O.slice_counts(Y, 0.1)
    assert c.shape == (3,) and np.all(c == 3)
    assert O.n_free_slices(16) == 9 and O.n_free_slices(5) == 3 and O.n_free_slices(1) == 1


# ----------------------------------------------------------------------------- tinv / tqr
@pytest.mark.parametrize("n,n3", [(1, 1), (3, 1), (4, 4), (5, 5), (6, 2), (3, 7)])
def test_tinv_def24(n, n3):
    A = _rand((n, n, n3), 10 * n + n3) + 2.0 * O.teye(n, n3)
    B = O.tinv(A)
    np.testing.assert_allclose(O.tprod(A, B), O.teye(n, n3), atol=1e-10)
    np.testing.assert_allclose(O.tprod(B, A), O.teye(n, n3), atol=1e-10)
    np.testing.assert_allclose(O.tinv_fourier(A), B, atol=1e-10)
    if n3 == 1:
        np.testing.assert_allclose(B[:, :, 0], np.linalg.inv(A[:, :, 0]), atol=1e-12)
    np.testing.assert_allclose(O.tinv(O.teye(n, n3)), O.teye(n, n3), atol=1e-13)


def test_tinv_rejects_non_square():
    with pytest.raises(ValueError):
        O.tinv(np.zeros((2, 3, 4)))


@pytest.mark.parametrize("shape", [(4, 3, 1), (4, 3, 4), (3, 5, 5), (4, 4, 6), (6, 2, 7), (1, 3, 2)])
def test_tqr_thm24(shape):
    n1, n2, n3 = shape
    A = _rand(shape, sum(shape) + 3)
    Q, R = O.tqr(A)
    assert Q.shape == (n1, n1, n3) and R.shape == (n1, n2, n3)
    np.testing.assert_allclose(O.tprod(Q, R), A, atol=1e-11)                 # Eq. 22
    np.testing.assert_allclose(O.tprod(O.tran(Q), Q), O.teye(n1, n3), atol=1e-11)
    np.testing.assert_allclose(O.tprod(Q, O.tran(Q)), O.teye(n1, n3), atol=1e-11)
    for k in range(n3):                                                      # f-upper triangular
        assert np.max(np.abs(np.tril(R[:, :, k], -1))) < 1e-12
    # every Fourier slice of R has a real non-negative diagonal (the normalisation)
    Rb = O.fft3(R)
    d = np.stack([np.diagonal(Rb[:, :, k]) for k in range(n3)])
    assert np.max(np.abs(d.imag)) < 1e-10 and np.min(d.real) > -1e-10


def test_tqr_n3_1_is_matrix_qr():
    A = _rand((5, 3, 1), 4)
    Q, R = O.tqr(A)
    q, r = np.linalg.qr(A[:, :, 0], mode="complete")
    s = np.sign(np.diagonal(r))
    np.testing.assert_allclose(R[:3, :, 0], s[:, None] * r[:3], atol=1e-12)
    np.testing.assert_allclose(Q[:, :3, 0], q[:, :3] * s, atol=1e-12)
