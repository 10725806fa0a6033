"""FP64 CPU oracle for the t-product toolbox (Lu, "Tensor-Tensor Product Toolbox").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module: only
`tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference`
legs of `bench.py` may call it.  It shares no code, table or helper with the CUDA
library; the only module both sides use is the seeded input generator
`paper_1806_07247_gb300.synth`, which holds none of the method's arithmetic.

Every function is the plain definition from the paper, in float64 (complex128),
with no blocking, fusion or symmetry trick beyond what the cited passage states:

* the mode-3 DFT is the O(n3^2) sum of Eq. 2 over all n3 frequencies, with the
  DFT matrix of Eq. 1 built from the exact index reduction (k*t) mod n3;
* the tensor inverse (Def. 2.4) is the first block column of bcirc(A)^-1, from Eq. 9 with
  A * B = I; the t-QR (Thm. 2.4, no algorithm given) is read as Algorithm 2's construction
  with a QR of each independent Fourier slice;
* the t-product is Def. 2.1 / Eq. 9 literally, fold(bcirc(A) . unfold(B)); the
  Fourier-domain form of Eq. 10 (all n3 slices, no mirror) is kept for sizes
  where the bcirc matrix does not fit in memory;
* SVDs of the Fourier slices use LAPACK (numpy.linalg.svd) as a library step,
  on all n3 slices;
* tnn, tsn, the tubal rank and the proximal operator follow Def. 2.7-2.9,
  Eq. 14, Eq. 17 and Thm. 2.3 / Algorithm 3.

Tensors are numpy arrays of shape (n1, n2, n3); entry (i, j, k) is A[i, j, k]
(0-based, so the paper's frontal slice A^(k+1) is A[:, :, k]).

Readings of passages where the paper is silent or inconsistent:

* tnn carries the 1/n3 of Def. 2.9 + Eq. 14; Eq. 18 omits it.  The 1/n3 form is
  the one under which Algorithm 3's per-slice threshold tau solves Eq. 19.
* The real Fourier slices (k = 0 and, for even n3, k = n3/2) are decomposed with
  a real SVD, so that U and V of Algorithm 2 come out real (Thm. 2.2 says they
  are real).
* The tubal rank's "nonzero" (Eq. 16) is "greater than tol"; the default tol is
  max(n1, n2) * 2^-23 * S(1,1,1), the matrix-rank convention at FP32 precision.
* Counts of kept singular values use the strict test sigma > tau.

Parity: every function here is pinned by `tests/test_oracle_pins.py` against
closed forms, brute force, library routines or the paper's printed examples.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "dft_matrix", "fft3", "ifft3", "circ", "bdiag", "bcirc", "unfold", "fold",
    "tprod", "tprod_fourier", "tprod_entries", "tran", "teye", "n_free_slices",
    "slice_svd", "tsvd", "tubal_singular_values", "tubalrank", "tnn", "tsn",
    "prox_tnn", "slice_counts", "slice_singular_values", "tinv", "tinv_fourier", "tqr",
]


# --------------------------------------------------------------------------- #
# §2.2  Discrete Fourier transform                                             #
# --------------------------------------------------------------------------- #
def dft_matrix(n: int) -> np.ndarray:
    """F_n of Eq. 1: F[k, t] = w^(k t), w = exp(-2 pi i / n).

    The exponent is reduced exactly, (k*t) mod n, before the angle is formed,
    so every entry is cos/sin of 2*pi*m/n with 0 <= m < n.
    """
    k = np.arange(n).reshape(n, 1)
    t = np.arange(n).reshape(1, n)
    m = (k * t) % n
    ang = -2.0 * np.pi * m.astype(np.float64) / n
    return np.cos(ang) + 1j * np.sin(ang)


def fft3(A: np.ndarray) -> np.ndarray:
    """Abar = fft(A, [], 3): the DFT of Eq. 2 applied to every tube A(i, j, :).

    Abar[i, j, k] = sum_t A[i, j, t] * F[k, t], over all n3 frequencies.
    """
    A = np.asarray(A)
    F = dft_matrix(A.shape[2])
    return np.einsum("ijt,kt->ijk", A.astype(np.complex128), F)


def ifft3(Abar: np.ndarray) -> np.ndarray:
    """A = ifft(Abar, [], 3), using F^-1 = F^* / n (consequence of Eq. 1)."""
    n3 = Abar.shape[2]
    F = dft_matrix(n3)
    return np.einsum("ijk,kt->ijt", np.asarray(Abar, dtype=np.complex128), np.conj(F)) / n3


def circ(v: np.ndarray) -> np.ndarray:
    """circ(v) of §2.2: column c is v cyclically shifted down by c, i.e. entry
    (r, c) is v[(r - c) mod n] (first column v_1..v_n, first row v_1, v_n, ..., v_2)."""
    v = np.asarray(v)
    n = v.shape[0]
    r = np.arange(n).reshape(n, 1)
    c = np.arange(n).reshape(1, n)
    return v[(r - c) % n]


# --------------------------------------------------------------------------- #
# §2.2 / §2.3  bdiag, bcirc, unfold, fold                                      #
# --------------------------------------------------------------------------- #
def bdiag(Abar: np.ndarray) -> np.ndarray:
    """Eq. 5: block-diagonal (n1 n3) x (n2 n3) matrix with Abar^(k) as block k."""
    n1, n2, n3 = Abar.shape
    out = np.zeros((n1 * n3, n2 * n3), dtype=Abar.dtype)
    for k in range(n3):
        out[k * n1:(k + 1) * n1, k * n2:(k + 1) * n2] = Abar[:, :, k]
    return out


def bcirc(A: np.ndarray) -> np.ndarray:
    """Eq. 6: block (r, c) of bcirc(A) is the frontal slice A^((r - c) mod n3)
    (0-based), so block row 0 reads A^(1), A^(n3), ..., A^(2) in the paper's
    1-based names."""
    n1, n2, n3 = A.shape
    out = np.zeros((n1 * n3, n2 * n3), dtype=A.dtype)
    for r in range(n3):
        for c in range(n3):
            out[r * n1:(r + 1) * n1, c * n2:(c + 1) * n2] = A[:, :, (r - c) % n3]
    return out


def unfold(A: np.ndarray) -> np.ndarray:
    """§2.3: stack the frontal slices A^(1), ..., A^(n3) into an (n1 n3) x n2 matrix."""
    n1, n2, n3 = A.shape
    return np.concatenate([A[:, :, k] for k in range(n3)], axis=0)


def fold(M: np.ndarray, n1: int, n2: int, n3: int) -> np.ndarray:
    """§2.3: inverse of unfold."""
    assert M.shape == (n1 * n3, n2)
    out = np.zeros((n1, n2, n3), dtype=M.dtype)
    for k in range(n3):
        out[:, :, k] = M[k * n1:(k + 1) * n1, :]
    return out


# --------------------------------------------------------------------------- #
# §2.3  t-algebra                                                              #
# --------------------------------------------------------------------------- #
def tprod(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Def. 2.1, Eq. 9: A * B = fold(bcirc(A) . unfold(B)), evaluated literally."""
    n1, n2, n3 = A.shape
    n2b, l, n3b = B.shape
    if n2b != n2 or n3b != n3:
        raise ValueError("tprod needs A: n1 x n2 x n3 and B: n2 x l x n3")
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    return fold(bcirc(A) @ unfold(B), n1, l, n3)


def tprod_fourier(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Eq. 10: unfold(Cbar) = bdiag(Abar) . unfold(Bbar), i.e. Cbar^(k) = Abar^(k) Bbar^(k)
    for every one of the n3 slices (no conjugate mirror), then the inverse DFT.

    Used where the bcirc matrix of Eq. 9 is too large to form; the real part is
    returned (the imaginary part is rounding, Lemma 2.1's converse).
    """
    n1, n2, n3 = A.shape
    if B.shape[0] != n2 or B.shape[2] != n3:
        raise ValueError("tprod needs A: n1 x n2 x n3 and B: n2 x l x n3")
    Ab = fft3(np.asarray(A, dtype=np.float64))
    Bb = fft3(np.asarray(B, dtype=np.float64))
    Cb = np.einsum("ijk,jlk->ilk", Ab, Bb)
    return ifft3(Cb).real


def tprod_entries(A: np.ndarray, B: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Selected entries of Eq. 9 without forming bcirc: entry (i, l, k) of
    fold(bcirc(A) unfold(B)) is row i of block row k of bcirc(A), i.e. the row
    [A^((k - c) mod n3)(i, :)]_c, times column l of unfold(B).

    idx: integer array of shape (s, 3) holding (i, l, k) triples (0-based).
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    n3 = A.shape[2]
    out = np.empty(len(idx), dtype=np.float64)
    c = np.arange(n3)
    for s, (i, l, k) in enumerate(np.asarray(idx)):
        row = A[i, :, (k - c) % n3]          # (n3 blocks, n2) -> block c is A^((k-c) mod n3)(i,:)
        col = B[:, l, c].T                   # block c of unfold(B)(:, l) is B^(c)(:, l)
        out[s] = float(np.sum(row * col))
    return out


def tran(A: np.ndarray) -> np.ndarray:
    """Def. 2.2: conjugate-transpose every frontal slice, then reverse the order of
    the transposed slices 2..n3 (0-based: output slice k is slice (n3 - k) mod n3)."""
    n1, n2, n3 = A.shape
    out = np.empty((n2, n1, n3), dtype=A.dtype)
    for k in range(n3):
        out[:, :, k] = np.conj(A[:, :, (n3 - k) % n3]).T
    return out


def teye(n: int, n3: int) -> np.ndarray:
    """Def. 2.3: first frontal slice I_n, the others zero."""
    out = np.zeros((n, n, n3), dtype=np.float64)
    out[:, :, 0] = np.eye(n)
    return out


def n_free_slices(n3: int) -> int:
    """ceil((n3 + 1) / 2), the number of Fourier slices Algorithms 1-3 compute
    directly; the rest are conjugate mirrors (Eq. 8)."""
    return (n3 + 2) // 2


# --------------------------------------------------------------------------- #
# Thm. 2.2 / Algorithm 2  t-SVD, and the singular values it defines            #
# --------------------------------------------------------------------------- #
def _is_real_slice(k: int, n3: int) -> bool:
    """Slice 0 and, for even n3, slice n3/2 are real by Eq. 8 (0-based)."""
    return k == 0 or (n3 % 2 == 0 and k == n3 // 2)


def slice_svd(M: np.ndarray, real: bool, full: bool = True):
    """SVD of one Fourier slice (library step).  A real slice gets a real SVD."""
    if real:
        return np.linalg.svd(np.ascontiguousarray(M.real), full_matrices=full)
    return np.linalg.svd(M, full_matrices=full)


def slice_singular_values(A: np.ndarray) -> np.ndarray:
    """sigma_i(Abar^(k)) for every k < n3, shape (n3, min(n1, n2)), decreasing in i."""
    Ab = fft3(A)
    n3 = A.shape[2]
    return np.stack([np.linalg.svd(Ab[:, :, k], compute_uv=False) for k in range(n3)])


def tsvd(A: np.ndarray, econ: bool = False):
    """Algorithm 2 (Thm. 2.2): A = U * S * V^*.

    Step 1: Abar = fft(A, [], 3).  Step 2: SVD of slices k < ceil((n3+1)/2); the
    remaining slices take conj(U), S, conj(V) of slice n3 - k.  Step 3: inverse DFT
    of all three.  Returns real U (n1 x n1 x n3), S (n1 x n2 x n3), V (n2 x n2 x n3);
    with econ=True, U is n1 x r, S is r x r and V is n2 x r, r = min(n1, n2).
    """
    n1, n2, n3 = A.shape
    r = min(n1, n2)
    Ab = fft3(np.asarray(A, dtype=np.float64))
    h = n_free_slices(n3)
    u_cols = r if econ else n1
    v_cols = r if econ else n2
    Ub = np.zeros((n1, u_cols, n3), dtype=np.complex128)
    Sb = np.zeros((r, r, n3) if econ else (n1, n2, n3), dtype=np.complex128)
    Vb = np.zeros((n2, v_cols, n3), dtype=np.complex128)
    for k in range(h):
        u, s, vh = slice_svd(Ab[:, :, k], _is_real_slice(k, n3), full=not econ)
        Ub[:, :, k] = u
        Vb[:, :, k] = np.conj(vh).T
        for i in range(r):
            Sb[i, i, k] = s[i]
    for k in range(h, n3):
        Ub[:, :, k] = np.conj(Ub[:, :, n3 - k])
        Sb[:, :, k] = Sb[:, :, n3 - k]
        Vb[:, :, k] = np.conj(Vb[:, :, n3 - k])
    return ifft3(Ub).real, ifft3(Sb).real, ifft3(Vb).real


def tubal_singular_values(A: np.ndarray) -> np.ndarray:
    """Eq. 14: S(i, i, 1) = (1/n3) sum_j Sbar(i, i, j), the singular values of A."""
    return slice_singular_values(A).mean(axis=0)


def tubalrank(A: np.ndarray, tol: float | None = None) -> int:
    """Def. 2.7 via Eq. 16: #{i : S(i, i, 1) > tol}."""
    s = tubal_singular_values(A)
    if tol is None:
        tol = max(A.shape[0], A.shape[1]) * 2.0 ** -23 * (s[0] if s.size else 0.0)
    return int(np.sum(s > tol))


def tnn(A: np.ndarray) -> float:
    """Def. 2.9: ||A||_* = sum_i S(i, i, 1) = (1/n3) sum_k sum_i sigma_i(Abar^(k)) (Eq. 14)."""
    return float(np.sum(tubal_singular_values(A)))


def tsn(A: np.ndarray) -> float:
    """Def. 2.8 through Eq. 17: ||A|| = ||bcirc(A)|| = max_k sigma_1(Abar^(k))."""
    return float(np.max(slice_singular_values(A)[:, 0]))


# --------------------------------------------------------------------------- #
# Eq. 19 / Thm. 2.3 / Algorithm 3  proximal operator of TNN                    #
# --------------------------------------------------------------------------- #
def prox_tnn(Y: np.ndarray, tau: float) -> np.ndarray:
    """Thm. 2.3: Prox(Y) = U * S_tau * V^*, S_tau = ifft((Sbar - tau)_+).

    In the Fourier domain this is matrix SVT at tau on each slice, Wbar^(k) =
    U diag((sigma - tau)_+) V^* (Algorithm 3, step 2), done here independently on
    all n3 slices; step 3 is the inverse DFT, whose real part is returned.
    """
    Yb = fft3(np.asarray(Y, dtype=np.float64))
    n1, n2, n3 = Y.shape
    Wb = np.zeros_like(Yb)
    for k in range(n3):
        u, s, vh = slice_svd(Yb[:, :, k], _is_real_slice(k, n3), full=False)
        Wb[:, :, k] = (u * np.maximum(s - tau, 0.0)) @ vh
    return ifft3(Wb).real


def slice_counts(Y: np.ndarray, tau: float) -> np.ndarray:
    """#{i : sigma_i(Ybar^(k)) > tau} for the ceil((n3+1)/2) directly computed
    slices of Algorithm 3 (strict test)."""
    sv = slice_singular_values(np.asarray(Y, dtype=np.float64))
    h = n_free_slices(Y.shape[2])
    return np.sum(sv[:h] > tau, axis=1).astype(np.int64)


# --------------------------------------------------------------------------- #
# Def. 2.4  tensor inverse;  Thm. 2.4  t-QR                                    #
# --------------------------------------------------------------------------- #
def tinv(A: np.ndarray) -> np.ndarray:
    """Def. 2.4: B with A * B = B * A = I.  By Eq. 9, A * B = I means
    bcirc(A) unfold(B) = unfold(I) = [I; 0; ...; 0], so unfold(B) is the first block column
    of bcirc(A)^-1 (the inverse of a block circulant matrix is block circulant)."""
    n, n_, n3 = A.shape
    if n != n_:
        raise ValueError("tinv needs an n x n x n3 tensor")
    Binv = np.linalg.inv(bcirc(np.asarray(A, dtype=np.float64)))
    return fold(Binv[:, :n], n, n, n3)


def tinv_fourier(A: np.ndarray) -> np.ndarray:
    """The same inverse through Eq. 7: the inverse of every Fourier slice (all n3 slices),
    then the inverse DFT (real part)."""
    Ab = fft3(np.asarray(A, dtype=np.float64))
    Bb = np.stack([np.linalg.inv(Ab[:, :, k]) for k in range(A.shape[2])], axis=2)
    return ifft3(Bb).real


def tqr(A: np.ndarray):
    """Thm. 2.4: A = Q * R with Q (n1 x n1 x n3) orthogonal and R (n1 x n2 x n3) f-upper
    triangular.  QR of the ceil((n3+1)/2) independent Fourier slices (real arithmetic on the
    real slices), diag(Rbar^(k)) made real non-negative, conjugate mirrors for the other
    slices, inverse DFT."""
    n1, n2, n3 = A.shape
    Ab = fft3(np.asarray(A, dtype=np.float64))
    h = n_free_slices(n3)
    Qb = np.zeros((n1, n1, n3), dtype=np.complex128)
    Rb = np.zeros((n1, n2, n3), dtype=np.complex128)
    for k in range(h):
        M = Ab[:, :, k].real if _is_real_slice(k, n3) else Ab[:, :, k]
        q, r = np.linalg.qr(M, mode="complete")
        d = np.diagonal(r).copy()
        ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1), 1.0)
        m = min(n1, n2)
        q[:, :m] = q[:, :m] * ph[:m]
        r[:m, :] = np.conj(ph[:m])[:, None] * r[:m, :]
        Qb[:, :, k] = q
        Rb[:, :, k] = r
    for k in range(h, n3):
        Qb[:, :, k] = np.conj(Qb[:, :, n3 - k])
        Rb[:, :, k] = np.conj(Rb[:, :, n3 - k])
    return ifft3(Qb).real, ifft3(Rb).real
