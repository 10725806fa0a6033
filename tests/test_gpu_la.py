"""GPU parity of the per-slice factorisations against the FP64 oracle: the tensor inverse
(Def. 2.4) and the t-QR (Thm. 2.4).

Bars: relative Frobenius error TOL_FP32 = 1e-5 against the oracle on well-conditioned inputs
(condition number about 2 for the inverse, about 5 for tall QR slices), the defining
identities A * B = I and Q * R = A, Q^T * Q = I to the same bound, and exact zeros below the
diagonal of every frontal slice of R.  The columns of a full Q beyond min(n1, n2) are not
unique and are checked through orthogonality only.
"""
import numpy as np
import pytest

from oracle import tproduct as O
from paper_1806_07247_gb300 import synth
from tests.helpers import TOL_FP32, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    import os

    from paper_1806_07247_gb300 import build, tp as _tp
    if not os.path.exists(_tp.LIB_PATH):
        build.build()
    _tp.lib()
    return _tp


def _inv_ref(A):
    n, _, n3 = A.shape
    A64 = A.astype(np.float64)
    return O.tinv(A64) if n * n3 <= 1200 else O.tinv_fourier(A64)


def _tprod_ref(A, B):
    n = A.shape[0] * A.shape[2]
    f = O.tprod if n <= 1200 else O.tprod_fourier
    return f(A.astype(np.float64), B.astype(np.float64))


# ----------------------------------------------------------------------------- tinv
# n <= 128 holds the slice in registers (32-, 64- and 128-wide tiles, full and ragged);
# n = 170 and 200 do not fit one CTA's shared memory and take the global-memory path
@pytest.mark.parametrize("n,n3", [(1, 1), (3, 1), (2, 2), (8, 4), (17, 7), (32, 3), (33, 6),
                                  (64, 16), (65, 2), (100, 5), (127, 3), (128, 6), (160, 3),
                                  (170, 3), (200, 4)])
def test_tinv_parity(tp, n, n3):
    A = synth.shifted_square(n, n3, seed=n + n3)
    B = tp.to_numpy(tp.tinv(tp.to_device(A)))
    assert np.all(np.isfinite(B))
    assert rel(B, _inv_ref(A)) < TOL_FP32
    eye = O.teye(n, n3)
    assert rel(_tprod_ref(A, B), eye) < TOL_FP32
    assert rel(_tprod_ref(B, A), eye) < TOL_FP32


def test_tinv_identity_and_n3_1(tp):
    # every Fourier slice of I is I, so only the two DFTs round
    eye = O.teye(12, 5).astype(np.float32)
    B = tp.to_numpy(tp.tinv(tp.to_device(np.asfortranarray(eye))))
    assert np.max(np.abs(B - eye)) < 1e-6
    A = synth.shifted_square(20, 1, seed=3)
    B = tp.to_numpy(tp.tinv(tp.to_device(A)))
    assert rel(B[:, :, 0], np.linalg.inv(A[:, :, 0].astype(np.float64))) < TOL_FP32


@pytest.mark.parametrize("kind", ["zero_column", "repeated_column", "zero_tensor"])
def test_tinv_singular(tp, kind):
    A = synth.shifted_square(9, 4, seed=5)
    if kind == "zero_column":
        A[:, 3, :] = 0.0
    elif kind == "repeated_column":
        A[:, 5, :] = A[:, 2, :]
    else:
        A[:] = 0.0
    with pytest.raises(tp.TpError) as e:
        tp.tinv(tp.to_device(A))
    assert e.value.status == tp.TP_ERR_SINGULAR
    # asynchronous call: no status, the output is NaN
    B = tp.empty(9, 9, 4, "cuda")
    o = tp.options(sync=False)
    st = tp.lib().tp_tinv(tp._ptr(tp.to_device(A)), tp._ptr(B), 9, 9, 4, tp.ctypes.byref(o), None)
    assert st == tp.TP_OK
    assert np.all(np.isnan(tp.to_numpy(B)))


def test_tinv_shape_and_empty(tp):
    with pytest.raises(tp.TpError) as e:
        tp.tinv(tp.to_device(np.zeros((3, 4, 2), dtype=np.float32, order="F")))
    assert e.value.status == tp.TP_ERR_SHAPE
    for shape in [(0, 0, 3), (4, 4, 0)]:
        out = tp.tinv(tp.to_device(np.zeros(shape, dtype=np.float32, order="F")))
        assert tuple(out.shape) == shape


# ----------------------------------------------------------------------------- tqr
QR_CASES = [
    ("gauss", 1, 1, 1), ("gauss", 5, 3, 1), ("gauss", 1, 4, 3), ("gauss", 6, 1, 2),
    ("gauss", 40, 20, 7), ("gauss", 64, 16, 8), ("gauss", 150, 60, 9),
    ("square", 3, 3, 4), ("square", 33, 33, 2), ("square", 64, 64, 16), ("square", 120, 120, 5),
    ("gauss", 100, 20, 3), ("gauss", 100, 50, 3), ("gauss", 128, 64, 6),  # register tiles
                                                     # 128 x 32 and 128 x 64 (economy Q)
    ("gauss", 240, 100, 4),  # global-memory path (A and Q exceed shared memory)
    ("wide", 12, 30, 6), ("wide", 12, 50, 3), ("wide", 30, 100, 3),  # 32 x 32, 64, 128 tiles
]


def _qr_input(kind, n1, n2, n3, seed):
    if kind == "square":
        return synth.shifted_square(n1, n3, seed)
    if kind == "wide":  # a wide tensor whose leading n1 x n1 block is well conditioned
        A = synth.gaussian(n1, n2, n3, seed) * np.float32(0.05)
        A[:, :n1, :] += synth.shifted_square(n1, n3, seed + 1)
        return np.asfortranarray(A)
    return synth.gaussian(n1, n2, n3, seed)


@pytest.mark.parametrize("econ", [False, True])
@pytest.mark.parametrize("kind,n1,n2,n3", QR_CASES)
def test_tqr_parity(tp, kind, n1, n2, n3, econ):
    A = _qr_input(kind, n1, n2, n3, seed=n1 * 7 + n2 + n3)
    Q, R = tp.tqr(tp.to_device(A), econ=econ)
    Q, R = tp.to_numpy(Q), tp.to_numpy(R)
    m = min(n1, n2)
    assert Q.shape == (n1, m if econ else n1, n3) and R.shape == (m if econ else n1, n2, n3)
    Qo, Ro = O.tqr(A.astype(np.float64))
    assert rel(R, Ro[:R.shape[0]]) < TOL_FP32
    assert rel(Q[:, :m], Qo[:, :m]) < TOL_FP32
    for k in range(n3):  # f-upper triangular, exactly
        assert np.all(np.tril(R[:, :, k], -1) == 0.0)
    assert rel(_tprod_ref(Q, R), A) < TOL_FP32
    QtQ = _tprod_ref(O.tran(Q), Q)
    assert np.max(np.abs(QtQ - O.teye(Q.shape[1], n3))) < 10 * TOL_FP32
    if not econ:
        QQt = _tprod_ref(Q, O.tran(Q))
        assert np.max(np.abs(QQt - O.teye(n1, n3))) < 10 * TOL_FP32


def test_tqr_real_slices_and_empty(tp):
    # n3 = 1 and n3 = 2 have only real Fourier slices: the factors are real matrix QRs
    A = synth.gaussian(7, 4, 1, 11)
    Q, R = tp.tqr(tp.to_device(A), econ=True)
    q, r = np.linalg.qr(A[:, :, 0].astype(np.float64))
    s = np.sign(np.diagonal(r))
    assert rel(tp.to_numpy(R)[:, :, 0], s[:, None] * r) < TOL_FP32
    assert rel(tp.to_numpy(Q)[:, :, 0], q * s) < TOL_FP32
    for shape in [(0, 3, 2), (3, 0, 2), (3, 3, 0)]:
        Q, R = tp.tqr(tp.to_device(np.zeros(shape, dtype=np.float32, order="F")))
        assert Q.numel() == 0 or R.numel() == 0


# ----------------------------------------------------------------------------- limits
@pytest.mark.parametrize("n,n3", [(512, 2), (300, 3), (4, 1024), (33, 1)])
def test_tinv_limits(tp, n, n3):
    """The largest slice (n = TP_MAX_SVD_DIM, 16 rows per lane, global-memory path), a slice
    just past the shared-memory path, the longest tubes (n3 = TP_MAX_N3, 513 slices)."""
    A = synth.shifted_square(n, n3, seed=n + n3)
    B = tp.to_numpy(tp.tinv(tp.to_device(A)))
    assert rel(B, O.tinv_fourier(A.astype(np.float64))) < TOL_FP32


@pytest.mark.parametrize("econ", [False, True])
@pytest.mark.parametrize("n1,n2,n3", [(512, 128, 2), (96, 512, 2), (6, 4, 1024)])
def test_tqr_limits(tp, n1, n2, n3, econ):
    A = synth.gaussian(n1, n2, n3, seed=n1 + n2) if n1 >= 2 * n2 else None
    if A is None:  # wide or small: a well-conditioned leading block
        A = synth.gaussian(n1, n2, n3, seed=n1 + n2) * np.float32(0.05)
        m = min(n1, n2)
        A[:m, :m, :] += synth.shifted_square(m, n3, seed=7)
        A = np.asfortranarray(A)
    Q, R = tp.tqr(tp.to_device(A), econ=econ)
    Q, R = tp.to_numpy(Q), tp.to_numpy(R)
    m = min(n1, n2)
    Qo, Ro = O.tqr(A.astype(np.float64))
    assert rel(R, Ro[:R.shape[0]]) < TOL_FP32
    assert rel(Q[:, :m], Qo[:, :m]) < TOL_FP32
