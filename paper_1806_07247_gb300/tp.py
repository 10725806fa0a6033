"""ctypes binding of libtp (include/tp.h): argument marshalling only.

Every operation runs in the CUDA library; this module only checks tensor types, passes
device pointers, sizes and the current torch CUDA stream, and turns status codes into
exceptions.  If libtp.so is missing the import of any operation raises: there is no
fallback.

Tensors are torch float32 CUDA tensors of logical shape (n1, n2, n3) in column-major
layout, strides (1, n1, n1*n2) -- entry (i, j, k) at offset i + n1*j + n1*n2*k.  Use
`empty`, `to_device` and `to_numpy` to move between that layout and numpy arrays in
Fortran order.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtp.so")

TP_OK, TP_ERR_INVALID_ARG, TP_ERR_SHAPE, TP_ERR_NO_MEMORY, TP_ERR_CUDA, \
    TP_ERR_NOT_CONVERGED, TP_ERR_UNSUPPORTED, TP_ERR_SINGULAR = range(8)
PRECISIONS = {"fp32": 0, "3xtf32": 1, "bf16x3": 2}
MAX_N3 = 1024
MAX_SVD_DIM = 512


class TpError(RuntimeError):
    def __init__(self, status: int, func: str):
        self.status = status
        extra = ""
        if status == TP_ERR_CUDA:
            extra = f" ({lib().tp_last_error_string().decode()})"
        super().__init__(f"{func} failed: {status_string(status)}{extra}")


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("econ", ctypes.c_int32),
                ("max_sweeps", ctypes.c_int32), ("sync", ctypes.c_int32),
                ("jacobi_tol", ctypes.c_double), ("sweeps_out", ctypes.c_void_p),
                ("stage_events", ctypes.c_void_p), ("method", ctypes.c_int32),
                ("slice_flags_out", ctypes.c_void_p), ("sketch_width_out", ctypes.c_void_p),
                ("host_parts", ctypes.c_int32), ("counts_out", ctypes.c_void_p),
                ("jacobi_fp64", ctypes.c_int32)]
STAGE_EVENTS = 6


class JacobiShape(ctypes.Structure):
    _fields_ = [("target_lane_pairs", ctypes.c_int32), ("max_warps", ctypes.c_int32),
                ("split_launches", ctypes.c_int32)]


class TensorDesc(ctypes.Structure):
    _fields_ = [("inp", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n1", ctypes.c_int64),
                ("n2", ctypes.c_int64), ("n3", ctypes.c_int64), ("tau", ctypes.c_double)]


_lib = None

_SIGS = {
    "tp_options_default": (None, [ctypes.POINTER(Options)]),
    "tp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tp_last_error_string": (ctypes.c_char_p, []),
    "tp_tprod": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int64] * 4 +
                 [ctypes.POINTER(Options), ctypes.c_void_p]),
    "tp_tran": (ctypes.c_int, [ctypes.c_void_p] * 2 + [ctypes.c_int64] * 3 + [ctypes.c_void_p]),
    "tp_tsvd": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int64] * 3 +
                [ctypes.POINTER(Options), ctypes.c_void_p]),
    "tp_tnn": (ctypes.c_int, [ctypes.c_void_p] * 2 + [ctypes.c_int64] * 3 +
               [ctypes.POINTER(Options), ctypes.c_void_p]),
    "tp_tsn": (ctypes.c_int, [ctypes.c_void_p] * 2 + [ctypes.c_int64] * 3 +
               [ctypes.POINTER(Options), ctypes.c_void_p]),
    "tp_tubalrank": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int64] * 3 +
                     [ctypes.c_double, ctypes.POINTER(Options), ctypes.c_void_p]),
    "tp_prox_tnn": (ctypes.c_int, [ctypes.c_void_p] * 2 + [ctypes.c_int64] * 3 +
                    [ctypes.c_double, ctypes.POINTER(Options), ctypes.c_void_p]),
    "tp_prox_tnn_batched": (ctypes.c_int, [ctypes.POINTER(TensorDesc), ctypes.c_int64,
                                           ctypes.POINTER(Options), ctypes.c_void_p]),
    "tp_prox_tnn_noalloc": (ctypes.c_int, [ctypes.c_void_p] * 2 + [ctypes.c_int64] * 3 +
                            [ctypes.c_double, ctypes.POINTER(Options), ctypes.c_void_p]),
    "tp_prox_tnn_batched_host": (ctypes.c_int, [ctypes.POINTER(TensorDesc), ctypes.c_int64,
                                                ctypes.POINTER(Options), ctypes.c_void_p]),
    "tp_proposer_train": (ctypes.c_int, [ctypes.POINTER(TensorDesc), ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_double, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "tp_tinv": (ctypes.c_int, [ctypes.c_void_p] * 2 + [ctypes.c_int64] * 3 +
                [ctypes.POINTER(Options), ctypes.c_void_p]),
    "tp_tqr": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int64] * 3 +
               [ctypes.POINTER(Options), ctypes.c_void_p]),
    "tp_prox_plan_create": (ctypes.c_int, [ctypes.POINTER(TensorDesc), ctypes.c_int64,
                                           ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_void_p)]),
    "tp_prox_plan_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "tp_prox_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "tp_jacobi_shape_get": (ctypes.c_int, [ctypes.POINTER(JacobiShape)]),
    "tp_jacobi_shape_set": (ctypes.c_int, [ctypes.POINTER(JacobiShape)]),
    "tp_autotune_jacobi": (ctypes.c_int, [ctypes.POINTER(TensorDesc), ctypes.c_int64, ctypes.c_int32,
                                          ctypes.POINTER(JacobiShape),
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "tp_proposer_get": (ctypes.c_int, [ctypes.c_void_p]),
    "tp_proposer_set": (ctypes.c_int, [ctypes.c_void_p]),
}
METHODS = {"jacobi": 0, "learned": 1}
PROPOSER_FLOATS = 64 * 12 + 64 + 64 * 64 + 64 + 64 + 1 + 2 * 12
NOALLOC_SCRATCH_BYTES = 16 << 20


def lib() -> ctypes.CDLL:
    """Load libtp.so (built in-tree by build.py); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtp.so not found at {LIB_PATH}: run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().tp_status_string(int(status)).decode()


def options(precision: str = "fp32", econ: bool = False, max_sweeps: int = 30, sync: bool = True,
            jacobi_tol: float = 0.0, sweeps_out: torch.Tensor | None = None,
            stage_events=None, method: str = "jacobi",
            slice_flags_out: torch.Tensor | None = None,
            sketch_width_out: torch.Tensor | None = None, host_parts: int = 2,
            counts_out: torch.Tensor | None = None, jacobi_fp64: bool = False) -> Options:
    """tp_options; stage_events is a list of STAGE_EVENTS recorded torch.cuda.Event (tp.h)."""
    o = Options()
    o.method = METHODS[method]
    o.jacobi_fp64 = int(bool(jacobi_fp64))
    for name, t in (("slice_flags_out", slice_flags_out), ("sketch_width_out", sketch_width_out),
                    ("counts_out", counts_out)):
        if t is not None:
            assert t.is_cuda and t.dtype == torch.int32
            setattr(o, name, t.data_ptr())
    o.precision = PRECISIONS[precision]
    o.host_parts = int(host_parts)
    o.econ = int(bool(econ))
    o.max_sweeps = int(max_sweeps)
    o.sync = int(bool(sync))
    o.jacobi_tol = float(jacobi_tol)
    if sweeps_out is not None:
        assert sweeps_out.is_cuda and sweeps_out.dtype == torch.int32
        o.sweeps_out = sweeps_out.data_ptr()
    if stage_events is not None:
        assert len(stage_events) == STAGE_EVENTS
        arr = (ctypes.c_void_p * STAGE_EVENTS)(*[ev.cuda_event for ev in stage_events])
        o._events_keepalive = arr
        o.stage_events = ctypes.cast(arr, ctypes.c_void_p).value
    return o


# ----------------------------------------------------------------------------- layout helpers
def empty(n1: int, n2: int, n3: int, device="cuda") -> torch.Tensor:
    """Uninitialised column-major float32 tensor of logical shape (n1, n2, n3)."""
    return torch.empty((n3, n2, n1), dtype=torch.float32, device=device).permute(2, 1, 0)


def is_colmajor(t: torch.Tensor) -> bool:
    if t.dim() != 3 or t.dtype != torch.float32:
        return False
    if t.numel() == 0:
        return True
    n1, n2, n3 = t.shape
    want = (1, n1, n1 * n2)
    return all(s == w or d <= 1 for s, w, d in zip(t.stride(), want, t.shape))


def colmajor(t: torch.Tensor) -> torch.Tensor:
    """t itself if already column-major float32, else a column-major copy."""
    if is_colmajor(t):
        return t
    return t.to(torch.float32).permute(2, 1, 0).contiguous().permute(2, 1, 0)


def to_device(a: np.ndarray, device="cuda") -> torch.Tensor:
    """numpy (n1, n2, n3) array -> column-major float32 CUDA tensor."""
    a = np.asarray(a, dtype=np.float32)
    if a.ndim == 2:
        a = a[:, :, None]
    host = torch.from_numpy(np.ascontiguousarray(a.transpose(2, 1, 0)))
    return host.to(device).permute(2, 1, 0)


def to_numpy(t: torch.Tensor) -> np.ndarray:
    """Column-major tensor -> numpy float32 (n1, n2, n3) array (Fortran order)."""
    return t.detach().permute(2, 1, 0).contiguous().cpu().numpy().transpose(2, 1, 0)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _check(status: int, func: str):
    if status != TP_OK:
        raise TpError(status, func)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _prep(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dim() != 3:
        raise ValueError(f"{name} must be 3-way (n1, n2, n3)")
    return colmajor(t)


# ----------------------------------------------------------------------------- operations
def tprod(A: torch.Tensor, B: torch.Tensor, out: torch.Tensor | None = None,
          precision: str = "fp32", opts: Options | None = None, stream=None) -> torch.Tensor:
    """C = A * B (Def. 2.1) via Algorithm 1."""
    A, B = _prep(A, "A"), _prep(B, "B")
    n1, n2, n3 = A.shape
    l = B.shape[1]
    if B.shape[0] != n2 or B.shape[2] != n3:
        raise ValueError("tprod needs A: n1 x n2 x n3 and B: n2 x l x n3")
    C = empty(n1, l, n3, A.device) if out is None else out
    assert is_colmajor(C)
    o = opts or options(precision=precision)
    _check(lib().tp_tprod(_ptr(A), _ptr(B), _ptr(C), n1, n2, l, n3, ctypes.byref(o),
                          _stream(stream)), "tp_tprod")
    return C


def tran(A: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Conjugate tensor transpose (Def. 2.2) of a real tensor."""
    A = _prep(A, "A")
    n1, n2, n3 = A.shape
    T = empty(n2, n1, n3, A.device) if out is None else out
    _check(lib().tp_tran(_ptr(A), _ptr(T), n1, n2, n3, _stream(stream)), "tp_tran")
    return T


def tsvd(A: torch.Tensor, econ: bool = False, opts: Options | None = None, stream=None):
    """t-SVD (Thm. 2.2) via Algorithm 2; returns (U, S, V)."""
    A = _prep(A, "A")
    n1, n2, n3 = A.shape
    r = min(n1, n2)
    U = empty(n1, r if econ else n1, n3, A.device)
    S = empty(r if econ else n1, r if econ else n2, n3, A.device)
    V = empty(n2, r if econ else n2, n3, A.device)
    o = opts or options(econ=econ)
    o.econ = int(bool(econ))
    _check(lib().tp_tsvd(_ptr(A), _ptr(U), _ptr(S), _ptr(V), n1, n2, n3, ctypes.byref(o),
                         _stream(stream)), "tp_tsvd")
    return U, S, V


def tinv(A: torch.Tensor, opts: Options | None = None, stream=None) -> torch.Tensor:
    """Tensor inverse (Def. 2.4) of an n x n x n3 tensor; TpError(TP_ERR_SINGULAR) if a
    Fourier slice is singular (synchronous calls)."""
    A = _prep(A, "A")
    n1, n2, n3 = A.shape
    B = empty(n1, n2, n3, A.device)
    o = opts or options()
    _check(lib().tp_tinv(_ptr(A), _ptr(B), n1, n2, n3, ctypes.byref(o), _stream(stream)), "tp_tinv")
    return B


def tqr(A: torch.Tensor, econ: bool = False, opts: Options | None = None, stream=None):
    """t-QR (Thm. 2.4); returns (Q, R)."""
    A = _prep(A, "A")
    n1, n2, n3 = A.shape
    r = min(n1, n2)
    Q = empty(n1, r if econ else n1, n3, A.device)
    R = empty(r if econ else n1, n2, n3, A.device)
    o = opts or options(econ=econ)
    o.econ = int(bool(econ))
    _check(lib().tp_tqr(_ptr(A), _ptr(Q), _ptr(R), n1, n2, n3, ctypes.byref(o), _stream(stream)),
           "tp_tqr")
    return Q, R


def _scalar(fn, name, A, opts, stream, out):
    A = _prep(A, "A")
    n1, n2, n3 = A.shape
    res = torch.empty(1, dtype=torch.float64, device=A.device) if out is None else out
    o = opts or options()
    _check(fn(_ptr(A), _ptr(res), n1, n2, n3, ctypes.byref(o), _stream(stream)), name)
    return res


def tnn(A: torch.Tensor, opts: Options | None = None, stream=None, out=None) -> torch.Tensor:
    """Tensor nuclear norm (Def. 2.9); a 1-element float64 device tensor."""
    return _scalar(lib().tp_tnn, "tp_tnn", A, opts, stream, out)


def tsn(A: torch.Tensor, opts: Options | None = None, stream=None, out=None) -> torch.Tensor:
    """Tensor spectral norm (Def. 2.8); a 1-element float64 device tensor."""
    return _scalar(lib().tp_tsn, "tp_tsn", A, opts, stream, out)


def tubalrank(A: torch.Tensor, tol: float = -1.0, opts: Options | None = None, stream=None):
    """(tubal rank as a 1-element int64 tensor, tensor singular values S(i,i,0) as float64)."""
    A = _prep(A, "A")
    n1, n2, n3 = A.shape
    rank = torch.zeros(1, dtype=torch.int64, device=A.device)
    svals = torch.zeros(max(min(n1, n2), 1), dtype=torch.float64, device=A.device)
    o = opts or options()
    _check(lib().tp_tubalrank(_ptr(A), _ptr(rank), _ptr(svals), n1, n2, n3, float(tol),
                              ctypes.byref(o), _stream(stream)), "tp_tubalrank")
    return rank, svals[:min(n1, n2)]


def prox_tnn(Y: torch.Tensor, tau: float, out: torch.Tensor | None = None,
             opts: Options | None = None, stream=None) -> torch.Tensor:
    """Proximal operator of TNN (Thm. 2.3) via Algorithm 3."""
    Y = _prep(Y, "Y")
    n1, n2, n3 = Y.shape
    X = empty(n1, n2, n3, Y.device) if out is None else out
    o = opts or options()
    _check(lib().tp_prox_tnn(_ptr(Y), _ptr(X), n1, n2, n3, float(tau), ctypes.byref(o),
                             _stream(stream)), "tp_prox_tnn")
    return X


def prox_tnn_noalloc(Y: torch.Tensor, tau: float, out: torch.Tensor | None = None,
                     opts: Options | None = None, stream=None) -> torch.Tensor:
    """prox_tnn through tp_prox_tnn_noalloc: the library allocates nothing during the call
    (its scratch is a fixed 16 MiB device array), for callers that cannot allocate device
    memory while they run. Calls must not overlap on the GPU; `out` must be preallocated by
    the caller if the caller itself cannot allocate."""
    Y = _prep(Y, "Y")
    n1, n2, n3 = Y.shape
    X = empty(n1, n2, n3, Y.device) if out is None else out
    o = opts or options()
    _check(lib().tp_prox_tnn_noalloc(_ptr(Y), _ptr(X), n1, n2, n3, float(tau), ctypes.byref(o),
                                     _stream(stream)), "tp_prox_tnn_noalloc")
    return X


def make_descs(Ys, Xs, taus):
    """ctypes array of tp_tensor_desc for prox_tnn_batched (keeps no tensor alive)."""
    arr = (TensorDesc * len(Ys))()
    for i, (Y, X, tau) in enumerate(zip(Ys, Xs, taus)):
        assert is_colmajor(Y) and is_colmajor(X)
        n1, n2, n3 = Y.shape
        arr[i].inp, arr[i].out = Y.data_ptr(), X.data_ptr()
        arr[i].n1, arr[i].n2, arr[i].n3, arr[i].tau = n1, n2, n3, float(tau)
    return arr


def prox_tnn_batched(Ys, taus, outs=None, opts: Options | None = None, stream=None, descs=None):
    """prox_tnn over many tensors in one batched call; returns the outputs."""
    Ys = [_prep(Y, "Y") for Y in Ys]
    Xs = [empty(*Y.shape, device=Y.device) for Y in Ys] if outs is None else outs
    d = make_descs(Ys, Xs, taus) if descs is None else descs
    o = opts or options()
    _check(lib().tp_prox_tnn_batched(d, len(Ys), ctypes.byref(o), _stream(stream)),
           "tp_prox_tnn_batched")
    return Xs


def pinned_tensors(shapes):
    """(slab, views): one page-locked host buffer holding column-major float32 tensors of the
    given (n1, n2, n3) shapes back to back, and a view of each."""
    total = sum(int(n1) * int(n2) * int(n3) for n1, n2, n3 in shapes)
    slab = torch.empty(max(total, 1), dtype=torch.float32, pin_memory=True)
    views, off = [], 0
    for n1, n2, n3 in shapes:
        n = int(n1) * int(n2) * int(n3)
        views.append(slab[off:off + n].view(n3, n2, n1).permute(2, 1, 0))
        off += n
    return slab, views


def _prep_host(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dim() != 3:
        raise TypeError(f"{name} must be a 3-way host tensor")
    if t.dtype == torch.float32 and is_colmajor(t):
        return t
    return t.to(torch.float32).permute(2, 1, 0).contiguous().permute(2, 1, 0)


def prox_tnn_batched_host(Ys, taus, outs=None, opts: Options | None = None, stream=None,
                          descs=None):
    """prox_tnn over many HOST tensors (page-locked for overlap); the copies in and out and the
    batched prox run inside the call, overlapped by chunks. Returns the host outputs."""
    Ys = [_prep_host(Y, "Y") for Y in Ys]
    if outs is None:
        _, outs = pinned_tensors([tuple(Y.shape) for Y in Ys])
    d = make_descs(Ys, outs, taus) if descs is None else descs
    o = opts or options()
    _check(lib().tp_prox_tnn_batched_host(d, len(Ys), ctypes.byref(o), _stream(stream)),
           "tp_prox_tnn_batched_host")
    return outs


class ProxPlan:
    """A recorded batched prox_tnn (tp_prox_plan_create): run() replays it as one CUDA graph on
    the same tensors (whose contents may change between runs)."""

    def __init__(self, Ys, taus, outs=None, opts: Options | None = None):
        self.Ys = [_prep(Y, "Y") for Y in Ys]
        self.Xs = [empty(*Y.shape, device=Y.device) for Y in self.Ys] if outs is None else outs
        self._descs = make_descs(self.Ys, self.Xs, taus)
        o = opts or options()
        h = ctypes.c_void_p()
        _check(lib().tp_prox_plan_create(self._descs, len(self.Ys), ctypes.byref(o),
                                         ctypes.byref(h)), "tp_prox_plan_create")
        self._h = h

    def run(self, stream=None):
        _check(lib().tp_prox_plan_run(self._h, _stream(stream)), "tp_prox_plan_run")
        return self.Xs

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().tp_prox_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def proposer_train(Ys, taus, steps: int = 300, lr: float = 3e-3, seed: int = 0, stream=None) -> float:
    """Fit the rank proposer of the learned prox method on the slices of these tensors
    (labelled by the plain Jacobi path); returns the final mean squared error."""
    Ys = [_prep(Y, "Y") for Y in Ys]
    d = make_descs(Ys, Ys, taus)
    mse = ctypes.c_double(0.0)
    _check(lib().tp_proposer_train(d, len(Ys), int(steps), float(lr), int(seed), ctypes.byref(mse),
                                   _stream(stream)), "tp_proposer_train")
    return mse.value


def proposer_get() -> np.ndarray:
    out = np.zeros(PROPOSER_FLOATS, dtype=np.float32)
    _check(lib().tp_proposer_get(out.ctypes.data), "tp_proposer_get")
    return out


def proposer_set(params: np.ndarray) -> None:
    params = np.ascontiguousarray(params, dtype=np.float32)
    assert params.size == PROPOSER_FLOATS
    _check(lib().tp_proposer_set(params.ctypes.data), "tp_proposer_set")


def _shape_dict(sh: JacobiShape) -> dict:
    return {"target_lane_pairs": sh.target_lane_pairs, "max_warps": sh.max_warps,
            "split_launches": sh.split_launches}


def jacobi_shape_get() -> dict:
    """The current device's Jacobi CTA shape (tp_jacobi_shape_get)."""
    sh = JacobiShape()
    _check(lib().tp_jacobi_shape_get(ctypes.byref(sh)), "tp_jacobi_shape_get")
    return _shape_dict(sh)


def jacobi_shape_set(shape: dict | None) -> None:
    """Replace the current device's Jacobi CTA shape; None restores the default."""
    if shape is None:
        _check(lib().tp_jacobi_shape_set(None), "tp_jacobi_shape_set")
        return
    sh = JacobiShape(int(shape["target_lane_pairs"]), int(shape["max_warps"]),
                     int(shape["split_launches"]))
    _check(lib().tp_jacobi_shape_set(ctypes.byref(sh)), "tp_jacobi_shape_set")


def autotune_jacobi(Ys, taus, reps: int = 2, stream=None):
    """Time the batched prox's Jacobi launches on these tensors' Fourier slices under each
    candidate CTA shape and keep the fastest (tp_autotune_jacobi). Returns (shape, default_ms,
    chosen_ms)."""
    Ys = [_prep(Y, "Y") for Y in Ys]
    d = make_descs(Ys, Ys, taus)
    sh = JacobiShape()
    ms = (ctypes.c_double * 2)()
    _check(lib().tp_autotune_jacobi(d, len(Ys), int(reps), ctypes.byref(sh), ms, _stream(stream)),
           "tp_autotune_jacobi")
    return _shape_dict(sh), ms[0], ms[1]


def exported_symbols():
    """Names of the C-ABI functions declared in include/tp.h."""
    return sorted(_SIGS)
