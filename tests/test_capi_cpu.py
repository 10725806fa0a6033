"""CPU-side checks of the C ABI: the library builds, loads and exports every function
that include/tp.h declares; argument validation that returns before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tp.h")


@pytest.fixture(scope="module")
def L():
    from paper_1806_07247_gb300 import build, tp
    if not os.path.exists(tp.LIB_PATH):
        build.build()
    return tp.lib()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tp_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for need in ["tp_tprod", "tp_tran", "tp_tsvd", "tp_tnn", "tp_tsn", "tp_prox_tnn",
                 "tp_prox_tnn_batched", "tp_tubalrank", "tp_status_string", "tp_options_default"]:
        assert need in names


def test_library_exports_every_declared_symbol(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1806_07247_gb300 import tp
    assert sorted(tp.exported_symbols()) == _declared()


def test_status_strings(L):
    from paper_1806_07247_gb300 import tp
    assert tp.status_string(0) == "TP_OK"
    assert tp.status_string(5) == "TP_ERR_NOT_CONVERGED"
    assert tp.status_string(99) == "TP_ERR_UNKNOWN"


def test_options_default(L):
    from paper_1806_07247_gb300 import tp
    o = tp.Options()
    L.tp_options_default(ctypes.byref(o))
    assert (o.precision, o.econ, o.max_sweeps, o.sync, o.jacobi_tol) == (0, 0, 30, 1, 0.0)
    assert o.sweeps_out is None
    assert o.host_parts == 2
    assert o.counts_out is None and o.jacobi_fp64 == 0


def test_negative_dims_rejected_before_any_cuda_call(L):
    from paper_1806_07247_gb300 import tp
    assert L.tp_tran(None, None, -1, 2, 3, None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_tprod(None, None, None, 2, -2, 2, 2, None, None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_tsvd(None, None, None, None, 2, 2, -1, None, None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_prox_tnn(None, None, -3, 2, 2, 0.5, None, None) == tp.TP_ERR_INVALID_ARG


def test_limits_and_bad_options_rejected(L):
    from paper_1806_07247_gb300 import tp
    assert L.tp_tran(None, None, 2, 2, tp.MAX_N3 + 1, None) == tp.TP_ERR_UNSUPPORTED
    o = tp.options()
    o.precision = 7
    assert L.tp_tprod(None, None, None, 2, 2, 2, 2, ctypes.byref(o), None) == tp.TP_ERR_INVALID_ARG
    o = tp.options()
    o.max_sweeps = -1
    assert L.tp_prox_tnn(None, None, 2, 2, 2, 0.5, ctypes.byref(o), None) == tp.TP_ERR_INVALID_ARG
    # tau must be >= 0 and not NaN; batched count must be >= 0
    assert L.tp_prox_tnn(None, None, 2, 2, 2, -0.5, None, None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_prox_tnn(None, None, 2, 2, 2, float("nan"), None, None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_prox_tnn_batched(None, -1, None, None) == tp.TP_ERR_INVALID_ARG
    for bad in (-1, 3):
        o = tp.options()
        o.host_parts = bad
        assert L.tp_prox_tnn_batched_host(None, 0, ctypes.byref(o), None) == tp.TP_ERR_INVALID_ARG
    # SVD size limit
    d = (tp.TensorDesc * 1)()
    d[0].inp, d[0].out, d[0].n1, d[0].n2, d[0].n3, d[0].tau = 16, 16, tp.MAX_SVD_DIM + 1, 4, 2, 0.1
    assert L.tp_prox_tnn_batched(d, 1, None, None) == tp.TP_ERR_UNSUPPORTED
    # null pointer for a non-empty tensor
    assert L.tp_tran(None, None, 2, 2, 2, None) == tp.TP_ERR_INVALID_ARG


def test_factorisation_argument_checks_before_any_cuda_call(L):
    """tinv (Def. 2.4) needs square frontal slices; both factorisations reject slices above the
    SVD size limit and null pointers of non-empty tensors, and return at once on empty ones."""
    from paper_1806_07247_gb300 import tp
    assert L.tp_tinv(None, None, 3, 4, 2, None, None) == tp.TP_ERR_SHAPE
    big = tp.MAX_SVD_DIM + 1
    assert L.tp_tinv(None, None, big, big, 2, None, None) == tp.TP_ERR_UNSUPPORTED
    assert L.tp_tinv(None, None, 0, 0, 2, None, None) == tp.TP_OK
    assert L.tp_tinv(None, None, 4, 4, 0, None, None) == tp.TP_OK
    assert L.tp_tinv(None, None, 4, 4, 2, None, None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_tinv(None, None, -1, -1, 2, None, None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_tqr(None, None, None, big, 4, 2, None, None) == tp.TP_ERR_UNSUPPORTED
    assert L.tp_tqr(None, None, None, 4, big, 2, None, None) == tp.TP_ERR_UNSUPPORTED
    assert L.tp_tqr(None, None, None, 0, 4, 2, None, None) == tp.TP_OK
    assert L.tp_tqr(None, None, None, 4, 3, 2, None, None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_tqr(None, None, None, 4, -3, 2, None, None) == tp.TP_ERR_INVALID_ARG


def test_jacobi_shape_and_autotune_argument_checks(L):
    from paper_1806_07247_gb300 import tp
    # every field out of range is rejected before the device is touched
    for bad in [(0, 32, 0), (9, 32, 0), (5, 1, 0), (5, 33, 0), (5, 16, 2), (5, 16, -1)]:
        sh = tp.JacobiShape(*bad)
        assert L.tp_jacobi_shape_set(ctypes.byref(sh)) == tp.TP_ERR_INVALID_ARG, bad
    assert L.tp_jacobi_shape_get(None) == tp.TP_ERR_INVALID_ARG
    d = (tp.TensorDesc * 1)()
    d[0].inp, d[0].out, d[0].n1, d[0].n2, d[0].n3, d[0].tau = 16, 16, 8, 8, 4, 0.1
    sh = tp.JacobiShape()
    ms = (ctypes.c_double * 2)()
    assert L.tp_autotune_jacobi(d, 1, 0, ctypes.byref(sh), ms, None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_autotune_jacobi(d, 1, 101, ctypes.byref(sh), ms, None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_autotune_jacobi(d, 1, 2, None, ms, None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_autotune_jacobi(None, -1, 2, ctypes.byref(sh), ms, None) == tp.TP_ERR_INVALID_ARG
    # a batch of empty tensors has nothing to time
    d[0].n3 = 0
    assert L.tp_autotune_jacobi(d, 1, 2, ctypes.byref(sh), ms, None) == tp.TP_ERR_INVALID_ARG
    d[0].n3, d[0].n1 = 4, tp.MAX_SVD_DIM + 1
    assert L.tp_autotune_jacobi(d, 1, 2, ctypes.byref(sh), ms, None) == tp.TP_ERR_UNSUPPORTED


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_compiles_as_plain_c_and_cxx(lang, std, tmp_path):
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if not cc:
        pytest.skip("no host compiler")
    src = tmp_path / ("use." + ("c" if lang == "c" else "cpp"))
    src.write_text('#include "tp.h"\n'
                   "int probe(void) { tp_options o; tp_options_default(&o);\n"
                   "  tp_jacobi_shape s; (void)s; return (int)o.host_parts + (int)TP_OK; }\n")
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        f"-I{os.path.dirname(HEADER)}", str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_noalloc_rejects_options_it_cannot_honour(L):
    # validated before the scratch array or any CUDA call is touched, so this runs on a CPU
    from paper_1806_07247_gb300 import tp
    Y = ctypes.c_void_p(16)  # never dereferenced: every call below returns during validation

    def call(o):
        return L.tp_prox_tnn_noalloc(Y, Y, 4, 4, 4, 0.5, ctypes.byref(o), None)

    cases = []
    o = tp.options(method="learned")
    cases.append(("method", o))
    o = tp.options()
    o.stage_events = 16
    cases.append(("stage_events", o))
    o = tp.options()
    o.slice_flags_out = 16
    cases.append(("slice_flags_out", o))
    o = tp.options()
    o.sketch_width_out = 16
    cases.append(("sketch_width_out", o))
    o = tp.options()
    o.host_parts = 3  # rejected by every entry point's option check
    cases.append(("host_parts", o))
    o = tp.options()
    o.jacobi_fp64 = 2
    cases.append(("jacobi_fp64", o))
    o = tp.options()
    o.method = 7
    cases.append(("method range", o))
    for name, o in cases:
        assert call(o) == tp.TP_ERR_INVALID_ARG, name


def test_bad_new_options_rejected_by_every_entry_point(L):
    from paper_1806_07247_gb300 import tp
    o = tp.options()
    o.jacobi_fp64 = 5
    assert L.tp_prox_tnn(None, None, 2, 2, 2, 0.5, ctypes.byref(o), None) == tp.TP_ERR_INVALID_ARG
    assert L.tp_tnn(None, None, 2, 2, 2, ctypes.byref(o), None) == tp.TP_ERR_INVALID_ARG
