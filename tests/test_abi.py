"""Host-only checks of the C ABI: the library builds, loads and exports every
entry point that include/lsplit.h declares; argument validation that happens
before any CUDA call returns the documented error codes."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_2103_14897_gb300 import build as B
    B.build()
    import paper_2103_14897_gb300 as P
    return P.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lsplit.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ls_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_binding_exports():
    import paper_2103_14897_gb300 as P
    assert sorted(P.EXPORTS) == declared_functions()


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_invalid_problems_rejected_before_cuda(lib):
    import workloads as W
    from paper_2103_14897_gb300._binding import make_problem_struct
    h = C.c_void_p()
    # d = 3
    st, keep = make_problem_struct(W.config_small_1d())
    st.d = 3
    assert lib.ls_create(C.byref(st), C.byref(h)) == -1
    assert b"d must be" in lib.ls_last_error()
    # 2D slice with non-power-of-two extent
    p = W.twisted_2d(q=6, hmax=1)
    st, keep = make_problem_struct(p)
    assert lib.ls_create(C.byref(st), C.byref(h)) == -1
    # 1D slice whose Bluestein length exceeds 8192
    st, keep = make_problem_struct(W.bilayer_1d(2100, 4, ecut=1.0))
    assert lib.ls_create(C.byref(st), C.byref(h)) == -1
    # complex128 slice whose transform length exceeds 4096 (q = 4097 -> 8192)
    st, keep = make_problem_struct(W.bilayer_1d(2048, 2, ecut=1.0))
    st.dtype = 1
    assert lib.ls_create(C.byref(st), C.byref(h)) == -1
    assert b"complex128" in lib.ls_last_error()
    # bad dtype, bad frac_den, NULL out
    st, keep = make_problem_struct(W.config_small_1d())
    st.dtype = 7
    assert lib.ls_create(C.byref(st), C.byref(h)) == -1
    st.dtype = 0
    st.frac_den = 0
    assert lib.ls_create(C.byref(st), C.byref(h)) == -1
    st.frac_den = 8
    st.mask_mode = 2
    assert lib.ls_create(C.byref(st), C.byref(h)) == -1
    assert b"mask_mode" in lib.ls_last_error()
    st.mask_mode = 0
    assert lib.ls_create(C.byref(st), None) == -1
    assert lib.ls_create(None, C.byref(h)) == -1


def test_null_context_calls(lib):
    p = C.c_int64()
    assert lib.ls_layout(None, C.byref(p), None, None) == -5
    assert lib.ls_step(None, None, 1, 0.1, 1, 0, 0, None) == -5
    assert lib.ls_destroy(None) == 0
    assert lib.ls_index_set(None, None, None) == -5
    assert lib.ls_step_host(None, None, None, 1, 0.1, 1, 0, 0, None) == -5
    assert lib.ls_batch_step_host(None, None, None, 1, 0.1, 1, 0, 0, None) == -5
    assert lib.ls_adjoint(None, None, None, 1, 0.1, 1, 0, 0, None, None, None, None, None) == -5


def test_batch_rejects_projection_before_cuda(lib):
    import workloads as W
    from paper_2103_14897_gb300._binding import make_problem_struct, LsProblem
    st, keep = make_problem_struct(W.config_small_1d(), mask_mode="project")
    arr = (LsProblem * 1)(st)
    h = C.c_void_p()
    assert lib.ls_batch_create(arr, 1, C.byref(h)) == -1
    assert b"LS_MASK_INIT_ONLY" in lib.ls_last_error()
