"""The C-ABI library loads and exports every entry point include/lhdm.h
declares; argument validation answers without touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lhdm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(lhdm_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2108_05345_gb300 import build
    build.build()
    return C.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lhdm_solve", "lhdm_solve_host", "lhdm_batch_create", "lhdm_batch_run",
                 "lhdm_backward", "lhdm_batch_backward", "lhdm_create", "lhdm_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_host_only_validation(lib):
    from paper_2108_05345_gb300 import lhdm
    L = lhdm.lib()
    p = lhdm.Params()
    assert L.lhdm_default_params(C.byref(p)) == 0
    assert (p.tau1, p.tau2, p.delta, p.k_max) == (0.6, 0.15, 0.9, 32)
    assert L.lhdm_default_params(None) == lhdm.LHDM_ERR_INVALID_ARG
    h = C.c_void_p()
    assert L.lhdm_create(C.byref(h), 0, 5, 0) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_create(C.byref(h), 5, 5, -1) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_create(None, 5, 5, 0) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_solve_batched(None, 0, None, None, None, None, None, None, None, None, None, None) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_backward_batched(None, None, None, None, None, None) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_set_wait_limit(None, 5) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_debug_commit_guard(None, 1) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_debug_fast_math(None, None, 3, None) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_debug_fast_math(None, None, -1, None) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_solve_l1(None, 1, 1, None, 1, None, 1.0, None, None, None, None, None) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_solve(None, 1, 1, None, 1, None, None, None, None, None, None) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_destroy(None) == lhdm.LHDM_ERR_INVALID_ARG
    assert L.lhdm_batch_run(None, None) == lhdm.LHDM_ERR_INVALID_ARG
    assert lhdm.status_string(lhdm.LHDM_ERR_TIMEOUT).startswith("a bounded")
