"""The C ABI's error contract, on CPU: every entry point validates its
arguments before any device work, so invalid calls return SOFA_ERR_INVALID_ARG
(or NULL for constructors) with a message from sofa_last_error(), and need
no GPU to do so."""
import ctypes
import os

import numpy as np
import pytest

from paper_2411_17483_gb300 import sofa

INVALID = -1


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(sofa.LIB_PATH):
        from paper_2411_17483_gb300 import _build
        _build.build_library(verbose=False)
    return sofa.load()


def last_error(lib):
    return lib.sofa_last_error().decode()


def host(a):
    return ctypes.c_void_p(a.ctypes.data)


@pytest.mark.parametrize("N,n,l,alphabet,msg", [
    (0, 64, 8, 256, "N must lie"),
    (1 << 31, 64, 8, 256, "N must lie"),
    (100, 3, 1, 256, "series length n"),
    (100, 2048, 8, 256, "series length n"),
    (100, 64, 0, 256, "word length l"),
    (100, 64, 33, 256, "word length l"),
    (100, 8, 8, 256, "word length l"),          # n = 8 has 7 candidate values
    (100, 64, 8, 1, "alphabet"),
    (100, 64, 8, 257, "alphabet"),
])
def test_build_rejects_bad_sizes(lib, N, n, l, alphabet, msg):
    x = np.zeros((4, 8), np.float32)
    assert not lib.sofa_build(host(x), N, n, l, alphabet)
    assert msg in last_error(lib)


def test_build_rejects_null_data_and_bad_options(lib):
    assert not lib.sofa_build(None, 100, 64, 8, 256)
    assert "data is NULL" in last_error(lib)
    x = np.zeros((4, 8), np.float32)
    for field, value, msg in (("precision", 3, "precision"), ("leaf_tiles", 300, "leaf_tiles"),
                              ("binning", 2, "binning"), ("select", -1, "select"),
                              ("sample_ratio", 1.5, "sample_ratio")):
        o = sofa.BuildOpts()
        setattr(o, field, value)
        assert not lib.sofa_build_ex(host(x), 100, 64, 8, 256, ctypes.byref(o), None), field
        assert msg in last_error(lib)
    sel = (ctypes.c_int32 * 8)(*range(7), 999)
    o = sofa.BuildOpts()
    o.user_sel = sel
    o.user_nsel = 8
    assert not lib.sofa_build_ex(host(x), 100, 64, 8, 256, ctypes.byref(o), None)
    assert "user_sel id out of range" in last_error(lib)


def test_calls_on_a_null_handle_are_refused(lib):
    q = np.zeros((2, 64), np.float32)
    i = np.zeros((2, 1), np.int64)
    d = np.zeros((2, 1), np.float32)
    assert lib.sofa_query(None, host(q), 2, 1, host(i), host(d), None) == INVALID
    assert lib.sofa_set_tuning(None, ctypes.byref(sofa.Tuning())) == INVALID
    assert lib.sofa_stats(None, ctypes.byref(sofa.Stats()), 0) == INVALID
    assert lib.sofa_info(None, ctypes.byref(sofa.Info())) == INVALID
    assert lib.sofa_lower_bounds_noalloc(None, host(q), 2, host(d), None) == INVALID
    assert lib.sofa_save(None, b"/nonexistent/x.sofa") == INVALID
    assert lib.sofa_query_multi(None, 1, host(q), None, None, None, 2, host(i), host(d), None, None) == INVALID
    d2 = np.zeros((2, 8), np.float64)
    c = np.zeros(2, np.int32)
    w = np.zeros((2, 8), np.int64)
    assert lib.sofa_query_window(None, host(q), 2, 1, 8, host(w), host(d2), host(c), None) == INVALID
    assert "handle is NULL" in last_error(lib)
    assert lib.sofa_insert(None, host(q), 2, None) == INVALID
    assert "handle is NULL" in last_error(lib)
    lib.sofa_free(None)                         # a no-op


def test_other_entry_points_validate_first(lib):
    x = np.zeros((2, 8), np.float32)
    assert lib.sofa_znorm(None, 2, 8, host(x), None) == INVALID
    assert lib.sofa_znorm(host(x), 2, 0, host(x), None) == INVALID
    assert not lib.sofa_load(None, None)
    assert "path is NULL" in last_error(lib)
    assert not lib.sofa_load(b"/nonexistent/index.sofa", None)
    assert "cannot open" in last_error(lib)
    p = np.zeros(16, np.float32)
    y = np.zeros(4, np.int32)
    loss = ctypes.c_float()
    assert lib.sofa_mlp_grad(0, 8, 4, host(p), host(p), host(y), 4, host(p), ctypes.byref(loss), None) == INVALID
    assert lib.sofa_mlp_grad(4, 8, 1, host(p), host(p), host(y), 4, host(p), ctypes.byref(loss), None) == INVALID
