"""The C-ABI library loads without a GPU and exports every symbol the header declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sofa.h")
LIB = os.path.join(ROOT, "paper_2411_17483_gb300", "libsofa.so")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sofa_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__ as g
        from paper_2411_17483_gb300 import _build
        _build.build_library(verbose=False)
        assert g is not None
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared()
    for must in ("sofa_build", "sofa_build_ex", "sofa_query", "sofa_query_multi", "sofa_train_proposal",
                 "sofa_set_seed_mode", "sofa_query_status", "sofa_stats", "sofa_free", "sofa_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2411_17483_gb300 import sofa
    src = open(sofa.__file__).read()
    for n in declared():
        assert f'"{n}"' in src, n


def test_invalid_arguments_rejected_before_device_work(lib):
    lib.sofa_build.restype = ctypes.c_void_p
    lib.sofa_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    lib.sofa_last_error.restype = ctypes.c_char_p
    assert not lib.sofa_build(None, 10, 64, 8, 256)
    assert b"NULL" in lib.sofa_last_error()
    buf = (ctypes.c_float * 64)()
    assert not lib.sofa_build(buf, 1, 64, 8, 1)             # alphabet < 2
    assert b"alphabet" in lib.sofa_last_error()
    assert not lib.sofa_build(buf, 1, 2, 1, 256)            # n < 4
    assert not lib.sofa_build(buf, 1, 8, 9, 256)            # l > candidate values (7 for n = 8)
    lib.sofa_query.restype = ctypes.c_int
    assert lib.sofa_query(None, None, 1, 1, None, None, None) == -1


def test_load_rejects_missing_and_foreign_files(tmp_path):
    """sofa_load fails cleanly (NULL and a message) without touching a GPU for
    files that are missing or not index files."""
    import ctypes
    from paper_2411_17483_gb300 import sofa
    lib = sofa.load()
    assert not lib.sofa_load(str(tmp_path / "absent.sofa").encode(), None)
    assert b"cannot open" in lib.sofa_last_error()
    bad = tmp_path / "foreign.bin"
    bad.write_bytes(b"NOTSOFA!" + b"\0" * 64)
    assert not lib.sofa_load(str(bad).encode(), None)
    assert b"not an index file" in lib.sofa_last_error()
