"""The C-ABI library builds, loads and exports every entry point that
include/rsgpu.h declares; host-only calls work without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsgpu.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1110_4372_gb300 import build
    return C.CDLL(build.build())


def test_header_declares_the_path():
    names = declared()
    for n in ("rs_fof3d", "rs_group_sort", "rs_refine6d", "rs_assign", "rs_find_halos", "rs_create",
              "rs_destroy", "rs_tree_free"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.rs_linking_length.restype = C.c_double
    lib.rs_linking_length.argtypes = [C.c_int64, C.c_double, C.c_double]
    l = lib.rs_linking_length(32768, 10.0, 0.28)
    assert abs(l - 0.0875) < 1e-15
    assert lib.rs_linking_length(0, 10.0, 0.28) == 0.0
    lib.rs_status_string.restype = C.c_char_p
    assert lib.rs_status_string(0) == b"ok"
    assert b"argument" in lib.rs_status_string(1)


def test_create_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    lib.rs_create.argtypes = [C.POINTER(C.c_void_p), C.c_void_p]
    st = lib.rs_create(C.byref(h), None)
    assert st != 0 and not h.value
