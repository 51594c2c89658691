"""The C-ABI library builds, loads and exports every entry point its header declares.

No test here touches a GPU: only argument checks that return before any CUDA call.
"""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sw.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1404_4152_gb300 import build
    import paper_1404_4152_gb300 as sw
    build.build()
    return sw.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "sw_db_load" in names and "sw_search" in names and len(names) >= 8
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/sw.h but not exported"


def test_binding_covers_the_header():
    import paper_1404_4152_gb300 as sw
    for n in declared_functions():
        assert n in sw.SIGNATURES, f"{n} has no Python binding"
        assert callable(getattr(sw, n)), f"paper_1404_4152_gb300.{n} missing"


def test_version_and_error_paths_without_gpu(lib):
    import paper_1404_4152_gb300 as sw
    assert sw.sw_version().startswith("swgb300")
    h = ctypes.c_void_p()
    # NULL out pointer, zero sequences, bad alphabet: rejected before any CUDA call
    assert lib.sw_db_load(None, None, 1, 20, None, None) == 1
    assert "out is NULL" in sw.sw_last_error()
    off = (ctypes.c_uint64 * 2)(0, 0)
    assert lib.sw_db_load(None, off, 0, 20, None, ctypes.byref(h)) == 1
    assert lib.sw_db_load(None, off, 1, 33, None, ctypes.byref(h)) == 1
    assert "alphabet" in sw.sw_last_error()
    assert lib.sw_search(None, None, 0, None, 1, 11, 10, None, None, None, None, None) == 1
    assert "db is NULL" in sw.sw_last_error()
    assert lib.sw_search_device(None, None, 1, None, 1, 11, 1, None, None, None, None) == 1
    assert lib.sw_db_get_info(None, None) == 1
