"""The C ABI: the library builds for sm_103a, loads, and exports every
function include/mrrr.h declares (CPU only: no compute call needs a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1205_2107_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mrrr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrrr_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_abi():
    names = declared_functions()
    assert names == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_built_for_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


def test_options_defaults(lib):
    o = _lib.Options()
    assert lib.mrrr_options_default(ctypes.byref(o)) == 0
    assert o.gap_tol == 1e-4  # floor; blocks of order m use max(gap_tol, 1/m)
    assert o.classify_rtol == 2.0 ** -20
    assert o.max_depth == 64 and o.threads_per_block % 32 == 0
    assert lib.mrrr_options_default(None) == _lib.ERR_ARG


def test_status_strings(lib):
    for code in range(9):
        s = lib.mrrr_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert lib.mrrr_version() >= 100


def test_null_plan_is_rejected(lib):
    sz = ctypes.c_size_t()
    assert lib.mrrr_workspace_size(None, 1, 10, 10, 10, ctypes.byref(sz)) == _lib.ERR_ARG
    assert lib.mrrr_stein(None, 10, None, None, 1, 10, None, None, 10, None, 0, None) == _lib.ERR_ARG
    assert lib.mrrr_plan_destroy(None) == _lib.ERR_ARG
    assert lib.mrrr_plan_create(None, None) == _lib.ERR_ARG
