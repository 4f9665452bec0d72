"""The C ABI library builds, loads without a GPU and exports every entry point that
include/octtrack.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "octtrack.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(ot_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2605_20565_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = declared_functions()
    for required in ("ot_octree_build", "ot_locate", "ot_interpolate", "ot_spread", "ot_index_train",
                     "ot_batch_create", "ot_batch_run"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_status_strings_without_gpu(lib):
    lib.ot_status_string.restype = ctypes.c_char_p
    assert lib.ot_status_string(0) == b"ok"
    assert b"argument" in lib.ot_status_string(-1)


def test_argument_validation_without_gpu(lib):
    """Null handles and bad enums are rejected on the host before any CUDA call."""
    assert lib.ot_locate(None, None, None, None, ctypes.c_int64(0), 0, None, None, None) == -1
    assert lib.ot_octree_build(None, 0, None, None, None) == -1


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2605_20565_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, fn
                assert "oracle.c" not in txt and "liboracle" not in txt, fn
