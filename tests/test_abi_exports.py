"""The C-ABI library builds, loads and exports every function include/abp.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1609_09833_gb300 import abp, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "abp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(abp_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_core_calls():
    names = _declared()
    for core in ("abp_create_grid", "abp_step", "abp_forces", "abp_bias_readout"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(_declared()) == set(abp.exported_symbols())


def test_version_and_error_string_without_gpu(lib):
    lib.abp_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.abp_version()
    lib.abp_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.abp_last_error(), bytes)


def test_null_arguments_are_rejected_without_touching_the_device(lib):
    # every entry point checks its handles before any CUDA call
    assert lib.abp_sync(None) == -1
    assert lib.abp_step(None, None, 0, None, 0, None, ctypes.c_int64(0)) == -1
    assert lib.abp_create_grid(None, None, None) == -1
