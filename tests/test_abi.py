"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/prosper.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "prosper.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(prosper_\w+)\s*\(", src)))


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ["prosper_init", "prosper_estep", "prosper_mstep", "prosper_encode",
                 "prosper_destroy", "prosper_last_error", "prosper_estep_host",
                 "prosper_serve_start", "prosper_serve_submit", "prosper_serve_wait",
                 "prosper_serve_stop"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1908_06843_gb300 import binding
    lib = binding.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in binding.ABI, f"binding does not declare {name}"
    assert lib.prosper_last_error() == b""


def test_init_rejects_bad_arguments_without_gpu_work():
    """Argument checks run before any device call."""
    from paper_1908_06843_gb300 import binding
    lib = binding.load()
    h = ctypes.c_void_p()
    assert lib.prosper_init(ctypes.byref(h), 7, 256, 256, 10, 5, 0, 0) == -1
    assert b"model" in lib.prosper_last_error()
    assert lib.prosper_init(ctypes.byref(h), 0, 256, 256, 11, 5, 0, 0) == -1
    assert lib.prosper_init(ctypes.byref(h), 0, 256, 256, 10, 11, 0, 0) == -1
    assert lib.prosper_init(ctypes.byref(h), 0, 25, 10, 6, 3, 1, 0) == -1   # BF16 needs D % 64
    assert lib.prosper_init(ctypes.byref(h), 2, 64, 32, 8, 4, 0, 0) == -1   # GSC gamma <= 3
    assert lib.prosper_destroy(None) == 0
