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
    assert lib.prosper_init(ctypes.byref(h), 0, 256, 256, 17, 5, 0, 0) == -1   # Hprime <= 16
    assert lib.prosper_init(ctypes.byref(h), 0, 256, 256, 16, 5, 0, 0) == -1   # 6,885 > 4,096 states
    assert b"states" in lib.prosper_last_error()
    assert lib.prosper_init(ctypes.byref(h), 0, 256, 256, 16, 9, 0, 0) == -1   # > 4,096 states
    assert lib.prosper_init(ctypes.byref(h), 0, 256, 256, 10, 11, 0, 0) == -1
    assert lib.prosper_init(ctypes.byref(h), 0, 25, 10, 6, 3, 1, 0) == -1   # BF16 needs D % 64
    assert lib.prosper_init(ctypes.byref(h), 2, 64, 32, 8, 4, 0, 0) == -1   # GSC gamma <= 3
    assert lib.prosper_init(ctypes.byref(h), 2, 64, 32, 11, 3, 0, 0) == -1  # GSC Hprime <= 10
    assert lib.prosper_init(ctypes.byref(h), 2, 256, 32, 10, 3, 0, 0) == -1  # GSC shared memory
    assert b"shared memory" in lib.prosper_last_error()
    assert lib.prosper_init(ctypes.byref(h), 1, 100, 20, 16, 4, 0, 0) == -1  # MCA: 2,517 > 1,024
    assert lib.prosper_init(ctypes.byref(h), 3, 256, 64, 8, 3, 1, 0) == -1   # TSC: FP32 only
    assert lib.prosper_init(ctypes.byref(h), 3, 256, 64, 10, 5, 0, 0) == -1  # TSC: 8,064 + .. states
    assert lib.prosper_init(ctypes.byref(h), 4, 256, 64, 8, 3, 0, 0) == -1   # DSC needs its values
    assert b"prosper_init_dsc" in lib.prosper_last_error()
    vals = (ctypes.c_float * 4)(0.5, 2.0, -1.5, 3.0)
    assert lib.prosper_init_dsc(ctypes.byref(h), 256, 64, 8, 3, 4, vals, 0) == -1   # m <= 3
    assert lib.prosper_init_dsc(ctypes.byref(h), 256, 64, 8, 9, 2, vals, 0) == -1   # gamma <= Hprime
    dup = (ctypes.c_float * 2)(1.0, 1.0)
    assert lib.prosper_init_dsc(ctypes.byref(h), 256, 64, 8, 3, 2, dup, 0) == -1
    zero = (ctypes.c_float * 2)(0.0, 1.0)
    assert lib.prosper_init_dsc(ctypes.byref(h), 256, 64, 8, 3, 2, zero, 0) == -1
    assert lib.prosper_destroy(None) == 0
