"""The C ABI library builds, loads without a GPU, and exports every symbol
that include/core_als.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "core_als.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(als_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_18024_gb300 import build
    path = build.build()
    return ctypes.CDLL(str(path))


def test_header_declares_the_calls():
    syms = declared_symbols()
    for name in ("als_create", "als_destroy", "als_half_sweep", "als_select", "als_assemble", "als_solve",
                 "als_eval_sse", "als_fit", "als_fit_host", "als_prepare", "als_status_string"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2509_18024_gb300 import binding
    assert set(declared_symbols()) == set(binding.SIGNATURES)


def test_status_strings_without_gpu(lib):
    lib.als_status_string.restype = ctypes.c_char_p
    assert lib.als_status_string(0) == b"ok"
    assert b"structure" in lib.als_status_string(-2)
    assert lib.als_status_string(12345) == b"unknown status"


def test_option_validation_without_gpu(lib):
    from paper_2509_18024_gb300 import binding as B
    opt = B.als_options()
    lib.als_default_options(ctypes.byref(opt))
    assert opt.n_f == 32 and abs(opt.budget - 0.25) < 1e-12 and opt.pivot_ratio_max == 1e6
    h = ctypes.c_void_p()
    bad = B.als_options.from_buffer_copy(opt)
    bad.n_f = 0
    assert lib.als_create(ctypes.byref(h), ctypes.byref(bad), None) == -1
    bad = B.als_options.from_buffer_copy(opt)
    bad.budget = 1.5
    assert lib.als_create(ctypes.byref(h), ctypes.byref(bad), None) == -1
    bad = B.als_options.from_buffer_copy(opt)
    bad.n_f = 129
    assert lib.als_create(ctypes.byref(h), ctypes.byref(bad), None) == -8
    bad = B.als_options.from_buffer_copy(opt)
    bad.precision = 7
    assert lib.als_create(ctypes.byref(h), ctypes.byref(bad), None) == -1
    assert lib.als_create(None, ctypes.byref(opt), None) == -1
    bad = B.als_options.from_buffer_copy(opt)
    bad.refine_steps = 4
    assert lib.als_create(ctypes.byref(h), ctypes.byref(bad), None) == -1
    bad.refine_steps = -2
    assert lib.als_create(ctypes.byref(h), ctypes.byref(bad), None) == -1
    assert opt.refine_steps == B.ALS_REFINE_AUTO


def test_binding_constants_match_the_header():
    from paper_2509_18024_gb300 import binding as B
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    defines = dict(re.findall(r"#define\s+(ALS_[A-Z0-9_]+)\s+\(?(-?\d+)\)?\s*$", text, flags=re.M))
    assert len(defines) >= 20
    for name, value in defines.items():
        if hasattr(B, name):
            assert getattr(B, name) == int(value), name
    for name in ("ALS_FP32", "ALS_TF32", "ALS_BF16", "ALS_FP32_TC", "ALS_REFINE_AUTO", "ALS_FLAG_FP64"):
        assert int(defines[name]) == getattr(B, name)
