"""The C ABI without a GPU: the library builds, loads, and exports every entry point that
include/fmg_eig.h declares (no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions() -> list[str]:
    text = open(os.path.join(ROOT, "include", "fmg_eig.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fmg_eig_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1502_04657_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("fmg_eig_create", "fmg_eig_solve", "fmg_eig_solve_dev", "fmg_eig_destroy",
                 "fmg_eig_strerror", "fmg_eig_correction", "fmg_eig_coarse_solve"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_exported_symbol():
    from paper_1502_04657_gb300 import fmg

    assert set(declared_functions()) == set(fmg.exported_symbols())


def test_strerror_without_gpu(lib):
    lib.fmg_eig_strerror.restype = ctypes.c_char_p
    assert lib.fmg_eig_strerror(0) == b"ok"
    assert lib.fmg_eig_strerror(-1) == b"invalid argument"


def test_create_rejects_bad_problem_before_touching_the_gpu(lib):
    from paper_1502_04657_gb300 import fmg

    p = fmg.Problem(levels=0).to_c()
    h = ctypes.c_void_p()
    assert lib.fmg_eig_create(ctypes.byref(p), ctypes.byref(h)) == fmg.FMG_EINVAL
    assert not h.value


def test_binding_constants_match_the_header():
    """Every integer #define of the header that the binding names has the header's value."""
    from paper_1502_04657_gb300 import fmg

    text = open(os.path.join(ROOT, "include", "fmg_eig.h")).read()
    defines = dict(re.findall(r"#define\s+(FMG_\w+)\s+(-?\d+)\b", text))
    shared = [k for k in defines if hasattr(fmg, k)]
    for must in ("FMG_FLAG_NO_AUTOTUNE", "FMG_FLAG_FP32_RHS", "FMG_FLAG_NO_TMA",
                 "FMG_FLAG_STAR_WALKS", "FMG_FLAG_SEPARATE_VCYCLE", "FMG_FLAG_EXPIRE_WAITS",
                 "FMG_SMOOTH_CG"):
        assert must in shared, must
    for k in shared:
        assert getattr(fmg, k) == int(defines[k]), k


def test_create_rejects_unknown_flag_bits_before_touching_the_gpu(lib):
    from paper_1502_04657_gb300 import fmg

    p = fmg.Problem(levels=2, flags=1 << 20).to_c()
    h = ctypes.c_void_p()
    assert lib.fmg_eig_create(ctypes.byref(p), ctypes.byref(h)) == fmg.FMG_EINVAL
    assert not h.value
