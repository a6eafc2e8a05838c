"""The C-ABI library builds, loads without a GPU and exports every symbol its
header declares; argument checks that need no device reject bad input."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "trajam.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"AM_API\s+[\w\s\*]*?\b(am_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2109_13030_b300 import build
    return build.build()


def test_header_declares_the_boundary_calls():
    names = declared_symbols()
    for required in ("am_init_problem", "am_set_obstacles", "am_solve_batch", "am_get_best"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(am_\w+)$", out, flags=re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for s in declared_symbols():
        getattr(lib, s)


def test_binding_exposes_the_same_names(lib_path):
    from paper_2109_13030_b300 import trajam
    assert sorted(trajam.EXPORTS) == declared_symbols()
    for s in declared_symbols():
        assert callable(getattr(trajam, s))


def test_null_and_bad_arguments_rejected_without_device(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.am_last_error.restype = ctypes.c_char_p
    assert lib.am_init_problem(None, None) == -1
    assert b"null" in lib.am_last_error()
    assert lib.am_solve_batch(None, 1, None, None, 1, None, 0) == -1
    assert lib.am_get_best(None, None, None, None, None) == -1
    from paper_2109_13030_b300 import trajam, workload
    pb = workload.make_problem("tiny", 0, B=2)
    for field, bad in (("q", 1), ("degree", 7), ("m", 5), ("v_max", -1.0), ("precision", 9)):
        d = trajam.make_desc(pb)
        setattr(d, field, bad)
        h = ctypes.c_void_p()
        assert lib.am_init_problem(ctypes.byref(d), ctypes.byref(h)) == -1, field
        assert h.value is None
