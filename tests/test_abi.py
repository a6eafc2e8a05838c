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


def test_group_and_server_argument_checks_without_device(lib_path):
    from paper_2109_13030_b300 import trajam as T
    L = T._lib
    g = ctypes.c_void_p()
    assert L.am_group_create(None, 1, ctypes.byref(g)) == T.AM_ERR_ARG
    assert L.am_group_solve(None, 10, None) == T.AM_ERR_ARG
    assert L.am_group_set_active(None, None, 0) == T.AM_ERR_ARG
    assert L.am_group_get_best(None, None, 0, None) == T.AM_ERR_ARG
    assert L.am_init_state(None, 1, None, None, None, 0) == T.AM_ERR_ARG
    s = ctypes.c_void_p()
    for kw in (dict(iters=0), dict(mode=7), dict(max_batch=-1)):
        d = T.AmServerDesc(1 << 30, kw.get("iters", 30), kw.get("mode", 0), kw.get("max_batch", 0), 0)
        assert L.am_server_create(ctypes.byref(d), ctypes.byref(s)) == T.AM_ERR_ARG, kw
        assert s.value is None
    assert L.am_server_submit(None, None, None) == T.AM_ERR_ARG
    assert L.am_server_poll(None, 1, None, 0) == T.AM_ERR_ARG


def test_scene_bytes_accounting(lib_path):
    """Admission arithmetic: the constant block, the obstacle tracks and the
    per-trajectory buffers (state 110, results 4, staging 33 + 55 floats)."""
    from paper_2109_13030_b300 import trajam as T
    assert T.am_scene_bytes(1, 3, 10, 1000) == 0
    assert T.am_scene_bytes(100, 5, 10, 1000) == 0
    assert T.am_scene_bytes(100, 3, 10, 0) == 0
    a = T.am_scene_bytes(100, 3, 10, 1000)
    b = T.am_scene_bytes(100, 3, 10, 2000)
    assert b - a == 1000 * (110 + 4 + 33 + 55) * 4
    c = T.am_scene_bytes(100, 3, 11, 1000)
    assert c - a >= (2 * 100 + 2) * 4   # one more obstacle track
    # 64 scenes of the largest mixed shape fit an 8 GB budget many times over
    assert 64 * T.am_scene_bytes(150, 4, 32, 2048) < 8 << 30
