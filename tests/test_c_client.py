"""A plain-C client of the library (tests/c_client/am_client.c).

Without a GPU: the client compiles as C11 against include/trajam.h with every
warning an error, links against libtrajam.so, and answers a wrong command
line before any CUDA call.  On the GPU: one solve through the C ABI alone, in
a process with no Python binding and no torch, gives the same state, results
and best trajectory, bit for bit, as the Python binding on the same inputs.
"""
import os
import subprocess

import numpy as np
import pytest

from paper_2109_13030_b300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIBDIR = os.path.join(ROOT, "paper_2109_13030_b300")
SRC = os.path.join(ROOT, "tests", "c_client", "am_client.c")
STATE_FLOATS = 110


def build_client(tmp_path):
    exe = str(tmp_path / "am_client")
    subprocess.run(["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    SRC, "-L", LIBDIR, "-ltrajam", f"-Wl,-rpath,{LIBDIR}", "-o", exe], check=True)
    return exe


def write_input(path, pb, iters, kernel):
    q, m, n, B = int(pb["q"]), int(pb["m"]), int(pb["n"]), int(pb["init"].shape[0])
    with open(path, "wb") as f:
        np.array([q, m, n, B, iters, kernel], dtype="<i4").tofile(f)
        np.array([pb["T"], pb["r_c"], pb["v_max"], pb["a_max"], pb["rho"], pb["rho_psi"]], dtype="<f8").tofile(f)
        np.concatenate([np.asarray(pb[k], dtype=np.float64) for k in ("x_bc", "y_bc", "psi_bc")]).astype("<f8").tofile(f)
        np.asarray(pb["r"], dtype="<f8").tofile(f)
        for k in ("xo", "yo", "ao", "bo"):
            np.asarray(pb[k], dtype="<f4").ravel().tofile(f)
        np.asarray(pb["init"], dtype="<f4").tofile(f)
    return B


def test_client_compiles_as_c_and_rejects_a_bad_command_line(tmp_path):
    exe = build_client(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 1 and "usage" in r.stderr


@pytest.mark.gpu
@pytest.mark.parametrize("kernel", [0, 3])  # AM_KERNEL_FUSED, AM_KERNEL_WARP
def test_c_client_equals_python_binding(tmp_path, kernel):
    from paper_2109_13030_b300 import trajam as T
    exe = build_client(tmp_path)
    pb = W.make_problem("paper", 3, B=64)
    iters = 10
    B = write_input(tmp_path / "in.bin", pb, iters, kernel)
    subprocess.run([exe, str(tmp_path / "in.bin"), str(tmp_path / "out.bin")], check=True)
    out = np.fromfile(tmp_path / "out.bin", dtype="<f4")
    assert out.size == B * STATE_FLOATS + 4 * B + 36
    state = out[:B * STATE_FLOATS].reshape(B, STATE_FLOATS)
    res = out[B * STATE_FLOATS:B * STATE_FLOATS + 4 * B].reshape(4, B)
    best = out[-36:]

    P = T.Problem(pb, kernel=kernel)
    P.solve(pb["init"].astype(np.float32), iters)
    r = P.results()
    b = P.best()
    np.testing.assert_array_equal(state, P.state())
    for i, k in enumerate(("res", "res_psi", "cost", "mind")):
        np.testing.assert_array_equal(res[i], r[k])
    assert int(best[0]) == b["index"] and best[1] == np.float32(b["cost"]) and best[2] == np.float32(b["res"])
    np.testing.assert_array_equal(best[3:], b["coeffs"].ravel())
    P.close()
