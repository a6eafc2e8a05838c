"""ctypes front end of the FP64 CPU oracle (am_oracle.c).

TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the CUDA product path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "am_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
NV = 11

_dp = C.POINTER(C.c_double)


class OrProblem(C.Structure):
    _fields_ = [("q", C.c_int), ("T", C.c_double), ("degree", C.c_int),
                ("m", C.c_int), ("r", _dp), ("r_c", C.c_double),
                ("n", C.c_int), ("xo", _dp), ("yo", _dp), ("ao", _dp), ("bo", _dp),
                ("v_max", C.c_double), ("a_max", C.c_double), ("rho", C.c_double),
                ("rho_psi", C.c_double),
                ("x_bc", C.c_double * 6), ("y_bc", C.c_double * 6), ("psi_bc", C.c_double * 6),
                ("alpha_mode", C.c_int), ("psi_dual_sign", C.c_int), ("cs_boundary", C.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O3, OpenMP, no fast-math)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "am_oracle.h"))):
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_DEFAULT_SOURCE", "-o", LIB, SRC, "-lm"])
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(LIB)
        _lib.or_solve.restype = C.c_int
        _lib.or_dense_solve.restype = C.c_int
        _lib.or_rows_per_side.restype = C.c_int
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


class _Keep:
    """Holds the numpy buffers an OrProblem points into."""


def make_struct(pb: dict, alpha_mode=0, psi_dual_sign=0, cs_boundary=1):
    keep = _Keep()
    keep.r = np.ascontiguousarray(pb["r"], dtype=np.float64)
    n, q = int(pb["n"]), int(pb["q"])
    keep.xo = np.ascontiguousarray(np.reshape(pb["xo"], (n, q)), dtype=np.float64)
    keep.yo = np.ascontiguousarray(np.reshape(pb["yo"], (n, q)), dtype=np.float64)
    keep.ao = np.ascontiguousarray(pb["ao"], dtype=np.float64)
    keep.bo = np.ascontiguousarray(pb["bo"], dtype=np.float64)
    s = OrProblem()
    s.q, s.T, s.degree = q, float(pb["T"]), int(pb.get("degree", 10))
    s.m, s.r, s.r_c = int(pb["m"]), _ptr(keep.r), float(pb["r_c"])
    s.n, s.xo, s.yo, s.ao, s.bo = n, _ptr(keep.xo), _ptr(keep.yo), _ptr(keep.ao), _ptr(keep.bo)
    s.v_max, s.a_max = float(pb["v_max"]), float(pb["a_max"])
    s.rho, s.rho_psi = float(pb["rho"]), float(pb["rho_psi"])
    for name in ("x_bc", "y_bc", "psi_bc"):
        arr = getattr(s, name)
        for i, v in enumerate(pb[name]):
            arr[i] = float(v)
    s.alpha_mode, s.psi_dual_sign, s.cs_boundary = alpha_mode, psi_dual_sign, cs_boundary
    keep.s = s
    return keep


def state_from_init(init: np.ndarray, degree: int = 10):
    """(B, 3, nv) initial (c_x, c_y, c_psi) -> xi1 (B, 4nv), xi2 (B, nv)."""
    init = np.asarray(init, dtype=np.float64)
    B, nv = init.shape[0], degree + 1
    xi1 = np.zeros((B, 4 * nv))
    xi1[:, 0:nv] = init[:, 0]
    xi1[:, 2 * nv:3 * nv] = init[:, 1]
    xi2 = np.ascontiguousarray(init[:, 2])
    return xi1, xi2


def solve(pb: dict, iters: int, init=None, state=None, nthreads: int = 0, hist: bool = False,
          alpha_mode=0, psi_dual_sign=0, cs_boundary=1) -> dict:
    """Run the AM loop.  Give either ``init`` (B, 3, nv) for a cold start or
    ``state`` = dict(xi1, xi2, lam, lampsi) to continue."""
    L = lib()
    nv = int(pb.get("degree", 10)) + 1
    if state is None:
        xi1, xi2 = state_from_init(init if init is not None else pb["init"], nv - 1)
        lam = np.zeros_like(xi1)
        lampsi = np.zeros_like(xi2)
    else:
        xi1 = np.array(state["xi1"], dtype=np.float64)
        xi2 = np.array(state["xi2"], dtype=np.float64)
        lam = np.array(state["lam"], dtype=np.float64)
        lampsi = np.array(state["lampsi"], dtype=np.float64)
    xi1, xi2 = np.ascontiguousarray(xi1), np.ascontiguousarray(xi2)
    lam, lampsi = np.ascontiguousarray(lam), np.ascontiguousarray(lampsi)
    B = xi1.shape[0]
    res, respsi, cost, mind = (np.zeros(B) for _ in range(4))
    h = np.zeros((B, iters, 3)) if hist else None
    keep = make_struct(pb, alpha_mode, psi_dual_sign, cs_boundary)
    rc = L.or_solve(C.byref(keep.s), B, int(iters), _ptr(xi1), _ptr(xi2), _ptr(lam),
                    _ptr(lampsi), _ptr(res), _ptr(respsi), _ptr(cost), _ptr(mind), _ptr(h),
                    int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle or_solve failed: {rc}")
    out = dict(xi1=xi1, xi2=xi2, lam=lam, lampsi=lampsi, res=res, res_psi=respsi,
               cost=cost, mind=mind)
    if hist:
        out["hist"] = h
    return out


def bernstein(degree: int, q: int, T: float):
    L = lib()
    nv = degree + 1
    P, Pd, Pdd = (np.zeros((q, nv)) for _ in range(3))
    L.or_bernstein(degree, q, C.c_double(T), _ptr(P), _ptr(Pd), _ptr(Pdd))
    return P, Pd, Pdd


def dense_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    rc = lib().or_dense_solve(A.shape[0], _ptr(A), _ptr(b), _ptr(x))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return x


def project_obstacle(xt, yt, a, b, alpha_mode=0):
    al, d = C.c_double(), C.c_double()
    lib().or_project_obstacle(C.c_double(xt), C.c_double(yt), C.c_double(a), C.c_double(b),
                              alpha_mode, C.byref(al), C.byref(d))
    return al.value, d.value


def project_bound(ux, uy, umax):
    al, d = C.c_double(), C.c_double()
    lib().or_project_bound(C.c_double(ux), C.c_double(uy), C.c_double(umax),
                           C.byref(al), C.byref(d))
    return al.value, d.value


def build_F(pb: dict) -> np.ndarray:
    keep = make_struct(pb)
    L = lib()
    R1 = L.or_rows_per_side(C.byref(keep.s))
    nv = int(pb.get("degree", 10)) + 1
    F = np.zeros((2 * R1, 4 * nv))
    L.or_build_F(C.byref(keep.s), _ptr(F))
    return F
