"""Thin ctypes binding of libtrajam.so (include/trajam.h).

Functions carry the C names and only marshal arguments: numpy arrays are
passed as host memory (AM_HOST), torch CUDA tensors as device memory
(AM_DEVICE).  There is no fallback: if the library is missing or fails to
load, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# TRAJAM_LIBRARY=libtrajam_debug.so selects the bounds-checking debug build
LIB_PATH = os.path.join(HERE, os.environ.get("TRAJAM_LIBRARY", "libtrajam.so"))

AM_OK, AM_ERR_ARG, AM_ERR_CUDA, AM_ERR_BUDGET, AM_ERR_TIMEOUT, AM_ERR_NAN, AM_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
AM_HOST, AM_DEVICE = 0, 1
AM_FP32, AM_TF32, AM_BF16, AM_SPLIT_BF16 = 0, 1, 2, 3
AM_KERNEL_FUSED, AM_KERNEL_PLAIN, AM_KERNEL_LARGE, AM_KERNEL_WARP, AM_KERNEL_AUTO = 0, 1, 2, 3, 4
AM_OPT_KERNEL, AM_OPT_TILE, AM_OPT_DIAG_STALL, AM_OPT_SELECT = 1, 2, 3, 4
AM_SELECT_COST, AM_SELECT_CLEARANCE = 0, 1
AM_GOPT_THREADS, AM_GOPT_GRAPH, AM_GOPT_WARP_SLOTS = 1, 2, 3
AM_PENDING = 1
AM_SRV_BATCHED, AM_SRV_SEQUENTIAL = 0, 1
AM_REQ_GOAL, AM_REQ_RESAMPLE, AM_REQ_SHIFT, AM_REQ_SCALE_LAMBDA = 1, 2, 4, 8
AM_NV, AM_STATE_FLOATS = 11, 110

EXPORTS = ["am_init_problem", "am_set_obstacles", "am_set_boundary", "am_solve_batch",
           "am_get_results", "am_get_best", "am_get_best_async", "am_get_state", "am_set_state", "am_set_history",
           "am_get_history", "am_set_option", "am_set_stream", "am_last_solve_stats",
           "am_solve_batch_noalloc", "am_init_state", "am_resample", "am_shift", "am_scale_multipliers", "am_plan_eval", "am_cem_solve",
           "am_cem_get_best", "am_cem_get_samples", "am_cem_score", "am_group_create", "am_group_solve",
           "am_group_autotune", "am_group_set_option", "am_group_get_option", "am_group_set_active", "am_group_get_best",
           "am_group_stats", "am_group_destroy", "am_server_create", "am_server_add_scene",
           "am_server_start", "am_server_submit", "am_server_poll", "am_server_stats",
           "am_server_destroy", "am_scene_bytes", "am_destroy", "am_last_error"]


class AmProblemDesc(C.Structure):
    _fields_ = [("q", C.c_int), ("T", C.c_double), ("degree", C.c_int), ("m", C.c_int),
                ("r", C.POINTER(C.c_double)), ("r_c", C.c_double),
                ("v_max", C.c_double), ("a_max", C.c_double), ("rho", C.c_double),
                ("rho_psi", C.c_double), ("x_bc", C.c_double * 6), ("y_bc", C.c_double * 6),
                ("psi_bc", C.c_double * 6), ("precision", C.c_int), ("alpha_mode", C.c_int),
                ("psi_dual_sign", C.c_int), ("cs_boundary", C.c_int)]


class AmServerDesc(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("iters", C.c_int), ("mode", C.c_int),
                ("max_batch", C.c_int), ("max_pending", C.c_int), ("lanes", C.c_int)]


class AmRequest(C.Structure):
    _fields_ = [("scene", C.c_int), ("advance", C.c_double),
                ("xo", C.c_void_p), ("yo", C.c_void_p), ("flags", C.c_int),
                ("goal", C.c_double * 9), ("seed", C.c_ulonglong), ("sigma", C.c_float),
                ("lambda_scale", C.c_float)]


class AmResult(C.Structure):
    _fields_ = [("status", C.c_int), ("index", C.c_int), ("cost", C.c_float),
                ("residual", C.c_float), ("coeffs", C.c_float * 33), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double), ("round", C.c_longlong),
                ("batch", C.c_int)]


class AmCemDesc(C.Structure):
    _fields_ = [("samples", C.c_int), ("elites", C.c_int), ("iters", C.c_int),
                ("sigma_xy", C.c_float), ("sigma_psi", C.c_float), ("alpha", C.c_float), ("reg", C.c_float),
                ("w_coll", C.c_float), ("w_bound", C.c_float), ("seed", C.c_ulonglong),
                ("warm", C.c_void_p), ("warm_dt", C.c_double)]


class TrajamError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"trajam error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built; run paper_2109_13030_b300/build.py")
    lib = C.CDLL(LIB_PATH)
    vp, ip, fp, dp = C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_double)
    sig = {
        "am_init_problem": ([C.POINTER(AmProblemDesc), C.POINTER(vp)], ip),
        "am_set_obstacles": ([vp, ip, fp, fp, fp, fp, ip], ip),
        "am_set_boundary": ([vp, dp, dp, dp], ip),
        "am_solve_batch": ([vp, ip, fp, fp, ip, vp, ip], ip),
        "am_get_results": ([vp, fp, fp, fp, fp, ip], ip),
        "am_get_best": ([vp, fp, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_int)], ip),
        "am_get_state": ([vp, fp, ip], ip),
        "am_get_best_async": ([vp, fp, ip, vp], ip),
        "am_set_state": ([vp, ip, fp, ip], ip),
        "am_set_history": ([vp, ip], ip),
        "am_get_history": ([vp, fp, ip], ip),
        "am_set_option": ([vp, ip, ip], ip),
        "am_set_stream": ([vp, vp], ip),
        "am_last_solve_stats": ([vp, C.POINTER(C.c_int)], ip),
        "am_solve_batch_noalloc": ([vp, ip, fp, fp, fp, fp, fp, ip, vp], ip),
        "am_init_state": ([vp, ip, fp, fp, vp, ip], ip),
        "am_resample": ([vp, C.c_ulonglong, C.c_float, vp], ip),
        "am_shift": ([vp, C.c_double, vp], ip),
        "am_scale_multipliers": ([vp, C.c_float, vp], ip),
        "am_cem_solve": ([vp, C.POINTER(AmCemDesc), vp], ip),
        "am_cem_get_best": ([vp, fp, C.POINTER(C.c_float), C.POINTER(C.c_float)], ip),
        "am_cem_get_samples": ([vp, fp, fp, fp, fp], ip),
        "am_cem_score": ([vp, ip, fp, C.c_float, C.c_float, fp, fp], ip),
        "am_plan_eval": ([fp, C.c_double, ip, fp, fp], ip),
        "am_group_create": ([C.POINTER(vp), ip, C.POINTER(vp)], ip),
        "am_group_solve": ([vp, ip, vp], ip),
        "am_group_autotune": ([vp, ip, vp, C.POINTER(C.c_int), C.POINTER(C.c_float)], ip),
        "am_group_set_option": ([vp, ip, ip], ip),
        "am_group_get_option": ([vp, ip, C.POINTER(C.c_int)], ip),
        "am_group_stats": ([vp, C.POINTER(C.c_int), C.POINTER(C.c_int)], ip),
        "am_group_set_active": ([vp, C.POINTER(C.c_int), ip], ip),
        "am_group_get_best": ([vp, fp, ip, vp], ip),
        "am_server_create": ([C.POINTER(AmServerDesc), C.POINTER(vp)], ip),
        "am_server_add_scene": ([vp, vp, ip, fp, ip, C.POINTER(C.c_int)], ip),
        "am_server_start": ([vp], ip),
        "am_server_submit": ([vp, C.POINTER(AmRequest), C.POINTER(C.c_longlong)], ip),
        "am_server_poll": ([vp, C.c_longlong, C.POINTER(AmResult), ip], ip),
        "am_server_stats": ([vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                             C.POINTER(C.c_size_t)], ip),
        "am_server_destroy": ([vp], None),
        "am_scene_bytes": ([ip, ip, ip, ip], C.c_size_t),
        "am_group_destroy": ([vp], None),
        "am_destroy": ([vp], None),
        "am_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def _check(rc):
    if rc != AM_OK:
        raise TrajamError(rc, _lib.am_last_error().decode())
    return rc


def _buf(a, dtype=np.float32):
    """(pointer, mem flag, keep-alive) for a numpy array, a torch tensor or None."""
    if a is None:
        return None, AM_HOST, None
    if isinstance(a, np.ndarray):
        arr = np.ascontiguousarray(a, dtype=dtype)
        return arr.ctypes.data, AM_HOST, arr
    # torch tensor
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if a.is_cuda:
        return a.data_ptr(), AM_DEVICE, a
    return a.data_ptr(), AM_HOST, a


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_desc(pb: dict, precision=AM_FP32, alpha_mode=0, psi_dual_sign=0, cs_boundary=1):
    d = AmProblemDesc()
    d.q, d.T, d.degree, d.m = int(pb["q"]), float(pb["T"]), int(pb.get("degree", 10)), int(pb["m"])
    r = (C.c_double * d.m)(*[float(v) for v in pb["r"]])
    d.r = C.cast(r, C.POINTER(C.c_double))
    d._keep = r
    d.r_c, d.v_max, d.a_max = float(pb["r_c"]), float(pb["v_max"]), float(pb["a_max"])
    d.rho, d.rho_psi = float(pb["rho"]), float(pb["rho_psi"])
    for name in ("x_bc", "y_bc", "psi_bc"):
        arr = getattr(d, name)
        for i, v in enumerate(pb[name]):
            arr[i] = float(v)
    d.precision, d.alpha_mode, d.psi_dual_sign, d.cs_boundary = precision, alpha_mode, psi_dual_sign, cs_boundary
    return d


# ------------------------------------------------------------ C-named calls

def am_init_problem(desc: AmProblemDesc) -> int:
    h = C.c_void_p()
    _check(_lib.am_init_problem(C.byref(desc), C.byref(h)))
    return h.value


def am_set_obstacles(h, n, xo, yo, a, b):
    px, mem, kx = _buf(xo)
    py, _, ky = _buf(yo)
    pa, _, ka = _buf(a)
    pb_, _, kb = _buf(b)
    _check(_lib.am_set_obstacles(h, int(n), px, py, pa, pb_, mem))


def am_set_boundary(h, x_bc, y_bc, psi_bc):
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (x_bc, y_bc, psi_bc)]
    ptrs = [a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs]
    _check(_lib.am_set_boundary(h, *ptrs))


def am_solve_batch(h, B, init, warm_lambda, iters, stream=None):
    pi, mem, ki = _buf(init)
    pw, memw, kw = _buf(warm_lambda)
    if init is not None and warm_lambda is not None and mem != memw:
        raise ValueError("init and warm_lambda must both be host or both be device memory")
    _check(_lib.am_solve_batch(h, int(B), pi, pw, int(iters), _stream_ptr(stream), mem))


def am_get_results(h, res=None, res_psi=None, cost=None, mind=None):
    bufs = [_buf(x) for x in (res, res_psi, cost, mind)]
    mems = {m for (p, m, k) in bufs if p is not None}
    if len(mems) > 1:
        raise ValueError("outputs must all be host or all be device memory")
    mem = mems.pop() if mems else AM_HOST
    _check(_lib.am_get_results(h, *[p for (p, m, k) in bufs], mem))


def am_get_best(h):
    coeffs = np.zeros(33, dtype=np.float32)
    cost, res, idx = C.c_float(), C.c_float(), C.c_int()
    _check(_lib.am_get_best(h, coeffs.ctypes.data, C.byref(cost), C.byref(res), C.byref(idx)))
    return dict(coeffs=coeffs.reshape(3, 11), cost=cost.value, res=res.value, index=idx.value)


def am_get_best_async(h, out, stream=None):
    """Queue the best selection into out (36 floats: index, cost, residual,
    coefficients), host (pinned) or device memory, without waiting."""
    p, mem, k = _buf(out)
    _check(_lib.am_get_best_async(h, p, mem, _stream_ptr(stream)))


def am_get_state(h, out):
    p, mem, k = _buf(out)
    _check(_lib.am_get_state(h, p, mem))


def am_set_state(h, B, state):
    p, mem, k = _buf(state)
    _check(_lib.am_set_state(h, int(B), p, mem))


def am_set_history(h, enable):
    _check(_lib.am_set_history(h, int(bool(enable))))


def am_get_history(h, out):
    p, mem, k = _buf(out)
    _check(_lib.am_get_history(h, p, mem))


def am_set_option(h, option, value):
    _check(_lib.am_set_option(h, int(option), int(value)))


def am_set_stream(h, stream):
    _check(_lib.am_set_stream(h, _stream_ptr(stream)))


def am_last_solve_stats(h) -> int:
    n = C.c_int()
    _check(_lib.am_last_solve_stats(h, C.byref(n)))
    return n.value


def am_solve_batch_noalloc(h, B, state, res, res_psi, cost, mind, iters, stream=None):
    """Allocation-free plain-loop solve on caller-owned device tensors."""
    bufs = [_buf(x) for x in (state, res, res_psi, cost, mind)]
    if any(m != AM_DEVICE for (_, m, _) in bufs):
        raise ValueError("am_solve_batch_noalloc takes device buffers only")
    _check(_lib.am_solve_batch_noalloc(h, int(B), *[p for (p, _, _) in bufs], int(iters),
                                       _stream_ptr(stream)))


def am_init_state(h, B, init, warm_lambda=None, stream=None):
    pi, mem, ki = _buf(init)
    pw, memw, kw = _buf(warm_lambda)
    if warm_lambda is not None and mem != memw:
        raise ValueError("init and warm_lambda must both be host or both be device memory")
    _check(_lib.am_init_state(h, int(B), pi, pw, _stream_ptr(stream), mem))


def am_resample(h, seed, sigma=1.0, stream=None):
    _check(_lib.am_resample(h, int(seed) & (2**64 - 1), float(sigma), _stream_ptr(stream)))


def am_shift(h, dt, stream=None):
    _check(_lib.am_shift(h, float(dt), _stream_ptr(stream)))


CEM_DEFAULTS = dict(samples=8000, elites=800, iters=15, sigma_xy=1.0, sigma_psi=0.3, alpha=0.8, reg=1e-3,
                    w_coll=1e4, w_bound=1e2, seed=0)


def am_cem_solve(h, stream=None, warm=None, warm_dt=0.0, **kw):
    """Cross-entropy method on the handle's problem (see am_cem_solve in the
    header); keyword arguments override CEM_DEFAULTS."""
    o = dict(CEM_DEFAULTS, **kw)
    keep = None
    d = AmCemDesc(int(o["samples"]), int(o["elites"]), int(o["iters"]), float(o["sigma_xy"]),
                  float(o["sigma_psi"]), float(o["alpha"]), float(o["reg"]), float(o["w_coll"]),
                  float(o["w_bound"]), int(o["seed"]) & (2**64 - 1), None, float(warm_dt))
    if warm is not None:
        keep = np.ascontiguousarray(warm, dtype=np.float32).reshape(33)
        d.warm = keep.ctypes.data
    _check(_lib.am_cem_solve(h, C.byref(d), _stream_ptr(stream)))


def am_cem_get_best(h):
    c = np.zeros(33, dtype=np.float32)
    cost, md = C.c_float(), C.c_float()
    _check(_lib.am_cem_get_best(h, c.ctypes.data, C.byref(cost), C.byref(md)))
    return dict(coeffs=c.reshape(3, 11), cost=cost.value, min_dist=md.value)


def am_cem_get_samples(h, n):
    z = np.zeros((n, 15), dtype=np.float32)
    cost = np.zeros(n, dtype=np.float32)
    mu = np.zeros(15, dtype=np.float32)
    sig = np.zeros((15, 15), dtype=np.float32)
    _check(_lib.am_cem_get_samples(h, z.ctypes.data, cost.ctypes.data, mu.ctypes.data, sig.ctypes.data))
    return dict(z=z, cost=cost, mu=mu, sigma=sig)


def am_cem_score(h, coeffs, w_coll=1e4, w_bound=1e2):
    c = np.ascontiguousarray(coeffs, dtype=np.float32).reshape(-1, 33)
    cost = np.zeros(c.shape[0], dtype=np.float32)
    md = np.zeros(c.shape[0], dtype=np.float32)
    _check(_lib.am_cem_score(h, c.shape[0], c.ctypes.data, float(w_coll), float(w_bound), cost.ctypes.data,
                             md.ctypes.data))
    return cost, md


def am_scale_multipliers(h, factor, stream=None):
    _check(_lib.am_scale_multipliers(h, float(factor), _stream_ptr(stream)))


def am_plan_eval(coeffs, T, t):
    """x, x', x'', y, y', y'', psi, psi', psi'' of a plan at the times t: (len(t), 9)."""
    c = np.ascontiguousarray(coeffs, dtype=np.float32).reshape(33)
    tt = np.ascontiguousarray(np.atleast_1d(t), dtype=np.float64)
    out = np.zeros((tt.size, 9))
    _check(_lib.am_plan_eval(c.ctypes.data, float(T), tt.size, tt.ctypes.data, out.ctypes.data))
    return out


def am_group_create(handles) -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    g = C.c_void_p()
    _check(_lib.am_group_create(arr, len(handles), C.byref(g)))
    return g.value


def am_group_solve(g, iters, stream=None):
    _check(_lib.am_group_solve(g, int(iters), _stream_ptr(stream)))


def am_group_autotune(g, iters, stream=None):
    t, ms = C.c_int(), C.c_float()
    _check(_lib.am_group_autotune(g, int(iters), _stream_ptr(stream), C.byref(t), C.byref(ms)))
    return t.value, ms.value


def am_group_set_option(g, option, value):
    _check(_lib.am_group_set_option(g, int(option), int(value)))


def am_group_get_option(g, option) -> int:
    v = C.c_int()
    _check(_lib.am_group_get_option(g, int(option), C.byref(v)))
    return v.value


def am_group_stats(g):
    n, k = C.c_int(), C.c_int()
    _check(_lib.am_group_stats(g, C.byref(n), C.byref(k)))
    return n.value, k.value


def am_group_set_active(g, idx):
    arr = (C.c_int * max(1, len(idx)))(*[int(i) for i in idx])
    _check(_lib.am_group_set_active(g, arr if len(idx) else None, len(idx)))


def am_group_get_best(g, count, stream=None):
    out = np.zeros((count, 36), dtype=np.float32)
    _check(_lib.am_group_get_best(g, out.ctypes.data, AM_HOST, _stream_ptr(stream)))
    return out


def am_group_destroy(g):
    _lib.am_group_destroy(g)


def am_server_create(budget_bytes, iters, mode=AM_SRV_BATCHED, max_batch=0, max_pending=0, lanes=0) -> int:
    d = AmServerDesc(int(budget_bytes), int(iters), int(mode), int(max_batch), int(max_pending), int(lanes))
    s = C.c_void_p()
    _check(_lib.am_server_create(C.byref(d), C.byref(s)))
    return s.value


def am_server_add_scene(s, h, B, init) -> int:
    p, mem, k = _buf(init)
    sc = C.c_int()
    _check(_lib.am_server_add_scene(s, h, int(B), p, mem, C.byref(sc)))
    return sc.value


def am_server_start(s):
    _check(_lib.am_server_start(s))


def am_server_submit(s, scene, advance=0.0, xo=None, yo=None, goal=None, resample_seed=None,
                     sigma=1.0, shift=False, lambda_scale=None) -> int:
    keep = []
    r = AmRequest(int(scene), float(advance), None, None)
    if shift:
        r.flags |= AM_REQ_SHIFT
    if lambda_scale is not None:
        r.flags |= AM_REQ_SCALE_LAMBDA
        r.lambda_scale = float(lambda_scale)
    if goal is not None:
        r.flags |= AM_REQ_GOAL
        for k, v in enumerate(np.asarray(goal, dtype=np.float64).reshape(9)):
            r.goal[k] = float(v)
    if resample_seed is not None:
        r.flags |= AM_REQ_RESAMPLE
        r.seed = int(resample_seed) & (2**64 - 1)
        r.sigma = float(sigma)
    if xo is not None:
        ax = np.ascontiguousarray(xo, dtype=np.float32)
        ay = np.ascontiguousarray(yo, dtype=np.float32)
        keep += [ax, ay]
        r.xo, r.yo = ax.ctypes.data, ay.ctypes.data
    t = C.c_longlong()
    _check(_lib.am_server_submit(s, C.byref(r), C.byref(t)))
    return t.value


def am_server_poll(s, ticket, timeout_ms=0):
    """dict of the result, or None while the request is pending."""
    r = AmResult()
    rc = _lib.am_server_poll(s, C.c_longlong(ticket), C.byref(r), int(timeout_ms))
    if rc == AM_PENDING:
        return None
    _check(rc)
    return dict(status=r.status, index=r.index, cost=r.cost, residual=r.residual,
                coeffs=np.array(r.coeffs, dtype=np.float32).reshape(3, 11), t_submit=r.t_submit,
                t_start=r.t_start, t_done=r.t_done, round=r.round, batch=r.batch)


def am_server_stats(s):
    r, c, b = C.c_longlong(), C.c_longlong(), C.c_size_t()
    _check(_lib.am_server_stats(s, C.byref(r), C.byref(c), C.byref(b)))
    return dict(rounds=r.value, completed=c.value, device_bytes=b.value)


def am_server_destroy(s):
    _lib.am_server_destroy(s)


def am_scene_bytes(q, m, n, B) -> int:
    return int(_lib.am_scene_bytes(int(q), int(m), int(n), int(B)))


def am_destroy(h):
    _lib.am_destroy(h)


def am_last_error() -> str:
    return _lib.am_last_error().decode()


# ------------------------------------------------------------ convenience

class Problem:
    """Owns one handle; methods forward to the C calls above."""

    def __init__(self, pb: dict, precision=AM_FP32, alpha_mode=0, psi_dual_sign=0, cs_boundary=1,
                 kernel=AM_KERNEL_FUSED, tile=0, select=AM_SELECT_COST):
        self.desc = make_desc(pb, precision, alpha_mode, psi_dual_sign, cs_boundary)
        self.h = am_init_problem(self.desc)
        self.q, self.m, self.n = int(pb["q"]), int(pb["m"]), int(pb["n"])
        self.precision = int(precision)
        self.kernel = int(kernel)
        self.B = 0
        self.iters = 0
        am_set_option(self.h, AM_OPT_KERNEL, kernel)
        am_set_option(self.h, AM_OPT_TILE, tile)
        am_set_option(self.h, AM_OPT_SELECT, select)
        if int(pb["n"]) > 0:
            self.set_obstacles(pb["xo"], pb["yo"], pb["ao"], pb["bo"])

    def set_obstacles(self, xo, yo, a, b):
        am_set_obstacles(self.h, len(a), xo, yo, a, b)

    def init_state(self, init, warm_lambda=None, stream=None):
        am_init_state(self.h, int(init.shape[0]), init, warm_lambda, stream)
        self.B = int(init.shape[0])
        return self

    def scale_multipliers(self, factor, stream=None):
        am_scale_multipliers(self.h, factor, stream)
        return self

    def shift(self, dt, stream=None):
        am_shift(self.h, dt, stream)
        return self

    def resample(self, seed, sigma=1.0, stream=None):
        am_resample(self.h, seed, sigma, stream)
        return self

    def set_boundary(self, x_bc, y_bc, psi_bc):
        am_set_boundary(self.h, x_bc, y_bc, psi_bc)
        return self

    def solve(self, init, iters, warm_lambda=None, stream=None, history=False):
        am_set_history(self.h, history)
        B = self.B if init is None else int(init.shape[0])
        am_solve_batch(self.h, B, init, warm_lambda, iters, stream)
        self.B, self.iters = B, iters
        return self

    def results(self):
        out = [np.zeros(self.B, dtype=np.float32) for _ in range(4)]
        am_get_results(self.h, *out)
        return dict(res=out[0], res_psi=out[1], cost=out[2], mind=out[3])

    def state(self):
        s = np.zeros((self.B, AM_STATE_FLOATS), dtype=np.float32)
        am_get_state(self.h, s)
        return s

    def history(self):
        hbuf = np.zeros((self.B, self.iters, 3), dtype=np.float32)
        am_get_history(self.h, hbuf)
        return hbuf

    def best(self):
        return am_get_best(self.h)

    def close(self):
        if self.h:
            am_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Many Problems advanced by one persistent launch per solve."""

    def __init__(self, problems, threads=0, graph=True):
        self.problems = list(problems)   # keeps the handles alive
        self.g = am_group_create([p.h for p in self.problems])
        am_group_set_option(self.g, AM_GOPT_THREADS, threads)
        am_group_set_option(self.g, AM_GOPT_GRAPH, int(bool(graph)))

    def solve(self, iters, stream=None):
        am_group_solve(self.g, iters, stream)
        for p in self.problems:
            p.iters = iters
        return self

    def autotune(self, iters, stream=None, cache=None, sms=0):
        """Time the block sizes (and, with problems on the warp-pair kernels,
        the caps on their trajectory slots per CTA) and keep the fastest;
        returns (threads, ms).  With cache (a JSON path), reuse a choice
        stored for the same shapes, kernel choices, precision, SM count and
        iterations (sms: the device's SM count, part of the key)."""
        if cache is None:
            return am_group_autotune(self.g, iters, stream)
        from . import tune_cache
        k = tune_cache.key([(p.q, p.m, p.n, p.B) for p in self.problems],
                           self.problems[0].precision, sms, iters, [p.kernel for p in self.problems])
        hit = tune_cache.lookup(cache, k)
        if hit is not None:
            am_group_set_option(self.g, AM_GOPT_THREADS, hit[0])
            am_group_set_option(self.g, AM_GOPT_WARP_SLOTS, hit[2])
            return hit[0], hit[1]
        threads, ms = am_group_autotune(self.g, iters, stream)
        tune_cache.store(cache, k, threads, ms, am_group_get_option(self.g, AM_GOPT_WARP_SLOTS))
        return threads, ms

    def warp_slots(self):
        """The cap on the warp-pair group kernels' trajectory slots per CTA
        (0: as many as fit)."""
        return am_group_get_option(self.g, AM_GOPT_WARP_SLOTS)

    def stats(self):
        return am_group_stats(self.g)

    def close(self):
        if self.g:
            am_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Re-planning server over resident scenes (Problems), see am_server_*."""

    def __init__(self, budget_bytes, iters, mode=AM_SRV_BATCHED, max_batch=0, max_pending=0, lanes=0):
        self.s = am_server_create(budget_bytes, iters, mode, max_batch, max_pending, lanes)
        self.scenes = []   # keeps the Problems alive while the server uses them

    def add_scene(self, problem, init):
        k = am_server_add_scene(self.s, problem.h, int(init.shape[0]), init)
        problem.B = int(init.shape[0])
        self.scenes.append(problem)
        return k

    def start(self):
        am_server_start(self.s)
        return self

    def submit(self, scene, advance=0.0, xo=None, yo=None, goal=None, resample_seed=None, sigma=1.0,
               shift=False, lambda_scale=None):
        """goal: 9 values (x, x', x'', y, y', y'', psi, psi', psi'' at t = T);
        resample_seed: re-draw the scene's batch around the new straight line
        with that seed (multipliers kept); shift: re-time the batch by the
        advance (am_shift); lambda_scale: scale the multipliers (am_scale_multipliers)."""
        return am_server_submit(self.s, scene, advance, xo, yo, goal, resample_seed, sigma, shift, lambda_scale)

    def poll(self, ticket, timeout_ms=0):
        return am_server_poll(self.s, ticket, timeout_ms)

    def wait(self, ticket, timeout_s=60.0):
        res = am_server_poll(self.s, ticket, int(timeout_s * 1000))
        if res is None:
            raise TimeoutError(f"request {ticket} not finished within {timeout_s} s")
        return res

    def stats(self):
        return am_server_stats(self.s)

    def close(self):
        if self.s:
            am_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def split_state(s: np.ndarray) -> dict:
    """B x 110 state -> dict(xi1, xi2, lam, lampsi) (float64)."""
    s = np.asarray(s, dtype=np.float64)
    return dict(xi1=s[:, 0:44], xi2=s[:, 44:55], lam=s[:, 55:99], lampsi=s[:, 99:110])
