"""Seeded synthetic workloads shaped like the paper's planning problems.

This module only draws inputs: obstacle tracks, robot geometry, boundary
conditions and initial coefficient samples.  It holds none of the optimizer's
arithmetic (no basis matrices, no QP, no projections), so that the CUDA path
and the CPU oracle can both be fed from it without sharing method code.

Every array is rounded to float32 and returned as float64, so the FP32 GPU
path and the FP64 oracle start from bit-identical values.

Workloads (shapes follow the paper's problem statement, Sec. II-B, and its
benchmarks in Sec. IV; the paper's own crowd scenes are not published, so
these synthetic scenes stand in for them):

* ``tiny``      32 trajectories, 50 steps over 5 s, 2 circles (r = +-0.3 m),
                4 static circular obstacles (radius 0.5 m), 100 iterations.
* ``paper``     1000 trajectories, 100 steps over 10 s, 3 circles
                (r in {-0.4, 0, 0.4} m), 10 moving ellipses, 100 iterations.
* ``precision`` the ``paper`` scene at 4096 trajectories.
* ``uneven``    64 independent problems of mixed batch, horizon, obstacle and
                circle counts.
* crowds        (``make_crowd``) the closed-loop benchmarks of Sec. IV: 30
                people walking on straight lines in a 10 m wide band ahead of a
                robot that should follow the x axis at 1 m/s (static crowd,
                same-direction flow up to 0.3 m/s, opposite flow up to 1.0 m/s).
"""
from __future__ import annotations

import numpy as np

NV = 11          # coefficients per polynomial (degree-10 Bernstein)
DEGREE = 10
START = (0.0, 0.0)
GOAL = (8.0, 8.0)


def _f32(a):
    """Round to float32 and hand back float64 (exactly representable)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def straight_line_coeffs(p0: float, p1: float) -> np.ndarray:
    """Control points of a straight line from p0 to p1 that rest at both ends.

    The first three and last three control points coincide with the end
    points; the five interior points are evenly spaced between them.
    """
    s = np.clip((np.arange(NV) - 2) / 6.0, 0.0, 1.0)
    return p0 + (p1 - p0) * s


def smoothness_covariance() -> np.ndarray:
    """STOMP-style covariance for the five interior control points.

    The inverse of R = D2^T D2 restricted to the interior points, where D2 is
    the second-difference operator on the 11 control points, scaled so the
    largest per-point standard deviation is 1 m.
    """
    d2 = np.zeros((NV - 2, NV))
    for k in range(NV - 2):
        d2[k, k:k + 3] = (1.0, -2.0, 1.0)
    r = (d2.T @ d2)[3:8, 3:8]
    cov = np.linalg.inv(r)
    return cov / np.max(np.diag(cov))


def _time_grid(q: int, T: float) -> np.ndarray:
    return np.linspace(0.0, T, q)


def _boundary():
    x_bc = np.array([START[0], 0, 0, GOAL[0], 0, 0], dtype=np.float64)
    y_bc = np.array([START[1], 0, 0, GOAL[1], 0, 0], dtype=np.float64)
    psi_bc = np.zeros(6)
    return x_bc, y_bc, psi_bc


def _init_gaussian(rng, B: int, sigma_iid: float | None) -> np.ndarray:
    """Initial (c_x, c_y, c_psi) samples, shape (B, 3, 11)."""
    init = np.zeros((B, 3, NV))
    init[:, 0, :] = straight_line_coeffs(START[0], GOAL[0])
    init[:, 1, :] = straight_line_coeffs(START[1], GOAL[1])
    if sigma_iid is not None:
        init[:, 0, 3:8] += rng.normal(0.0, sigma_iid, size=(B, 5))
        init[:, 1, 3:8] += rng.normal(0.0, sigma_iid, size=(B, 5))
    else:
        L = np.linalg.cholesky(smoothness_covariance())
        init[:, 0, 3:8] += rng.standard_normal((B, 5)) @ L.T
        init[:, 1, 3:8] += rng.standard_normal((B, 5)) @ L.T
    return _f32(init)


def _moving_ellipses(rng, n: int, q: int, T: float):
    """n axis-aligned ellipses with constant velocities.

    Semi-axes uniform in [0.4, 0.8] m, centres uniform in [1, 9]^2 m,
    velocities uniform in [-1, 1]^2 m/s.  A draw whose centre starts within
    1.5 m of the start or ends within 1.5 m of the goal is redrawn.
    """
    t = _time_grid(q, T)
    xo = np.zeros((n, q))
    yo = np.zeros((n, q))
    ao = np.zeros(n)
    bo = np.zeros(n)
    j = 0
    while j < n:
        a, b = rng.uniform(0.4, 0.8, size=2)
        cx, cy = rng.uniform(1.0, 9.0, size=2)
        vx, vy = rng.uniform(-1.0, 1.0, size=2)
        ex, ey = cx + vx * T, cy + vy * T
        if np.hypot(cx - START[0], cy - START[1]) < 1.5:
            continue
        if np.hypot(ex - GOAL[0], ey - GOAL[1]) < 1.5:
            continue
        xo[j] = cx + vx * t
        yo[j] = cy + vy * t
        ao[j], bo[j] = a, b
        j += 1
    return _f32(xo), _f32(yo), _f32(ao), _f32(bo)


def _static_circles(rng, n: int, q: int, radius: float):
    xo = np.zeros((n, q))
    yo = np.zeros((n, q))
    j = 0
    while j < n:
        cx, cy = rng.uniform(0.0, 10.0, size=2)
        if np.hypot(cx - START[0], cy - START[1]) < 1.5:
            continue
        if np.hypot(cx - GOAL[0], cy - GOAL[1]) < 1.5:
            continue
        xo[j] = cx
        yo[j] = cy
        j += 1
    return _f32(xo), _f32(yo), _f32(np.full(n, radius)), _f32(np.full(n, radius))


def make_problem(name: str, seed: int = 0, B: int | None = None) -> dict:
    """One planning problem plus its initial samples.

    Returns a dict with the problem description (q, T, m, r, r_c, n, obstacle
    tracks xo/yo of shape (n, q), semi-axes ao/bo, v_max, a_max, rho,
    rho_psi, boundary conditions) and ``init`` of shape (B, 3, 11) holding
    c_x, c_y, c_psi per trajectory, plus ``iters``.
    """
    rng = np.random.default_rng(seed)
    x_bc, y_bc, psi_bc = _boundary()
    if name == "tiny":
        q, T, Bd = 50, 5.0, 32
        r = np.array([-0.3, 0.3])
        xo, yo, ao, bo = _static_circles(rng, 4, q, 0.5)
        v_max = a_max = 4.0
        init = _init_gaussian(rng, B or Bd, sigma_iid=0.5)
    elif name in ("paper", "precision"):
        q, T = 100, 10.0
        Bd = 1000 if name == "paper" else 4096
        r = np.array([-0.4, 0.0, 0.4])
        xo, yo, ao, bo = _moving_ellipses(rng, 10, q, T)
        v_max = a_max = 2.0
        init = _init_gaussian(rng, B or Bd, sigma_iid=None)
    else:
        raise ValueError(f"unknown workload {name!r}")
    return dict(name=name, seed=seed, q=q, T=T, degree=DEGREE, m=len(r), r=_f32(r),
                r_c=0.35, n=xo.shape[0], xo=xo, yo=yo, ao=ao, bo=bo,
                v_max=v_max, a_max=a_max, rho=1.0, rho_psi=1.0,
                x_bc=x_bc, y_bc=y_bc, psi_bc=psi_bc,
                B=init.shape[0], init=init, iters=100)


def make_uneven(seed: int = 0, count: int = 64, scale: float = 1.0) -> list[dict]:
    """Mixed problems for the uneven-batching workload.

    Per problem: batch uniform over the integers 128..2048 (times ``scale``,
    at least 1), horizon in {50, 100, 150} steps over q/10 s, 2..32 moving
    ellipses, 2..4 circles evenly spaced over [-0.4, 0.4] m.
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        B = max(1, int(round(rng.integers(128, 2049) * scale)))
        q = int(rng.choice([50, 100, 150]))
        T = q / 10.0
        n = int(rng.integers(2, 33))
        m = int(rng.integers(2, 5))
        r = np.linspace(-0.4, 0.4, m)
        xo, yo, ao, bo = _moving_ellipses(rng, n, q, T)
        x_bc, y_bc, psi_bc = _boundary()
        init = _init_gaussian(rng, B, sigma_iid=None)
        out.append(dict(name=f"uneven{k}", seed=seed, q=q, T=T, degree=DEGREE, m=m,
                        r=_f32(r), r_c=0.35, n=n, xo=xo, yo=yo, ao=ao, bo=bo,
                        v_max=2.0, a_max=2.0, rho=1.0, rho_psi=1.0,
                        x_bc=x_bc, y_bc=y_bc, psi_bc=psi_bc,
                        B=B, init=init, iters=100))
    return out


def make_shape(seed: int, B: int, q: int, n: int, m: int) -> dict:
    """A problem of an arbitrary shape (for edge cases: the largest horizons and
    obstacle counts, single steps of the size range): q steps over q/10 s, n
    moving ellipses as in ``paper``, m circles evenly spaced over
    [-0.4, 0.4] m (0 m for m = 1), B initial samples as in ``paper``."""
    rng = np.random.default_rng(seed)
    T = q / 10.0
    r = np.linspace(-0.4, 0.4, m) if m > 1 else np.zeros(1)
    xo, yo, ao, bo = _moving_ellipses(rng, n, q, T)
    x_bc, y_bc, psi_bc = _boundary()
    init = _init_gaussian(rng, B, sigma_iid=None)
    return dict(name=f"shape_q{q}_n{n}_m{m}", seed=seed, q=q, T=T, degree=DEGREE, m=m,
                r=_f32(r), r_c=0.35, n=n, xo=xo, yo=yo, ao=ao, bo=bo,
                v_max=2.0, a_max=2.0, rho=1.0, rho_psi=1.0,
                x_bc=x_bc, y_bc=y_bc, psi_bc=psi_bc, B=B, init=init, iters=100)


def with_obstacles_removed(pb: dict, v_max: float = 1e6, a_max: float = 1e6) -> dict:
    """Copy of a problem with no obstacles and (by default) inactive bounds."""
    out = dict(pb)
    q = pb["q"]
    out.update(n=0, xo=np.zeros((0, q)), yo=np.zeros((0, q)), ao=np.zeros(0),
               bo=np.zeros(0), v_max=v_max, a_max=a_max)
    return out


CROWD_KINDS = ("static", "same", "opposite")


def make_crowd(kind: str, seed: int, n: int = 30, radius: float = 0.3, v_des: float = 1.0,
               width: float = 5.0) -> dict:
    """One closed-loop benchmark scene (Sec. IV, Benchmarks 1-3), synthetic.

    n people of radius ``radius`` with centres uniform in x in [3, 25] m
    (static, same) or [6, 36] m (opposite, walking towards the robot) and y in
    [-width, width] m, at least 1.2 m apart and 2 m from the robot's start (0, 0);
    velocities 0 (static), vx uniform in [0, 0.3] m/s (same direction as the
    robot), or vx uniform in [-1.0, -0.3] m/s (opposite), with vy uniform in
    [-0.05, 0.05] m/s for the moving crowds.  The desired motion is
    (v_des t, 0).  Rejection draws are part of the seeded stream.
    """
    if kind not in CROWD_KINDS:
        raise ValueError(f"unknown crowd {kind!r}")
    rng = np.random.default_rng(seed)
    xlo, xhi = (6.0, 36.0) if kind == "opposite" else (3.0, 25.0)
    pos = []
    while len(pos) < n:
        p = np.array([rng.uniform(xlo, xhi), rng.uniform(-width, width)])
        if np.hypot(*p) < 2.0 or any(np.hypot(*(p - o)) < 1.2 for o in pos):
            continue
        pos.append(p)
    pos = np.array(pos)
    if kind == "static":
        vel = np.zeros((n, 2))
    elif kind == "same":
        vel = np.stack([rng.uniform(0.0, 0.3, n), rng.uniform(-0.05, 0.05, n)], 1)
    else:
        vel = np.stack([rng.uniform(-1.0, -0.3, n), rng.uniform(-0.05, 0.05, n)], 1)
    return dict(kind=kind, seed=seed, n=n, p0=_f32(pos), v=_f32(vel), radius=float(np.float32(radius)),
                v_des=v_des)


def crowd_positions(crowd: dict, t) -> tuple[np.ndarray, np.ndarray]:
    """Centres of the crowd at the times t (any shape): xo, yo of shape (n,) + t.shape."""
    t = np.asarray(t, dtype=np.float64)
    xo = crowd["p0"][:, 0].reshape((-1,) + (1,) * t.ndim) + crowd["v"][:, 0].reshape((-1,) + (1,) * t.ndim) * t
    yo = crowd["p0"][:, 1].reshape((-1,) + (1,) * t.ndim) + crowd["v"][:, 1].reshape((-1,) + (1,) * t.ndim) * t
    return xo, yo
