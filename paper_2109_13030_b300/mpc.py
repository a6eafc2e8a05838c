"""Closed-loop model-predictive control on crowd scenes (Sec. IV).

The paper runs its batch optimizer as an MPC: every control step re-plans
from the robot's current state, with the batch drawn around a straight line
and the multipliers warm-started from the previous step, and reports the
success rate (episodes without a collision), the tracking error against a
straight line at constant speed, and the acceleration used (Table III), for
batch sizes from 1 to 1000.

Here every episode is one scene of a re-planning server (``trajam.Server``),
so the control steps of all episodes go through the GPU in batched rounds.
Per control step and episode the request carries:

* advance = dt: the start state is the previous best plan at t = dt (the
  robot executes each plan for one control period);
* the crowd's predicted centre tracks over the horizon (constant velocity,
  which is also how the simulated people move);
* the goal: the desired motion at the horizon's end, (v_des (t + T), 0) with
  velocity (v_des, 0), zero acceleration and heading 0, moved sideways when a
  person will be there (the paper's cost has no tracking term; the moving goal
  is how the plans follow the line);
* with ``resample``, a re-draw of the batch around the straight line from start
  to goal with the multipliers kept (``am_resample``, the paper's reading of
  the warm start).  By default the batch instead keeps its coefficients,
  re-timed by the control period (``am_shift``), and its multipliers, scaled
  by ``lambda_decay`` (``am_scale_multipliers``); only the first step draws.
  Kept coefficients let ten iterations per step add up instead of
  restarting.  Kept multipliers carry the collision avoidance built up so
  far, but also pull the plans back towards the previous window.  The
  default keeps them whole (the paper's warm start), which succeeds most
  often; a decay of 0.9 per step halves the tracking error and costs success
  in dense crowds (measured on 60 episodes per crowd).

The planner sees the people with ``margin`` added to their radius, and picks,
when no plan of the batch is collision-free, the one with the most clearance
(AM_SELECT_CLEARANCE).  The executed motion is the best plan of each step over
[0, dt], evaluated at ``substeps`` points (``am_plan_eval``).  A collision is a
robot circle (body offsets r_i along the heading, radius r_c) whose centre
comes within 0.99 (r_c + radius) of a person (true radius, no margin), the
same 0.99 as the best-trajectory rule of the solver.
"""
from __future__ import annotations

import statistics
import time
from dataclasses import dataclass

import numpy as np

from . import trajam as TJ
from . import workload as W

R_BODY = (-0.4, 0.0, 0.4)
R_C = 0.35


@dataclass
class MPCConfig:
    batch: int = 1000        # trajectories per re-plan
    iters: int = 10          # AM iterations per re-plan (the paper's MPC: 10)
    dt: float = 0.1          # control period (s)
    duration: float = 20.0   # episode length (s)
    q: int = 100             # planning steps
    horizon: float = 10.0    # planning horizon T (s)
    sigma: float = 1.0       # scale of the batch draw around the straight line (m)
    substeps: int = 5        # evaluation points of the executed motion per control period
    v_max: float = 2.0
    a_max: float = 2.0
    seed: int = 0            # seed of the batch draws
    free_goal: bool = True   # move the goal sideways off people (see goal_state)
    resample: bool = False   # re-draw the batch every step (else keep xi as well as lambda)
    shift: bool = True       # kept xi: re-time it by the control period (am_shift)
    lambda_decay: float = 1.0  # multipliers scaled by this at each step (1 keeps them, 0 resets)
    select: int = TJ.AM_SELECT_CLEARANCE  # when no plan is collision-free, take the one with the most clearance
    margin: float = 0.2      # added to the people's radius in the planner only (m)


def _problem(crowd: dict, cfg: MPCConfig) -> dict:
    """The planning problem of an episode at t = 0 (start at rest at the origin)."""
    tg = np.linspace(0.0, cfg.horizon, cfg.q)
    xo, yo = W.crowd_positions(crowd, tg)
    v = crowd["v_des"]
    n = crowd["n"]
    line = np.zeros((cfg.batch, 3, W.NV))
    line[:, 0, :] = W.straight_line_coeffs(0.0, v * cfg.horizon)
    return dict(q=cfg.q, T=cfg.horizon, degree=W.DEGREE, m=len(R_BODY), r=np.array(R_BODY), r_c=R_C,
                n=n, xo=xo, yo=yo, ao=np.full(n, crowd["radius"] + cfg.margin),
                bo=np.full(n, crowd["radius"] + cfg.margin),
                v_max=cfg.v_max, a_max=cfg.a_max, rho=1.0, rho_psi=1.0,
                x_bc=np.array([0.0, 0.0, 0.0, v * cfg.horizon, v, 0.0]), y_bc=np.zeros(6),
                psi_bc=np.zeros(6), B=cfg.batch, init=line)


GOAL_OFFSETS = np.concatenate([[0.0], np.repeat(np.arange(1, 21) * 0.25, 2) * np.tile([1.0, -1.0], 20)])


def goal_state(crowd: dict, t: float, cfg: MPCConfig) -> np.ndarray:
    """Goal at the end of the horizon started at t: the desired motion
    (v_des (t + T), 0) at heading 0.  With free_goal, a goal whose robot
    circles would come within 1.2 (r_c + radius) of a person at t + T moves
    sideways to the nearest free offset (steps of 0.25 m up to 5 m): a goal
    inside a person leaves no collision-free trajectory in the batch."""
    v = crowd["v_des"]
    x = v * (t + cfg.horizon)
    y = 0.0
    if cfg.free_goal:
        xo, yo = W.crowd_positions(crowd, np.array([t + cfg.horizon]))
        for dy in GOAL_OFFSETS:
            d = min(np.hypot(x + r - xo[:, 0], dy - yo[:, 0]).min() for r in R_BODY)
            if d >= 1.2 * (R_C + crowd["radius"]):
                y = dy
                break
    return np.array([x, v, 0.0, y, 0.0, 0.0, 0.0, 0.0, 0.0])


def circle_clearance(states: np.ndarray, crowd: dict, t: np.ndarray) -> np.ndarray:
    """Smallest distance from any robot circle centre to any person, over the
    crowd, divided by (r_c + radius): one value per row of states (x, ., ., y,
    ., ., psi, ., .) at the times t."""
    xo, yo = W.crowd_positions(crowd, t)          # (n, len(t))
    out = np.full(len(t), np.inf)
    for r in R_BODY:
        cx = states[:, 0] + r * np.cos(states[:, 6])
        cy = states[:, 3] + r * np.sin(states[:, 6])
        d = np.hypot(cx[None, :] - xo, cy[None, :] - yo).min(axis=0)
        out = np.minimum(out, d)
    return out / (R_C + crowd["radius"])


def episode_metrics(states: np.ndarray, t: np.ndarray, crowd: dict) -> dict:
    """Success, tracking error and acceleration of an executed motion (Sec. IV metrics).

    states: (len(t), 9) rows x, x', x'', y, y', y'', psi, psi', psi''.
    Tracking error: mean over time of the distance to the desired point
    (v_des t, 0) (and that distance at the last sample); acceleration: mean
    over time of |(x'', y'')|.
    """
    clear = circle_clearance(states, crowd, t)
    hit = np.nonzero(clear < 0.99)[0]
    err = np.hypot(states[:, 0] - crowd["v_des"] * t, states[:, 3])
    acc = np.hypot(states[:, 2], states[:, 5])
    return dict(success=bool(hit.size == 0), collision_time=float(t[hit[0]]) if hit.size else None,
                min_clearance=float(clear.min()), tracking_error=float(err.mean()),
                final_tracking_error=float(err[-1]), acceleration=float(acc.mean()))


def run(crowds: list[dict], cfg: MPCConfig, budget_bytes: int = 16 << 30) -> dict:
    """Run one closed-loop episode per crowd, all through one server, and
    return the per-episode metrics and the re-plan latencies."""
    steps = int(round(cfg.duration / cfg.dt))
    problems, server = [], None
    try:
        server = TJ.Server(budget_bytes, cfg.iters, mode=TJ.AM_SRV_BATCHED)
        for crowd in crowds:
            pb = _problem(crowd, cfg)
            P = TJ.Problem(pb, select=cfg.select)
            problems.append(P)
            server.add_scene(P, pb["init"].astype(np.float32))
        server.start()
        sub = np.arange(cfg.substeps) * (cfg.dt / cfg.substeps)
        traj = [[] for _ in crowds]
        feasible = [0 for _ in crowds]
        lat, batches = [], []
        tg = np.linspace(0.0, cfg.horizon, cfg.q)
        t_wall = time.perf_counter()
        for k in range(steps):
            t = k * cfg.dt
            tickets = []
            for e, crowd in enumerate(crowds):
                xo, yo = W.crowd_positions(crowd, t + tg)
                seed = ((cfg.seed * 1_000_003 + e) * 1_000_033 + k) & (2**64 - 1)
                tickets.append(server.submit(e, advance=cfg.dt if k else 0.0, xo=xo, yo=yo,
                                             goal=goal_state(crowd, t, cfg),
                                             resample_seed=seed if (cfg.resample or k == 0) else None,
                                             sigma=cfg.sigma, shift=cfg.shift,
                                             lambda_scale=(cfg.lambda_decay if k > 0 and cfg.lambda_decay != 1.0
                                                           else None)))
            for e, tk in enumerate(tickets):
                r = server.wait(tk)
                if r["status"] != TJ.AM_OK:
                    raise TJ.TrajamError(r["status"], f"episode {e} step {k} failed")
                lat.append(r["t_done"] - r["t_submit"])
                batches.append(r["batch"])
                traj[e].append(TJ.am_plan_eval(r["coeffs"], cfg.horizon, sub))
                plan = TJ.am_plan_eval(r["coeffs"], cfg.horizon, tg)
                feasible[e] += int(circle_clearance(plan, crowds[e], k * cfg.dt + tg).min() >= 0.99)
        wall = time.perf_counter() - t_wall
    finally:
        if server is not None:
            server.close()
        for P in problems:
            P.close()
    times = np.arange(steps * cfg.substeps) * (cfg.dt / cfg.substeps)
    episodes = [dict(kind=c["kind"], seed=c["seed"], feasible_plans=f / steps,
                     **episode_metrics(np.concatenate(s), times, c))
                for c, s, f in zip(crowds, traj, feasible)]
    lat_ms = sorted(1e3 * x for x in lat)
    return dict(episodes=episodes, steps=steps, wall_s=wall,
                replan_ms={"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1, int(0.99 * len(lat_ms)))]},
                mean_round_batch=statistics.mean(batches))


def run_cem(crowds: list[dict], cfg: MPCConfig, **cem) -> dict:
    """The same closed loop with the CEM comparator as the planner (Sec. IV,
    Table IV): per step and episode one ``am_cem_solve`` on the episode's own
    problem, warm-started from the previous best plan re-timed by dt.  The
    boundary, goal, obstacle tracks, planning margin and metrics are those of
    ``run``; the episodes are planned one after another.  Keyword arguments
    override ``trajam.CEM_DEFAULTS``."""
    steps = int(round(cfg.duration / cfg.dt))
    tg = np.linspace(0.0, cfg.horizon, cfg.q)
    sub = np.arange(cfg.substeps) * (cfg.dt / cfg.substeps)
    problems = [TJ.Problem(_problem(c, cfg)) for c in crowds]
    traj = [[] for _ in crowds]
    feasible = [0 for _ in crowds]
    plans = [None for _ in crowds]
    lat = []
    t_wall = time.perf_counter()
    try:
        for k in range(steps):
            t = k * cfg.dt
            for e, crowd in enumerate(crowds):
                P = problems[e]
                xo, yo = W.crowd_positions(crowd, t + tg)
                rad = np.full(crowd["n"], crowd["radius"] + cfg.margin)
                P.set_obstacles(xo, yo, rad, rad)
                start = np.zeros(9) if plans[e] is None else TJ.am_plan_eval(plans[e], cfg.horizon, [cfg.dt])[0]
                g = goal_state(crowd, t, cfg)
                P.set_boundary(np.r_[start[0:3], g[0:3]], np.r_[start[3:6], g[3:6]], np.r_[start[6:9], g[6:9]])
                t0 = time.perf_counter()
                seed = ((cfg.seed * 1_000_003 + e) * 1_000_033 + k) & (2**64 - 1)
                TJ.am_cem_solve(P.h, warm=plans[e], warm_dt=cfg.dt if plans[e] is not None else 0.0,
                                **dict(dict(seed=seed), **cem))
                best = TJ.am_cem_get_best(P.h)
                lat.append(time.perf_counter() - t0)
                plans[e] = best["coeffs"]
                traj[e].append(TJ.am_plan_eval(plans[e], cfg.horizon, sub))
                plan = TJ.am_plan_eval(plans[e], cfg.horizon, tg)
                feasible[e] += int(circle_clearance(plan, crowd, t + tg).min() >= 0.99)
        wall = time.perf_counter() - t_wall
    finally:
        for P in problems:
            P.close()
    times = np.arange(steps * cfg.substeps) * (cfg.dt / cfg.substeps)
    episodes = [dict(kind=c["kind"], seed=c["seed"], feasible_plans=f / steps,
                     **episode_metrics(np.concatenate(s), times, c))
                for c, s, f in zip(crowds, traj, feasible)]
    lat_ms = sorted(1e3 * x for x in lat)
    return dict(episodes=episodes, steps=steps, wall_s=wall,
                replan_ms={"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1, int(0.99 * len(lat_ms)))]})


def summarize(episodes: list[dict]) -> dict:
    """Table III-style statistics: success rate, tracking error and
    acceleration as mean / max / min over episodes (and the share of control
    steps whose chosen plan was collision-free over its whole horizon)."""
    def mmm(key):
        v = [e[key] for e in episodes]
        return {"mean": float(np.mean(v)), "max": float(np.max(v)), "min": float(np.min(v))}
    return {"episodes": len(episodes),
            "success_rate": float(np.mean([e["success"] for e in episodes])),
            "tracking_error_m": mmm("tracking_error"), "acceleration_mps2": mmm("acceleration"),
            **({"feasible_plan_share": float(np.mean([e["feasible_plans"] for e in episodes]))}
               if all("feasible_plans" in e for e in episodes) else {})}
