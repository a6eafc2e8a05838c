"""The closed loop of Sec. IV on the GPU: the batch re-draw, the server's goal
and advance updates, and whole episodes.

am_resample's draw is checked against its definition: trajectory 0 is the
straight line, the boundary control points are the line's, the interior
deviations of c_x and c_y have mean 0 and the covariance of
``workload.smoothness_covariance`` (an independent numpy statement of the
same matrix), their whitened values are standard normal (Kolmogorov-Smirnov),
x and y are independent, and the multipliers are untouched.
"""
import numpy as np
import pytest
from scipy import stats

from paper_2109_13030_b300 import mpc as M
from paper_2109_13030_b300 import workload as W

pytestmark = pytest.mark.gpu


def tj():
    from paper_2109_13030_b300 import trajam
    return trajam


def line_points(p0, p1):
    w = np.clip((np.arange(11) - 2) / 6.0, 0.0, 1.0)
    return p0 + (p1 - p0) * w


@pytest.fixture(scope="module")
def drawn():
    T = tj()
    pb = W.make_problem("paper", 0, B=4096)
    P = T.Problem(pb).init_state(pb["init"].astype(np.float32))
    s = P.state()
    rng = np.random.default_rng(4)
    s[:, 55:] = rng.normal(size=(pb["B"], 55)).astype(np.float32)
    T.am_set_state(P.h, pb["B"], s)
    P.resample(seed=7, sigma=1.0)
    a = P.state()
    P.resample(seed=7, sigma=1.0)
    b = P.state()
    P.resample(seed=8, sigma=1.0)
    c = P.state()
    P.resample(seed=8, sigma=0.0)
    z = P.state()
    P.close()
    return pb, s, a, b, c, z


def test_resample_keeps_multipliers_and_is_seeded(drawn):
    pb, s, a, b, c, z = drawn
    np.testing.assert_array_equal(a[:, 55:], s[:, 55:])
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a[1:, :55], c[1:, :55])


def test_resample_line_and_boundary_points(drawn):
    pb, s, a, b, c, z = drawn
    lx = line_points(pb["x_bc"][0], pb["x_bc"][3])
    ly = line_points(pb["y_bc"][0], pb["y_bc"][3])
    lp = line_points(pb["psi_bc"][0], pb["psi_bc"][3])
    for st in (a, z):
        np.testing.assert_allclose(st[:, [0, 1, 2, 8, 9, 10]], np.broadcast_to(lx[[0, 1, 2, 8, 9, 10]], (pb["B"], 6)), atol=1e-6)
        np.testing.assert_allclose(st[:, 44:55], np.broadcast_to(lp, (pb["B"], 11)), atol=1e-6)
        np.testing.assert_allclose(st[:, 11:22], np.cos(st[:, 44:55]), atol=1e-6)
        np.testing.assert_allclose(st[:, 33:44], np.sin(st[:, 44:55]), atol=1e-6)
    np.testing.assert_allclose(a[0, 0:11], lx, atol=1e-5)      # trajectory 0: no perturbation
    np.testing.assert_allclose(a[0, 22:33], ly, atol=1e-5)
    np.testing.assert_allclose(z[:, 0:11], np.broadcast_to(lx, (pb["B"], 11)), atol=1e-5)  # sigma = 0


def test_resample_distribution(drawn):
    pb, s, a, b, c, z = drawn
    lx = line_points(pb["x_bc"][0], pb["x_bc"][3])
    ly = line_points(pb["y_bc"][0], pb["y_bc"][3])
    dx = a[1:, 3:8].astype(np.float64) - lx[3:8]
    dy = a[1:, 25:30].astype(np.float64) - ly[3:8]
    n = dx.shape[0]
    cov = W.smoothness_covariance()
    for d in (dx, dy):
        assert np.all(np.abs(d.mean(0)) <= 5.0 / np.sqrt(n))
        assert np.abs(np.cov(d.T) - cov).max() <= 0.1
        w = np.linalg.solve(np.linalg.cholesky(cov), d.T).ravel()   # whitened: iid N(0, 1)
        assert stats.kstest(w, "norm").pvalue > 1e-4
    assert np.abs(np.cov(dx.T, dy.T)[:5, 5:]).max() <= 0.1


def test_resample_argument_checks():
    T = tj()
    pb = W.make_problem("tiny", 0)
    P = T.Problem(pb)
    with pytest.raises(T.TrajamError) as e:
        P.resample(1)
    assert e.value.code == T.AM_ERR_STATE
    P.init_state(pb["init"].astype(np.float32))
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(T.TrajamError) as e:
            P.resample(1, sigma=bad)
        assert e.value.code == T.AM_ERR_ARG
    P.close()


def test_server_goal_and_advance():
    """A request's goal becomes the plan's end state; with advance the plan
    starts where the previous best plan was at t = advance."""
    T = tj()
    crowd = W.make_crowd("static", 1, n=4)
    cfg = M.MPCConfig(batch=128, iters=30)
    pb = M._problem(crowd, cfg)
    P = T.Problem(pb)
    S = T.Server(1 << 30, cfg.iters)
    S.add_scene(P, pb["init"].astype(np.float32))
    S.start()
    try:
        xo, yo = W.crowd_positions(crowd, np.linspace(0, cfg.horizon, cfg.q))
        g1 = np.array([9.0, 0.8, 0.0, 0.5, 0.0, 0.0, 0.1, 0.0, 0.0])
        r1 = S.wait(S.submit(0, xo=xo, yo=yo, goal=g1, resample_seed=3))
        e1 = T.am_plan_eval(r1["coeffs"], cfg.horizon, [0.0, 0.1, cfg.horizon])
        np.testing.assert_allclose(e1[2], g1, atol=2e-3)
        np.testing.assert_allclose(e1[0], [0, 0, 0, 0, 0, 0, 0, 0, 0], atol=2e-3)
        g2 = np.array([10.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
        r2 = S.wait(S.submit(0, advance=0.1, xo=xo, yo=yo, goal=g2, resample_seed=4))
        e2 = T.am_plan_eval(r2["coeffs"], cfg.horizon, [0.0, cfg.horizon])
        np.testing.assert_allclose(e2[0], e1[1], atol=2e-3)
        np.testing.assert_allclose(e2[1], g2, atol=2e-3)
        with pytest.raises(T.TrajamError):
            S.submit(0, goal=np.full(9, np.nan))
        with pytest.raises(T.TrajamError):
            S.submit(0, resample_seed=1, sigma=-1.0)
    finally:
        S.close()
        P.close()


def test_closed_loop_free_space():
    """One person far off the line: every episode succeeds, and the robot,
    which starts at rest behind the desired point, catches up (its final
    distance to the desired point is below its mean distance)."""
    far = dict(kind="static", seed=0, n=1, p0=np.array([[10.0, 30.0]]), v=np.zeros((1, 2)),
               radius=0.3, v_des=1.0)
    cfg = M.MPCConfig(batch=64, duration=12.0)
    out = M.run([far, dict(far, seed=1)], cfg)
    s = M.summarize(out["episodes"])
    assert s["success_rate"] == 1.0
    for e in out["episodes"]:
        assert e["final_tracking_error"] < e["tracking_error"] < 4.0
    assert s["acceleration_mps2"]["max"] < cfg.a_max
    assert out["steps"] == 120 and out["replan_ms"]["p50"] > 0


@pytest.mark.parametrize("batch", [1, 256])
def test_closed_loop_crowds_run(batch):
    crowds = [W.make_crowd(k, 11) for k in W.CROWD_KINDS]
    out = M.run(crowds, M.MPCConfig(batch=batch, duration=4.0))
    assert len(out["episodes"]) == 3 and out["mean_round_batch"] >= 1
    for e in out["episodes"]:
        assert np.isfinite(e["tracking_error"]) and np.isfinite(e["acceleration"])
        assert e["min_clearance"] > 0


def expected_best(res, rule):
    """The selection rule written out: collision-free (smallest distance >=
    0.99) by cost first; otherwise the lowest cost (AM_SELECT_COST) or the
    largest smallest distance (AM_SELECT_CLEARANCE); ties to the lower index."""
    mind, cost = res["mind"], res["cost"]
    free = np.nonzero(mind >= np.float32(0.99))[0]
    if free.size:
        return int(free[np.argmin(cost[free])])
    return int(np.argmin(cost)) if rule == 0 else int(np.argmax(mind))


@pytest.mark.parametrize("blocked", [False, True])
def test_selection_rules(blocked):
    """Both rules against their definition on the solver's own results.  With
    obstacle 0 made a static disc of radius 4.5 m halfway between start and
    goal (inflated, it still leaves both outside), every trajectory collides
    after three iterations, each to its own depth, which exercises the
    fallback."""
    T = tj()
    pb = W.make_problem("paper", 0, B=512)
    if blocked:
        pb = dict(pb, xo=pb["xo"].copy(), yo=pb["yo"].copy(), ao=pb["ao"].copy(), bo=pb["bo"].copy())
        pb["xo"][0, :] = 4.0
        pb["yo"][0, :] = 4.0
        pb["ao"][0] = pb["bo"][0] = 4.5
    picks = {}
    for rule in (T.AM_SELECT_COST, T.AM_SELECT_CLEARANCE):
        P = T.Problem(pb, select=rule)
        P.solve(pb["init"].astype(np.float32), 3)
        r = P.results()
        assert P.best()["index"] == expected_best(r, rule)
        picks[rule] = P.best()["index"]
        if blocked:
            assert np.all(r["mind"] < 0.99) and np.unique(r["mind"]).size > 100
        P.close()
    if not blocked:
        assert picks[0] == picks[1]


def test_shift_retimes_every_polynomial():
    """After am_shift(dt) each polynomial of the batch evaluated at t equals the
    old one at t + dt (values and both derivatives), for the five polynomials;
    the multipliers are untouched; dt = 0 is the identity."""
    T = tj()
    pb = W.make_problem("paper", 0, B=256)
    P = T.Problem(pb)
    P.solve(pb["init"].astype(np.float32), 5)
    old = P.state()
    dt = 0.37
    P.shift(dt)
    new = P.state()
    np.testing.assert_array_equal(new[:, 55:], old[:, 55:])
    t = np.linspace(0.0, pb["T"] - dt, 23)
    for l in (0, 17, 255):
        for base in (0, 11, 22, 33, 44):
            a = np.zeros(33, np.float32)
            b = np.zeros(33, np.float32)
            a[:11] = new[l, base:base + 11]
            b[:11] = old[l, base:base + 11]
            ea = T.am_plan_eval(a, pb["T"], t)[:, :3]
            eb = T.am_plan_eval(b, pb["T"], t + dt)[:, :3]
            scale = np.abs(b[:11]).max() + 1.0
            for d, unit in enumerate((1.0, 10.0 / pb["T"], 100.0 / pb["T"] ** 2)):
                np.testing.assert_allclose(ea[:, d], eb[:, d], atol=2e-5 * scale * unit)
    P.shift(0.0)
    np.testing.assert_allclose(P.state(), new, atol=1e-6)
    for bad in (-0.1, pb["T"] + 0.1, float("nan")):
        with pytest.raises(T.TrajamError) as e:
            P.shift(bad)
        assert e.value.code == T.AM_ERR_ARG
    P.close()


def test_closed_loop_with_cem_runs():
    from paper_2109_13030_b300 import mpc as M2
    crowds = [W.make_crowd(k, 12) for k in W.CROWD_KINDS]
    out = M2.run_cem(crowds, M2.MPCConfig(duration=2.0), samples=1024, elites=100, iters=5)
    assert len(out["episodes"]) == 3 and out["steps"] == 20
    for e in out["episodes"]:
        assert np.isfinite(e["tracking_error"]) and e["min_clearance"] > 0


def test_scale_multipliers_touches_lambda_only():
    T = tj()
    pb = W.make_problem("paper", 0, B=200)
    P = T.Problem(pb)
    P.solve(pb["init"].astype(np.float32), 5)
    before = P.state()
    assert np.abs(before[:, 55:]).max() > 0
    P.scale_multipliers(0.5)
    half = P.state()
    np.testing.assert_array_equal(half[:, :55], before[:, :55])
    np.testing.assert_array_equal(half[:, 55:], before[:, 55:] * np.float32(0.5))
    P.scale_multipliers(1.0)
    np.testing.assert_array_equal(P.state(), half)
    P.scale_multipliers(0.0)
    zero = P.state()
    np.testing.assert_array_equal(zero[:, :55], before[:, :55])
    assert not zero[:, 55:].any()
    for bad in (-0.5, float("nan")):
        with pytest.raises(T.TrajamError) as e:
            P.scale_multipliers(bad)
        assert e.value.code == T.AM_ERR_ARG
    P.close()
    Q = T.Problem(pb)
    with pytest.raises(T.TrajamError) as e:
        Q.scale_multipliers(0.0)
    assert e.value.code == T.AM_ERR_STATE
    Q.close()
