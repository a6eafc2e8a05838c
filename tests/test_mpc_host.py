"""Host side of the closed loop (Sec. IV): plan evaluation, the crowd scenes,
the goal, and the metrics.  No device work.

am_plan_eval is pinned by exact polynomial reproduction: a polynomial
p(tau) = sum_i a_i tau^i of degree <= 10 has the Bernstein control points
c_k = sum_{i <= k} a_i C(k, i) / C(10, i) (degree elevation of the monomials),
so the evaluated value and time derivatives must equal p, p' / T, p'' / T^2.
"""
from math import comb

import numpy as np
import pytest

from paper_2109_13030_b300 import mpc as M
from paper_2109_13030_b300 import trajam as TJ
from paper_2109_13030_b300 import workload as W


def bernstein_points(a):
    """Control points of sum_i a_i tau^i (degree elevation to 10)."""
    return np.array([sum(a[i] * comb(k, i) / comb(10, i) for i in range(min(k, len(a) - 1) + 1))
                     for k in range(11)])


@pytest.mark.parametrize("T", [1.0, 5.0, 10.0])
def test_plan_eval_reproduces_polynomials(T):
    rng = np.random.default_rng(1)
    polys = [rng.uniform(-2, 2, size=d + 1) for d in (1, 3, 5)]
    coeffs = np.concatenate([bernstein_points(a) for a in polys]).astype(np.float32)
    t = np.concatenate([[0.0, T], rng.uniform(0, T, 20)])
    out = TJ.am_plan_eval(coeffs, T, t)
    tau = t / T
    for s, a in enumerate(polys):
        p = np.polynomial.Polynomial(a)
        scale = np.abs(a).sum()
        np.testing.assert_allclose(out[:, 3 * s], p(tau), atol=2e-6 * scale)
        np.testing.assert_allclose(out[:, 3 * s + 1], p.deriv(1)(tau) / T, atol=2e-5 * scale / T)
        np.testing.assert_allclose(out[:, 3 * s + 2], p.deriv(2)(tau) / T ** 2, atol=2e-4 * scale / T ** 2)


def test_plan_eval_ends_and_clamping():
    c = np.random.default_rng(2).uniform(-1, 1, 33).astype(np.float32)
    T = 4.0
    out = TJ.am_plan_eval(c, T, [-1.0, 0.0, T, T + 3.0])
    for s in range(3):
        cs = c[11 * s: 11 * s + 11].astype(np.float64)
        assert out[1, 3 * s] == pytest.approx(cs[0], abs=1e-12)
        assert out[2, 3 * s] == pytest.approx(cs[10], abs=1e-12)
        assert out[1, 3 * s + 1] == pytest.approx(10 * (cs[1] - cs[0]) / T, rel=1e-12, abs=1e-12)
        assert out[2, 3 * s + 2] == pytest.approx(90 * (cs[10] - 2 * cs[9] + cs[8]) / T ** 2, rel=1e-12, abs=1e-12)
    np.testing.assert_array_equal(out[0], out[1])   # clamped to [0, T]
    np.testing.assert_array_equal(out[3], out[2])


def test_plan_eval_rejects_bad_arguments():
    c = np.zeros(33, np.float32)
    with pytest.raises(TJ.TrajamError):
        TJ.am_plan_eval(c, 0.0, [0.0])
    with pytest.raises(TJ.TrajamError):
        TJ.am_plan_eval(c, 1.0, [np.nan])
    bad = c.copy()
    bad[5] = np.inf
    with pytest.raises(TJ.TrajamError):
        TJ.am_plan_eval(bad, 1.0, [0.5])


@pytest.mark.parametrize("kind", W.CROWD_KINDS)
def test_crowd_scene(kind):
    c = W.make_crowd(kind, 5)
    again = W.make_crowd(kind, 5)
    np.testing.assert_array_equal(c["p0"], again["p0"])
    p, v = c["p0"], c["v"]
    assert p.shape == (30, 2) and v.shape == (30, 2)
    d = np.hypot(p[:, None, 0] - p[None, :, 0], p[:, None, 1] - p[None, :, 1]) + 10 * np.eye(30)
    assert d.min() >= 1.2 - 1e-6 and np.hypot(p[:, 0], p[:, 1]).min() >= 2.0 - 1e-6
    assert np.all(np.abs(p[:, 1]) <= 5.0)
    assert np.all(np.abs(W.make_crowd(kind, 5, width=3.0)["p0"][:, 1]) <= 3.0)
    if kind == "static":
        assert np.all(v == 0)
    elif kind == "same":
        assert np.all((v[:, 0] >= 0) & (v[:, 0] <= 0.3))
    else:
        assert np.all((v[:, 0] >= -1.0) & (v[:, 0] <= -0.3))
    xo, yo = W.crowd_positions(c, np.array([0.0, 2.0]))
    np.testing.assert_allclose(xo[:, 1] - xo[:, 0], 2.0 * v[:, 0])
    np.testing.assert_allclose(yo[:, 0], p[:, 1])


def test_goal_is_the_desired_motion_at_the_horizon_end():
    cfg = M.MPCConfig(horizon=8.0, free_goal=False)
    g = M.goal_state(dict(v_des=1.5), 2.0, cfg)
    np.testing.assert_array_equal(g, [15.0, 1.5, 0, 0, 0, 0, 0, 0, 0])


def test_free_goal_moves_off_a_person():
    cfg = M.MPCConfig(horizon=8.0)
    crowd = dict(n=2, p0=np.array([[15.0, 0.0], [30.0, 0.0]]), v=np.zeros((2, 2)), radius=0.3, v_des=1.5)
    g = M.goal_state(crowd, 2.0, cfg)
    # the first offset (0.25 m steps, + before -) clearing 1.2 (r_c + 0.3) = 0.78 m
    # from every circle centre (x +- 0.4, y)
    assert g[3] == 1.0 and g[0] == 15.0
    crowd["p0"][0] = [40.0, 0.0]
    assert M.goal_state(crowd, 2.0, cfg)[3] == 0.0


def _line(t, v=1.0, y=0.0):
    s = np.zeros((len(t), 9))
    s[:, 0] = v * t
    s[:, 1] = v
    s[:, 3] = y
    return s


def test_metrics_of_exact_tracking_and_of_a_collision():
    t = np.arange(0, 10, 0.02)
    far = dict(kind="static", seed=0, n=1, p0=np.array([[5.0, 10.0]]), v=np.zeros((1, 2)), radius=0.3,
               v_des=1.0)
    m = M.episode_metrics(_line(t), t, far)
    assert m["success"] and m["tracking_error"] == 0.0 and m["acceleration"] == 0.0
    # clearance: nearest circle centre (x = 5 +- 0.4 at t = 5 +- 0.4) is 10 m away
    assert m["min_clearance"] == pytest.approx(10.0 / (M.R_C + 0.3))
    # a person on the line at x = 5: the front circle (x + 0.4) reaches
    # 0.99 (r_c + 0.3) of it first
    on = dict(far, p0=np.array([[5.0, 0.0]]))
    m = M.episode_metrics(_line(t, y=0.0), t, on)
    assert not m["success"]
    reach = 5.0 - 0.4 - 0.99 * (M.R_C + 0.3)
    assert reach <= m["collision_time"] <= reach + 0.02 + 1e-9
    # a parallel line 1 m off: tracking error 1, no collision at 1 m / 0.65 m clearance
    m = M.episode_metrics(_line(t, y=1.0), t, on)
    assert m["success"] and m["tracking_error"] == pytest.approx(1.0)
    assert m["min_clearance"] == pytest.approx(1.0 / (M.R_C + 0.3))


def test_summary_statistics():
    eps = [dict(success=True, tracking_error=1.0, acceleration=0.1),
           dict(success=False, tracking_error=3.0, acceleration=0.3)]
    s = M.summarize(eps)
    assert s["success_rate"] == 0.5 and s["episodes"] == 2
    assert s["tracking_error_m"] == {"mean": 2.0, "max": 3.0, "min": 1.0}
    assert s["acceleration_mps2"]["mean"] == pytest.approx(0.2)
