"""Serving on the GPU: resident scenes, rounds of continuous batching.

A request served in a round together with other scenes' requests must give
the result it gives alone: every scene is advanced by the same per-tile code
whatever else shares the launch, and every per-trajectory sum has a fixed
order whatever the tile and block size, so the result is the same bit for bit
(checked in test_result_alone_equals_result_in_mix; the other comparisons use
the FP32 tolerance of two solves of one problem, 2e-4 relative).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_13030_b300 import workload as W

from test_gpu_parity import COEF_TOL, coef_err
from test_gpu_group import coef_tolerance

pytestmark = pytest.mark.gpu

GB = 1 << 30


def tj():
    from paper_2109_13030_b300 import trajam
    return trajam


def scenes(count=4, seed=21, scale=1.0 / 64):
    return W.make_uneven(seed, count=count, scale=scale)


def make_server(pbs, iters, mode=0, budget=8 * GB, start=True, **kw):
    T = tj()
    S = T.Server(budget, iters, mode=mode, **kw)
    probs = []
    for pb in pbs:
        P = T.Problem(pb)
        S.add_scene(P, pb["init"].astype(np.float32))
        probs.append(P)
    return (S.start() if start else S), probs


def close(S, probs):
    S.close()
    for P in probs:
        P.close()


def assert_same(a, b, tol=2 * COEF_TOL):
    ca, cb = np.asarray(a["coeffs"], np.float64), np.asarray(b["coeffs"], np.float64)
    err = np.max(np.abs(ca - cb)) / max(1.0, np.max(np.abs(cb)))
    assert err <= tol, err
    assert a["cost"] == pytest.approx(b["cost"], rel=1e-3)


def test_result_alone_equals_result_in_mix():
    pbs = scenes()
    S, probs = make_server(pbs, 10)
    alone = S.wait(S.submit(0))
    close(S, probs)
    assert alone["status"] == 0 and alone["batch"] == 1

    S, probs = make_server(pbs, 10, start=False)
    # queued before the start: the first round serves all four together
    tickets = [S.submit(k) for k in range(len(pbs))]
    S.start()
    mixed = [S.wait(t) for t in tickets]
    stats = S.stats()
    close(S, probs)
    assert all(r["status"] == 0 for r in mixed)
    assert stats["completed"] == len(pbs)
    assert all(r["batch"] == len(pbs) for r in mixed)
    assert_same(mixed[0], alone)
    # stronger: the grouped kernel's tiles give the single-problem kernel's bits
    np.testing.assert_array_equal(np.asarray(mixed[0]["coeffs"]), np.asarray(alone["coeffs"]))


def test_request_arriving_during_a_round_overlaps_it():
    """Continuous batching with rounds in flight: with one request per round
    and two lanes, a request for another scene submitted while a long round is
    on the GPU is issued on the second lane and starts before the first round
    completes; both results equal their scenes served alone, bit for bit."""
    big = W.make_shape(31, B=6000, q=100, n=10, m=3)
    small = W.make_shape(32, B=64, q=50, n=4, m=2)
    pbs = [big, small]
    alone = []
    for k in range(2):
        S, probs = make_server(pbs, 200, max_batch=1)
        alone.append(S.wait(S.submit(k)))
        close(S, probs)
    S, probs = make_server(pbs, 200, max_batch=1, lanes=2)
    ta = S.submit(0)
    tb = S.submit(1)
    ra, rb = S.wait(ta), S.wait(tb)
    close(S, probs)
    assert ra["status"] == 0 and rb["status"] == 0
    assert ra["round"] != rb["round"] and ra["batch"] == rb["batch"] == 1
    assert rb["t_start"] < ra["t_done"], (rb["t_start"], ra["t_done"])
    for r, a in zip((ra, rb), alone):
        np.testing.assert_array_equal(np.asarray(r["coeffs"]), np.asarray(a["coeffs"]))
        assert r["cost"] == a["cost"]


@pytest.mark.parametrize("kernel", ["small_tile", "auto"])
def test_full_size_scenes_alone_equal_in_a_round(kernel):
    """Four scenes of the benchmark's serving mix at full size (batches of a
    few hundred to 2048 trajectories), 30 iterations per request: each scene
    served alone, then all four in one grouped round, give the same bits."""
    T = tj()
    k = T.AM_KERNEL_AUTO if kernel == "auto" else T.AM_KERNEL_FUSED
    pbs = W.make_uneven(0, count=64)[:4]
    assert max(pb["B"] for pb in pbs) > 1000

    def serve(ks, start_after_submit):
        S = T.Server(8 * GB, 30)
        probs = []
        for pb in pbs:
            P = T.Problem(pb, kernel=k)
            S.add_scene(P, pb["init"].astype(np.float32))
            probs.append(P)
        if not start_after_submit:
            S.start()
        tickets = [S.submit(i) for i in ks]
        if start_after_submit:
            S.start()
        out = [S.wait(t) for t in tickets]
        close(S, probs)
        return out

    alone = [serve([i], False)[0] for i in range(len(pbs))]
    mixed = serve(range(len(pbs)), True)
    assert all(r["status"] == 0 for r in alone + mixed)
    assert all(r["batch"] == len(pbs) and r["round"] == 0 for r in mixed)
    for a, m in zip(alone, mixed):
        np.testing.assert_array_equal(np.asarray(m["coeffs"]), np.asarray(a["coeffs"]))
        assert m["cost"] == a["cost"] and m["index"] == a["index"]


def test_round_groups_from_three_admissible_requests():
    """Two queued requests for different scenes go to two lanes as rounds of
    one (grouping two costs what two launches cost); three queued requests
    form one grouped round.  Every result equals its scene served alone, bit
    for bit."""
    pbs = scenes(count=3, seed=25)
    alone = []
    for k in range(3):
        S, probs = make_server(pbs, 10)
        alone.append(S.wait(S.submit(k)))
        close(S, probs)
    for count in (2, 3):
        S, probs = make_server(pbs, 10, start=False)
        tickets = [S.submit(k) for k in range(count)]
        S.start()
        rs = [S.wait(t) for t in tickets]
        close(S, probs)
        assert all(r["status"] == 0 for r in rs)
        if count == 2:
            assert all(r["batch"] == 1 for r in rs) and rs[0]["round"] != rs[1]["round"]
        else:
            assert all(r["batch"] == 3 and r["round"] == 0 for r in rs)
        for r, a in zip(rs, alone):
            np.testing.assert_array_equal(np.asarray(r["coeffs"]), np.asarray(a["coeffs"]))


def test_batched_round_holds_many_scenes_and_matches_oracle():
    """One round advances six scenes of different shapes; a second request for
    a scene already in the round waits for the next round."""
    pbs = scenes(count=6, seed=23)
    S, probs = make_server(pbs, 10, start=False)
    tickets = [S.submit(k) for k in range(len(pbs))]
    extra = S.submit(2)
    S.start()
    results = [S.wait(t) for t in tickets]
    again = S.wait(extra)
    S.close()
    states = [T_state(P) for P in probs]
    close(S, probs)
    assert all(r["batch"] == 6 and r["round"] == 0 for r in results)
    assert again["round"] == 1 and again["batch"] == 1
    for k, (pb, P, r) in enumerate(zip(pbs, probs, results)):
        if k == 2:
            continue   # advanced twice
        st = states[k]
        o, tol = coef_tolerance(pb, 10)
        for key in ("xi1", "xi2"):
            assert coef_err(st[key], o[key]).max() <= tol, key
        i = r["index"]
        assert np.allclose(r["coeffs"][0], st["xi1"][i, 0:11], atol=1e-6)


def T_state(P):
    T = tj()
    return T.split_state(P.state())


def test_warm_start_continues_the_iteration():
    """Two requests on one scene (no updates) equal one 20-iteration solve: the
    state (xi, lambda) stays resident between requests."""
    T = tj()
    pb = scenes(count=1, seed=25)[0]
    S, probs = make_server([pb], 10)
    S.wait(S.submit(0))
    S.wait(S.submit(0))
    S.close()
    st = T.split_state(probs[0].state())
    close(S, probs)
    o, tol = coef_tolerance(pb, 20)
    for key in ("xi1", "xi2"):
        assert coef_err(st[key], o[key]).max() <= tol, key


def test_sequential_mode_matches_batched():
    pbs = scenes(count=3, seed=27)
    S, probs = make_server(pbs, 10, mode=1)
    seq = [S.wait(S.submit(k)) for k in range(3)]
    close(S, probs)
    S, probs = make_server(pbs, 10, mode=0)
    bat = [S.wait(t) for t in [S.submit(k) for k in range(3)]]
    close(S, probs)
    assert all(r["batch"] == 1 for r in seq)
    for a, b in zip(seq, bat):
        assert_same(a, b)


def test_advance_moves_the_start_to_the_previous_plan():
    """advance = 0.1 s: the next plan starts at the previous best plan's
    position, velocity and acceleration at t = 0.1 s (equality rows of the
    position QP hold them exactly up to FP32 rounding)."""
    pb = scenes(count=1, seed=29)[0]
    S, probs = make_server([pb], 10)
    r1 = S.wait(S.submit(0))
    r2 = S.wait(S.submit(0, advance=0.1))
    close(S, probs)
    T = pb["T"]
    tau = 0.1 / T
    from math import comb
    k = np.arange(11)
    B = np.array([comb(10, i) for i in k]) * tau ** k * (1 - tau) ** (10 - k)
    for blk in range(3):   # x, y, psi
        c1 = r1["coeffs"][blk].astype(np.float64)
        want = B @ c1
        got = float(r2["coeffs"][blk][0])   # a Bernstein curve starts at its first control point
        assert got == pytest.approx(want, abs=1e-4 * max(1.0, abs(want)))


def test_obstacle_track_update_matches_oracle():
    """A request carrying new obstacle tracks (shifted by 0.1 s along their
    velocities) solves the scene with those tracks."""
    pb = scenes(count=1, seed=31)[0]
    xo, yo = pb["xo"], pb["yo"]
    vx = (xo[:, -1] - xo[:, 0]) / pb["T"]
    vy = (yo[:, -1] - yo[:, 0]) / pb["T"]
    xo2 = (xo + 0.1 * vx[:, None]).astype(np.float32)
    yo2 = (yo + 0.1 * vy[:, None]).astype(np.float32)
    S, probs = make_server([pb], 10)
    r = S.wait(S.submit(0, xo=xo2, yo=yo2))
    S.close()
    assert r["status"] == 0
    st = T_state(probs[0])
    close(S, probs)
    pb2 = dict(pb, xo=xo2, yo=yo2)
    o, tol = coef_tolerance(pb2, 10)
    for key in ("xi1", "xi2"):
        assert coef_err(st[key], o[key]).max() <= tol, key


def test_budget_admission_and_errors():
    T = tj()
    pbs = scenes(count=2, seed=33)
    need = [T.am_scene_bytes(pb["q"], pb["m"], pb["n"], pb["B"]) for pb in pbs]
    S = T.Server(need[0] + need[1] // 2, 10)
    P0, P1 = T.Problem(pbs[0]), T.Problem(pbs[1])
    assert S.add_scene(P0, pbs[0]["init"].astype(np.float32)) == 0
    with pytest.raises(T.TrajamError) as e:
        S.add_scene(P1, pbs[1]["init"].astype(np.float32))
    assert e.value.code == T.AM_ERR_BUDGET
    assert "budget" in T.am_last_error()
    assert S.stats()["device_bytes"] == need[0]
    S.start()
    with pytest.raises(T.TrajamError) as e:
        S.add_scene(P1, pbs[1]["init"].astype(np.float32))   # after the start
    assert e.value.code == T.AM_ERR_STATE
    with pytest.raises(T.TrajamError):
        S.submit(5)          # unknown scene
    with pytest.raises(T.TrajamError):
        S.poll(12345)        # unknown ticket
    r = S.wait(S.submit(0))
    assert r["status"] == 0
    S.close()
    P0.close()
    P1.close()
