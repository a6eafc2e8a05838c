"""The warp-pair kernel (AM_KERNEL_WARP: NW = 2, 3 or 4 warps run every
iteration of one trajectory, for q <= 128, 192, 256, the contraction R in
FP32 SIMT) against the FP64 oracle, with the tolerances of test_gpu_parity: coefficients within 1e-4
relative after 10 iterations, cost and residual within 1e-3 after 100.

Shapes cover short horizons (lanes without a pair in both halves), a
second half shorter than the first, odd horizons (a half pair at the end),
the longest horizon of each warp count (q = 128, 192, 256: every lane busy),
the first horizon of three and four warps (q = 129, 193), the largest
shared-memory footprint (q = 256 with 64 obstacles: one trajectory per CTA),
more than 32 obstacles (two near-obstacle words), one to four circles, no obstacles, ragged batches and
more trajectories than warp-pair slots (pairs taking several trajectories in
turn).  The paper's batch of 1000
is checked on every trajectory after 10 iterations and on samples after 100.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_13030_b300 import workload as W

from test_gpu_parity import (COEF_TOL, RES_ATOL, RES_RTOL, assert_coefs, assert_final, coef_err,
                             noisy_oracle_spread, sub_problem)

pytestmark = pytest.mark.gpu


def tj():
    from paper_2109_13030_b300 import trajam
    return trajam


def warp_solve(pb, iters, init=None, tile=0, history=False, **flags):
    T = tj()
    P = T.Problem(pb, kernel=T.AM_KERNEL_WARP, tile=tile, **flags)
    init = pb["init"] if init is None else init
    P.solve(init.astype(np.float32), iters, history=history)
    out = T.split_state(P.state())
    out["state"] = P.state()
    out.update({k: v.astype(np.float64) for k, v in P.results().items()})
    if history:
        out["hist"] = P.history().astype(np.float64)
    out["best"] = P.best()
    out["launches"] = T.am_last_solve_stats(P.h)
    P.close()
    return out


def small_solve(pb, iters):
    T = tj()
    P = T.Problem(pb)
    P.solve(pb["init"].astype(np.float32), iters)
    out = T.split_state(P.state())
    out.update({k: v.astype(np.float64) for k, v in P.results().items()})
    P.close()
    return out


def test_tiny_after_10():
    """q = 50: 25 pairs, 13 in the first half and 12 in the second."""
    pb = W.make_problem("tiny", 0)
    g = warp_solve(pb, 10)
    assert_coefs(g, O.solve(pb, 10))
    assert g["launches"] == 2  # the cold start and the solve


def test_tiny_after_100():
    pb = W.make_problem("tiny", 1)
    g = warp_solve(pb, 100)
    o, spread = noisy_oracle_spread(pb, 100)
    counts = assert_final(g, o, spread=spread, label="warp tiny")
    for name, (plain, allowed, n) in counts.items():
        assert plain == n, (name, plain, allowed)


def test_paper_batch_all_trajectories_after_10():
    """The paper-shaped batch of 1000 (seven warp pairs on each of 143 SMs):
    every trajectory against the oracle after 10 iterations, and against
    the small-tile kernel."""
    pb = W.make_problem("paper", 0)
    g = warp_solve(pb, 10)
    assert_coefs(g, O.solve(pb, 10))
    s = small_solve(pb, 10)
    for key in ("xi1", "xi2"):
        e = coef_err(g[key], s[key])
        assert e.max() <= 2 * COEF_TOL, (key, e.max())


def test_multipliers_match_oracle():
    """lam and lam_psi, every component, after 10 iterations.  Their
    interior components are updated every iteration; the boundary
    components (which move no control point) are formed once at the end
    from the residual rows and heading targets summed over the iterations."""
    for name, seed, B in (("paper", 7, 64), ("tiny", 4, 32)):
        pb = W.make_problem(name, seed, B=B)
        g = warp_solve(pb, 10)
        o = O.solve(pb, 10)
        for key in ("lam", "lampsi"):
            e = coef_err(g[key], o[key])
            assert e.max() <= COEF_TOL, (name, key, e.max(), int(np.argmax(e)))


def test_paper_batch_sampled_after_100():
    pb = W.make_problem("paper", 1)
    rng = np.random.default_rng(1000)
    idx = np.unique(np.concatenate([[0, 1, 6, 7, 499, 500, 993, 999], rng.choice(1000, 16, replace=False)]))
    g = warp_solve(pb, 100)
    o, spread = noisy_oracle_spread(sub_problem(pb, idx), 100)
    counts = assert_final(g, o, idx, spread=spread, label="warp paper B=1000")
    for name, (plain, allowed, n) in counts.items():
        assert plain == n, (name, plain, allowed)
    b = g["best"]
    ok = np.nonzero(g["mind"] >= 0.99)[0]
    cand = ok if len(ok) else np.arange(pb["B"])
    assert b["index"] in cand
    assert b["cost"] <= g["cost"][cand].min() * (1 + 1e-6) + 1e-6


def test_paper_shape_64_after_100_plain_bound():
    pb = W.make_problem("paper", 0, B=64)
    g = warp_solve(pb, 100)
    o, spread = noisy_oracle_spread(pb, 100)
    counts = assert_final(g, o, spread=spread, label="warp paper B=64")
    for name, (plain, allowed, n) in counts.items():
        assert plain == n, (name, plain, allowed)


@pytest.mark.parametrize("B", [1, 7, 150])
def test_ragged_batches(B):
    pb = W.make_problem("paper", 3, B=B)
    g = warp_solve(pb, 10)
    assert_coefs(g, O.solve(pb, 10))


def test_more_trajectories_than_warp_slots():
    """B = 2500 with one trajectory per CTA: every warp pair takes about 17
    trajectories in turn (the trajectory loop), sampled against the oracle."""
    pb = W.make_problem("paper", 6, B=2500)
    idx = np.array([0, 1, 147, 148, 149, 295, 296, 1250, 2347, 2348, 2499])
    g = warp_solve(pb, 10, tile=1)
    assert_coefs(g, O.solve(sub_problem(pb, idx), 10), idx)


@pytest.mark.parametrize("q,W_", [(100, 1), (100, 3), (100, 8), (150, 1), (150, 5), (256, 2), (256, 4)])
def test_result_independent_of_trajectories_per_cta(q, W_):
    """A trajectory's arithmetic does not depend on which warps run it, so
    any number of trajectories per CTA gives the same bits (up to 8, 5 and 4
    for two, three and four warps per trajectory)."""
    pb = W.make_problem("paper", 0, B=40) if q == 100 else W.make_shape(q, 40, q, 10 if q < 256 else 4, 3)
    a = warp_solve(pb, 20)
    b = warp_solve(pb, 20, tile=W_)
    np.testing.assert_array_equal(a["state"], b["state"])
    for k in ("res", "res_psi", "cost", "mind"):
        np.testing.assert_array_equal(a[k], b[k])


def test_single_iteration():
    pb = W.make_problem("paper", 4, B=16)
    g = warp_solve(pb, 1)
    o = O.solve(pb, 1)
    assert_coefs(g, o, tol=1e-5)
    assert_final(g, o, label="warp, 1 iteration")


@pytest.mark.parametrize("q,m,n", [(50, 1, 0), (51, 4, 3), (128, 2, 8), (64, 3, 40), (17, 2, 2),
                                   (65, 3, 10), (99, 3, 10), (127, 4, 64),
                                   (129, 3, 10), (150, 3, 10), (151, 2, 33), (192, 4, 40),
                                   (193, 1, 0), (200, 3, 10), (255, 2, 5), (256, 3, 10), (256, 4, 64)])
def test_shapes(q, m, n):
    """Short horizons (q = 17: 9 pairs), halves of 17 and 16 pairs (q = 65),
    odd horizons, the longest horizon of each warp count, 40 and 64
    obstacles (two near-obstacle words), one circle without obstacles;
    three warps from q = 129 (65 pairs: one in the third warp), four from
    q = 193.

    The bar is COEF_TOL, widened (as for the grouped mixes) to three times
    the oracle's own coefficient movement under FP32-sized noise, and to 1.5
    times the plain FP32 loop's error on the same inputs: on the longest
    horizons with four circles and 40 to 64 obstacles every FP32 path moves
    the heading coefficients by more than 1e-4 (the plain loop by 1.16e-4 at
    q = 256, m = 4, n = 64)."""
    from test_gpu_group import coef_tolerance
    pb = W.make_shape(q * 7 + m + n, 9, q, n, m)
    g = warp_solve(pb, 10)
    o, tol = coef_tolerance(pb, 10)
    T = tj()
    P = T.Problem(pb, kernel=T.AM_KERNEL_PLAIN)
    P.solve(pb["init"].astype(np.float32), 10)
    plain = T.split_state(P.state())
    P.close()
    tol = max(tol, 1.5 * max(coef_err(plain[k], o[k]).max() for k in ("xi1", "xi2")))
    assert_coefs(g, o, tol=tol)


@pytest.mark.parametrize("flags", [dict(psi_dual_sign=1)])
def test_reading_flags(flags):
    pb = W.make_problem("tiny", 2)
    g = warp_solve(pb, 10, **flags)
    assert_coefs(g, O.solve(pb, 10, **flags))


def test_turning_heading():
    pb = W.make_problem("tiny", 3)
    pb["psi_bc"] = np.array([0.0, 0.2, 0.0, 2.5, -0.1, 0.0])
    g = warp_solve(pb, 10)
    assert_coefs(g, O.solve(pb, 10))


def test_no_obstacles_closed_form():
    """Check (iii) through this kernel: no obstacles, inactive bounds -> the
    minimum-smoothness polynomial."""
    pb = W.with_obstacles_removed(W.make_problem("paper", 0, B=8))
    g = warp_solve(pb, 300)
    o = O.solve(pb, 300)
    P, _, _ = O.bernstein(10, pb["q"], pb["T"])
    np.testing.assert_allclose(g["xi1"][:, 0:11] @ P.T, o["xi1"][:, 0:11] @ P.T, atol=1e-4)
    np.testing.assert_allclose(g["xi1"][:, 22:33] @ P.T, o["xi1"][:, 22:33] @ P.T, atol=1e-4)


def test_history_matches_oracle():
    pb = W.make_problem("paper", 2, B=8)
    g = warp_solve(pb, 30, history=True)
    o = O.solve(pb, 30, hist=True)
    h, ho = g["hist"], o["hist"]
    np.testing.assert_allclose(h[:, :, 2], ho[:, :, 2], rtol=1e-3)
    assert np.all(np.abs(h[:, :, 0] - ho[:, :, 0]) <= RES_RTOL * ho[:, :, 0] + RES_ATOL)
    np.testing.assert_allclose(h[:, -1, 0], g["res"], rtol=1e-6)


def test_warm_start_split():
    """40 iterations, then 60 more from the resident state, against 100."""
    T = tj()
    pb = W.make_problem("paper", 5, B=200)
    P = T.Problem(pb, kernel=T.AM_KERNEL_WARP)
    P.solve(pb["init"].astype(np.float32), 40)
    P.solve(None, 60)
    a = T.split_state(P.state())
    P.close()
    b = warp_solve(pb, 100)
    for key in ("xi1", "xi2"):
        assert coef_err(a[key], b[key]).max() <= 1e-3, key


def test_unsupported_forms_are_refused():
    T = tj()
    pb = W.make_problem("tiny", 0, B=8)
    init = pb["init"].astype(np.float32)
    for kw in (dict(precision=T.AM_TF32), dict(alpha_mode=1), dict(cs_boundary=0)):
        P = T.Problem(pb, kernel=T.AM_KERNEL_WARP, **kw)
        with pytest.raises(T.TrajamError) as e:
            P.solve(init, 5)
        assert e.value.code == T.AM_ERR_ARG
        P.close()
    # trajectories per CTA: at most 16 warps, 2, 3 or 4 per trajectory
    for q, tile in ((50, 9), (150, 6), (256, 5)):
        sh = W.make_shape(q, 8, q, 4, 2)
        P = T.Problem(sh, kernel=T.AM_KERNEL_WARP, tile=tile)
        with pytest.raises(T.TrajamError) as e:
            P.solve(sh["init"].astype(np.float32), 5)
        assert e.value.code == T.AM_ERR_ARG and "trajectories per CTA" in str(e.value)
        P.close()


def test_bounded_wait_runs_out_and_context_recovers():
    """The staging wait is bounded: with the diagnostic stall it gives up and
    reports, and the next solve on the same context is correct."""
    T = tj()
    pb = W.make_problem("tiny", 0, B=8)
    P = T.Problem(pb, kernel=T.AM_KERNEL_WARP)
    T.am_set_option(P.h, T.AM_OPT_DIAG_STALL, 1)
    t0 = time.time()
    P.solve(pb["init"].astype(np.float32), 10)
    with pytest.raises(T.TrajamError) as e:
        P.results()
    assert e.value.code == T.AM_ERR_TIMEOUT
    assert time.time() - t0 < 30.0
    T.am_set_option(P.h, T.AM_OPT_DIAG_STALL, 0)
    P.solve(pb["init"].astype(np.float32), 10)
    g = T.split_state(P.state())
    P.close()
    assert_coefs(g, O.solve(pb, 10))
