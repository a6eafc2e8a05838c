"""The large-batch kernel (AM_KERNEL_LARGE: tiles of 128 trajectories, the
position step, trajectory values, P^T delta and R on tcgen05 tensor cores in
three TF32 products) against the FP64 oracle, with the tolerances of the
small-tile kernel (test_gpu_parity): coefficients within 1e-4 relative after
10 iterations, cost and residual within 1e-3 after 100.  Shapes cover a
single partial tile, two tiles, a ragged last tile, odd and maximal horizons,
more than 32 obstacles (two near-obstacle words), one circle and no
obstacles; the batch of 16384 is checked on sampled trajectories spread over
all tiles."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_13030_b300 import workload as W

from test_gpu_parity import COEF_TOL, assert_coefs, assert_final, coef_err, noisy_oracle_spread, sub_problem

pytestmark = pytest.mark.gpu


def tj():
    from paper_2109_13030_b300 import trajam
    return trajam


def large_solve(pb, iters, init=None, **flags):
    T = tj()
    P = T.Problem(pb, kernel=T.AM_KERNEL_LARGE, **flags)
    init = pb["init"] if init is None else init
    P.solve(init.astype(np.float32), iters)
    out = T.split_state(P.state())
    out.update({k: v.astype(np.float64) for k, v in P.results().items()})
    out["best"] = P.best()
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


def test_tiny_partial_tile():
    """32 trajectories: one partial tile (rows 32..127 idle)."""
    pb = W.make_problem("tiny", 0)
    g = large_solve(pb, 10)
    assert_coefs(g, O.solve(pb, 10))


def test_paper_shape_two_tiles_against_oracle_and_small_tiles():
    pb = W.make_problem("paper", 1, B=256)
    g = large_solve(pb, 10)
    assert_coefs(g, O.solve(pb, 10))
    s = small_solve(pb, 10)
    for key in ("xi1", "xi2"):
        e = coef_err(g[key], s[key])
        assert e.max() <= 2 * COEF_TOL, (key, e.max())


@pytest.mark.parametrize("B", [1, 129, 200])
def test_ragged_batches(B):
    pb = W.make_problem("paper", 3, B=B)
    g = large_solve(pb, 10)
    assert_coefs(g, O.solve(pb, 10))


def test_single_iteration():
    """One iteration (the first sweep, one position and heading step, the
    last sweep's sums from the given heading) to 1e-5."""
    pb = W.make_problem("paper", 4, B=16)
    g = large_solve(pb, 1)
    o = O.solve(pb, 1)
    assert_coefs(g, o, tol=1e-5)
    assert_final(g, o, label="large, 1 iteration")


def test_paper_shape_after_100_plain_bound():
    """A full tile of paper-shaped trajectories after 100 iterations: every
    trajectory within the plain 1e-3 bound on cost and residual."""
    pb = W.make_problem("paper", 0, B=128)
    g = large_solve(pb, 100)
    o, spread = noisy_oracle_spread(pb, 100)
    counts = assert_final(g, o, spread=spread, label="large paper B=128")
    for name, (plain, allowed, n) in counts.items():
        assert plain == n, (name, plain, allowed)


def test_batch_16384_sampled():
    """The large-batch configuration: 16384 paper-shaped trajectories (128
    tiles), the oracle recomputing trajectories at tile edges and at random
    over the batch, after 10 and after 100 iterations."""
    pb = W.make_problem("paper", 2, B=16384)
    rng = np.random.default_rng(16384)
    idx = np.unique(np.concatenate([[0, 1, 127, 128, 129, 8191, 8192, 16255, 16256, 16383],
                                    rng.choice(16384, 22, replace=False)]))
    g10 = large_solve(pb, 10)
    assert_coefs(g10, O.solve(sub_problem(pb, idx), 10), idx)
    g100 = large_solve(pb, 100)
    o100, spread = noisy_oracle_spread(sub_problem(pb, idx), 100)
    counts = assert_final(g100, o100, idx, spread=spread, label="large B=16384")
    for name, (plain, allowed, n) in counts.items():
        assert plain == n, (name, plain, allowed)
    b = g100["best"]
    ok = np.nonzero(g100["mind"] >= 0.99)[0]
    cand = ok if len(ok) else np.arange(pb["B"])
    assert b["index"] in cand
    assert b["cost"] <= g100["cost"][cand].min() * (1 + 1e-6) + 1e-6


@pytest.mark.parametrize("q,m,n", [(50, 1, 0), (51, 4, 3), (128, 2, 8), (64, 3, 40), (17, 2, 2)])
def test_shapes(q, m, n):
    """Odd horizon (a half pair at the end), the longest horizon (q = 128:
    eight full chunks), more than 32 obstacles, a short horizon (two chunks,
    one partial), one circle without obstacles."""
    pb = W.make_shape(q * 7 + m + n, 9, q, n, m)
    g = large_solve(pb, 10)
    assert_coefs(g, O.solve(pb, 10))


@pytest.mark.parametrize("flags", [dict(psi_dual_sign=1), dict(cs_boundary=0)])
def test_reading_flags(flags):
    pb = W.make_problem("tiny", 2)
    g = large_solve(pb, 10, **flags)
    assert_coefs(g, O.solve(pb, 10, **flags))


def test_turning_heading():
    pb = W.make_problem("tiny", 3)
    pb["psi_bc"] = np.array([0.0, 0.2, 0.0, 2.5, -0.1, 0.0])
    g = large_solve(pb, 10)
    assert_coefs(g, O.solve(pb, 10))


def test_no_obstacles_closed_form():
    """Check (iii) through the large-batch kernel: no obstacles, inactive
    bounds -> the minimum-smoothness polynomial."""
    pb = W.with_obstacles_removed(W.make_problem("paper", 0, B=8))
    g = large_solve(pb, 300)
    o = O.solve(pb, 300)
    P, _, _ = O.bernstein(10, pb["q"], pb["T"])
    np.testing.assert_allclose(g["xi1"][:, 0:11] @ P.T, o["xi1"][:, 0:11] @ P.T, atol=1e-4)
    np.testing.assert_allclose(g["xi1"][:, 22:33] @ P.T, o["xi1"][:, 22:33] @ P.T, atol=1e-4)


def test_warm_start_split():
    """40 iterations, then 60 more from the resident state, against 100."""
    T = tj()
    pb = W.make_problem("paper", 5, B=200)
    P = T.Problem(pb, kernel=T.AM_KERNEL_LARGE)
    P.solve(pb["init"].astype(np.float32), 40)
    P.solve(None, 60)
    a = T.split_state(P.state())
    P.close()
    b = large_solve(pb, 100)
    for key in ("xi1", "xi2"):
        assert coef_err(a[key], b[key]).max() <= 1e-3, key


def test_unsupported_forms_are_refused():
    T = tj()
    pb = W.make_problem("tiny", 0, B=8)
    init = pb["init"].astype(np.float32)
    for kw, hist in ((dict(precision=T.AM_TF32), False), (dict(alpha_mode=1), False), ({}, True)):
        P = T.Problem(pb, kernel=T.AM_KERNEL_LARGE, **kw)
        with pytest.raises(T.TrajamError) as e:
            P.solve(init, 5, history=hist)
        assert e.value.code == T.AM_ERR_ARG
        P.close()
    long = W.make_shape(1, 4, 150, 4, 2)
    P = T.Problem(long, kernel=T.AM_KERNEL_LARGE)
    with pytest.raises(T.TrajamError) as e:
        P.solve(long["init"].astype(np.float32), 5)
    assert e.value.code == T.AM_ERR_ARG and "q <= 128" in str(e.value)
    P.close()


def test_bounded_wait_runs_out_and_context_recovers():
    """The staging wait of the large-batch kernel is bounded too: with the
    diagnostic stall it gives up, frees its tensor memory and reports."""
    T = tj()
    pb = W.make_problem("tiny", 0, B=8)
    P = T.Problem(pb, kernel=T.AM_KERNEL_LARGE)
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
