"""Failure detection without a GPU fault.

* Host inputs with a non-finite value are refused with AM_ERR_ARG.
* The fused kernel's only device-side wait (the constant copy) is bounded by
  about a second of the global timer: a diagnostic option stages without the
  copy, so nothing completes the wait; the kernel records the failure and
  returns, the getters report AM_ERR_TIMEOUT, and the same handle solves
  correctly afterwards (the context stays usable).
* A batch whose trajectories are all non-finite (device inputs are not
  scanned) makes the best selection report AM_ERR_NAN.
* A server destroyed with requests still queued stops cleanly.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_13030_b300 import workload as W

from test_gpu_parity import assert_coefs

pytestmark = pytest.mark.gpu


def tj():
    from paper_2109_13030_b300 import trajam
    return trajam


def test_non_finite_host_inputs_refused():
    T = tj()
    pb = W.make_problem("tiny", 0, B=4)
    P = T.Problem(pb)
    xo = pb["xo"].astype(np.float32).copy()
    xo[1, 3] = np.nan
    with pytest.raises(T.TrajamError) as e:
        T.am_set_obstacles(P.h, pb["n"], xo, pb["yo"].astype(np.float32), pb["ao"].astype(np.float32),
                           pb["bo"].astype(np.float32))
    assert e.value.code == T.AM_ERR_ARG and "track" in str(e.value)
    init = pb["init"].astype(np.float32).copy()
    init[2, 0, 5] = np.inf
    with pytest.raises(T.TrajamError) as e:
        P.solve(init, 5)
    assert e.value.code == T.AM_ERR_ARG
    P.solve(pb["init"].astype(np.float32), 5)   # the handle is unharmed
    # a refused input for a larger batch leaves the state of the last solve
    # as it was: its warm continuation equals an undisturbed one
    big = np.tile(pb["init"].astype(np.float32), (3, 1, 1))
    big[7, 1, 4] = np.nan
    with pytest.raises(T.TrajamError) as e:
        T.am_solve_batch(P.h, 12, big, None, 5)
    assert e.value.code == T.AM_ERR_ARG
    P.solve(None, 5)
    Q = T.Problem(pb)
    Q.solve(pb["init"].astype(np.float32), 5)
    Q.solve(None, 5)
    np.testing.assert_array_equal(P.state(), Q.state())
    Q.close()
    P.close()


def test_bounded_device_wait_runs_out_and_context_recovers():
    T = tj()
    pb = W.make_problem("tiny", 0, B=8)
    P = T.Problem(pb)
    T.am_set_option(P.h, T.AM_OPT_DIAG_STALL, 1)
    t0 = time.time()
    P.solve(pb["init"].astype(np.float32), 10)
    with pytest.raises(T.TrajamError) as e:
        P.results()
    took = time.time() - t0
    assert e.value.code == T.AM_ERR_TIMEOUT
    assert took < 30.0
    T.am_set_option(P.h, T.AM_OPT_DIAG_STALL, 0)
    P.solve(pb["init"].astype(np.float32), 10)
    g = T.split_state(P.state())
    P.close()
    assert_coefs(g, O.solve(pb, 10))


def test_group_reports_the_stalled_wait():
    T = tj()
    pbs = W.make_uneven(41, count=2, scale=1.0 / 128)
    probs = [T.Problem(pb).init_state(pb["init"].astype(np.float32)) for pb in pbs]
    T.am_set_option(probs[1].h, T.AM_OPT_DIAG_STALL, 1)
    G = T.Group(probs, graph=False)
    G.solve(5)
    with pytest.raises(T.TrajamError) as e:
        T.am_group_get_best(G.g, 2)
    assert e.value.code == T.AM_ERR_TIMEOUT
    G.close()
    for P in probs:
        P.close()


def test_all_non_finite_batch_reports_nan():
    import torch
    T = tj()
    pb = W.make_problem("tiny", 0, B=4)
    P = T.Problem(pb)
    init = torch.full((4, 3, 11), float("nan"), device="cuda")
    P.solve(init, 3)
    with pytest.raises(T.TrajamError) as e:
        P.best()
    assert e.value.code == T.AM_ERR_NAN
    # one finite trajectory among non-finite ones is still selected
    good = torch.tensor(pb["init"][:1], dtype=torch.float32, device="cuda")
    init[0] = good[0]
    P.solve(init, 3)
    b = P.best()
    assert b["index"] == 0 and np.isfinite(b["cost"])
    P.close()


def test_server_destroyed_with_requests_queued():
    T = tj()
    pbs = W.make_uneven(43, count=3, scale=1.0 / 64)
    S = T.Server(1 << 30, 30)
    probs = []
    for pb in pbs:
        P = T.Problem(pb)
        S.add_scene(P, pb["init"].astype(np.float32))
        probs.append(P)
    tickets = [S.submit(k % 3) for k in range(60)]   # queued before the start
    S.start()
    first = S.wait(tickets[0])
    assert first["status"] == 0
    S.close()                                           # many still queued or in flight
    for P in probs:
        P.close()
