"""Grouped (uneven) batching on the GPU: many problems of different shapes in
one persistent launch, against the same problems solved one by one and
against the FP64 oracle.

A group runs the same per-tile code as a single-problem solve; only the tile
size and the order in which CTAs take tiles differ.  Every per-trajectory sum
has a fixed order, so a problem gives the same bits alone and in a group;
the general check below still compares them at twice the coefficient
tolerance (2e-4 relative), and the mixed-precision test asserts equality.

Against the oracle the mixed problems get the coefficient tolerance 1e-4,
widened where the problem itself is more sensitive: the 15 s, 150-step
horizons of the mix move the FP64 oracle by up to ~1.4e-4 after 10
iterations when its state is perturbed by FP32-sized (1e-6 relative) noise
at iteration 5, so each problem admits three times that movement
(coef_tolerance).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_13030_b300 import workload as W

from test_gpu_parity import COEF_TOL, assert_coefs, coef_err

pytestmark = pytest.mark.gpu


def tj():
    from paper_2109_13030_b300 import trajam
    return trajam


def mix(count=10, scale=1.0 / 64, seed=3):
    return W.make_uneven(seed, count=count, scale=scale)


def coef_tolerance(pb, iters, eps=1e-6, reps=2, seed=23):
    """COEF_TOL, or three times the oracle's own coefficient movement under
    eps-relative noise injected half way, whichever is larger."""
    clean = O.solve(pb, iters)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(reps):
        st = O.solve(pb, iters // 2)
        for k in ("xi1", "xi2", "lam", "lampsi"):
            st[k] = st[k] * (1 + eps * rng.standard_normal(st[k].shape))
        st = O.solve(pb, iters - iters // 2, state=st)
        for k in ("xi1", "xi2"):
            worst = max(worst, coef_err(st[k], clean[k]).max())
    return clean, max(COEF_TOL, 3 * worst)


def check_oracle(pb, g, iters=10):
    o, tol = coef_tolerance(pb, iters)
    assert_coefs(g, o, tol=tol)


def split_all(P):
    T = tj()
    out = T.split_state(P.state())
    out.update({k: v.astype(np.float64) for k, v in P.results().items()})
    return out


def solve_alone(pb, iters):
    T = tj()
    P = T.Problem(pb)
    P.solve(pb["init"].astype(np.float32), iters)
    out = split_all(P)
    P.close()
    return out


def group_solve(pbs, iters, threads=0, graph=True, stream=None, reps=1):
    T = tj()
    probs = [T.Problem(pb).init_state(pb["init"].astype(np.float32), stream=stream) for pb in pbs]
    G = T.Group(probs, threads=threads, graph=graph)
    for _ in range(reps):
        G.solve(iters, stream=stream)
    outs = [split_all(P) for P in probs]
    stats = G.stats()
    G.close()
    for P in probs:
        P.close()
    return outs, stats


def assert_close(a, b, tol):
    for key in ("xi1", "xi2"):
        e = coef_err(a[key], b[key])
        assert e.max() <= tol, (key, e.max())
    for key in ("cost", "res", "mind"):
        assert np.allclose(a[key], b[key], rtol=1e-3, atol=5e-4), key


def test_mixed_precision_group():
    """The uneven-batching form with BF16 contractions: a group holding FP32 and
    BF16 problems (each its own variant kernel in one launch) gives every
    problem the same bits as a lone solve in its precision, and each BF16
    problem stays within the reduced form's stated bound of the FP64 oracle
    after 10 iterations (30 u on coefficients, u = 2^-8)."""
    T = tj()
    pbs = mix(count=6, seed=5)
    precs = [T.AM_BF16 if i % 2 == 0 else T.AM_FP32 for i in range(len(pbs))]
    probs = [T.Problem(pb, precision=pr).init_state(pb["init"].astype(np.float32)) for pb, pr in zip(pbs, precs)]
    G = T.Group(probs)
    G.solve(10)
    outs = [split_all(P) for P in probs]
    G.close()
    for P in probs:
        P.close()
    for pb, pr, g in zip(pbs, precs, outs):
        P = T.Problem(pb, precision=pr)
        P.solve(pb["init"].astype(np.float32), 10)
        alone = split_all(P)
        P.close()
        for key in ("xi1", "xi2", "cost", "res"):
            np.testing.assert_array_equal(g[key], alone[key], err_msg=key)
        if pr == T.AM_BF16:
            o = O.solve(pb, 10)
            for key in ("xi1", "xi2"):
                e = coef_err(g[key], o[key])
                assert np.all(np.isfinite(e)) and e.max() <= 30 * 2.0 ** -8, (key, e.max())
        else:
            check_oracle(pb, g)


def test_group_matches_alone_and_oracle():
    """Ten mixed problems (q in {50, 100, 150}, m 2..4, n 2..32, B 2..32)."""
    pbs = mix()
    outs, (launches, items) = group_solve(pbs, 10)
    assert launches == len({pb["m"] for pb in pbs})   # one kernel per circle count present
    assert items >= len(pbs)
    for pb, g in zip(pbs, outs):
        alone = solve_alone(pb, 10)
        assert_close(g, alone, 2 * COEF_TOL)
        check_oracle(pb, g)


@pytest.mark.parametrize("threads", [128, 256])
def test_group_block_sizes(threads):
    """Smaller blocks give smaller tiles (more work items); results agree."""
    pbs = mix(count=6, seed=5)
    outs, _ = group_solve(pbs, 10, threads=threads)
    for pb, g in zip(pbs, outs):
        check_oracle(pb, g)


def test_group_graph_replay_on_stream():
    """On a side stream the solve is captured once and replayed: two 5-iteration
    solves match one 10-iteration solve of the oracle."""
    import torch
    s = torch.cuda.Stream()
    pbs = mix(count=6, seed=7)
    outs, (launches, _) = group_solve(pbs, 5, stream=s, reps=2)
    s.synchronize()
    assert launches == 2 * len({pb["m"] for pb in pbs})
    for pb, g in zip(pbs, outs):
        check_oracle(pb, g)


def test_group_without_graph_matches():
    pbs = mix(count=4, seed=9)
    a, _ = group_solve(pbs, 10, graph=False)
    b, _ = group_solve(pbs, 10, graph=True)
    for x, y in zip(a, b):
        assert_close(x, y, 2 * COEF_TOL)


def test_group_with_single_trajectory_problems():
    """Problems of one trajectory each (one ragged tile apiece)."""
    pbs = mix(count=8, scale=1e-6, seed=11)
    assert all(pb["B"] == 1 for pb in pbs)
    outs, (_, items) = group_solve(pbs, 10)
    assert items == 8
    for pb, g in zip(pbs, outs):
        check_oracle(pb, g)


def test_group_autotune_restores_state():
    T = tj()
    pbs = mix(count=5, seed=13)
    probs = [T.Problem(pb).init_state(pb["init"].astype(np.float32)) for pb in pbs]
    before = [P.state() for P in probs]
    G = T.Group(probs)
    threads, ms = G.autotune(10)
    assert 128 <= threads <= 384 and threads % 32 == 0 and ms > 0
    for P, s in zip(probs, before):
        assert np.array_equal(P.state(), s)
    G.solve(10)
    for pb, P in zip(pbs, probs):
        check_oracle(pb, split_all(P))
    G.close()
    for P in probs:
        P.close()


def test_group_autotune_cache(tmp_path):
    """A stored choice is reused for a group of the same key without timing."""
    T = tj()
    pbs = mix(count=3, seed=19)
    cache = str(tmp_path / "tune.json")
    probs = [T.Problem(pb).init_state(pb["init"].astype(np.float32)) for pb in pbs]
    G = T.Group(probs)
    threads, ms = G.autotune(10, cache=cache, sms=148)
    G.close()
    from paper_2109_13030_b300 import tune_cache
    k = tune_cache.key([(pb["q"], pb["m"], pb["n"], pb["B"]) for pb in pbs], 0, 148, 10)
    assert tune_cache.lookup(cache, k) == (threads, ms, 0)  # no warp-pair problems: no slot cap
    tune_cache.store(cache, k, 256, 0.5)
    G = T.Group(probs)
    assert G.autotune(10, cache=cache, sms=148) == (256, 0.5)
    G.solve(10)
    for pb, P in zip(pbs, probs):
        check_oracle(pb, split_all(P))
    G.close()
    for P in probs:
        P.close()


def test_group_best_and_results_per_problem():
    pbs = mix(count=3, seed=17)
    T = tj()
    probs = [T.Problem(pb).init_state(pb["init"].astype(np.float32)) for pb in pbs]
    G = T.Group(probs).solve(10)
    for pb, P in zip(pbs, probs):
        r = P.results()
        b = P.best()
        o = O.solve(pb, 10)
        ok = np.where(r["mind"] >= 0.99)[0]
        cand = ok if len(ok) else np.arange(pb["B"])
        assert b["index"] in cand
        assert abs(b["cost"] - r["cost"][b["index"]]) <= 1e-6 * max(1.0, abs(b["cost"]))
        assert np.allclose(r["cost"], o["cost"], rtol=1e-3)
    G.close()
    for P in probs:
        P.close()


def test_group_errors():
    T = tj()
    pb = mix(count=1, seed=19)[0]
    P = T.Problem(pb)
    G = T.Group([P])
    with pytest.raises(T.TrajamError) as e:
        G.solve(10)   # no state yet
    assert e.value.code == T.AM_ERR_STATE
    with pytest.raises(T.TrajamError):
        T.am_group_set_option(G.g, T.AM_GOPT_THREADS, 100)
    with pytest.raises(T.TrajamError):
        T.am_group_set_option(G.g, 99, 0)
    with pytest.raises(T.TrajamError):
        T.am_group_solve(G.g, 0)
    G.close()
    P.close()
