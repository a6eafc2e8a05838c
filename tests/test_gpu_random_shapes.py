"""Randomized shapes against the FP64 oracle: seeded draws of the horizon
(4..199 steps), circle count (1..4), obstacle count (0..39) and batch size
(1..301) for the fused and the plain kernels, and random mixes of problems in
grouped launches with random block sizes.  Sampled trajectories after 10
iterations, with the mixed-problem tolerance (the larger of 1e-4 and three
times the oracle's own movement under FP32-sized noise)."""
import numpy as np
import pytest

from paper_2109_13030_b300 import workload as W

from test_gpu_group import coef_tolerance
from test_gpu_parity import coef_err

pytestmark = pytest.mark.gpu


def tj():
    from paper_2109_13030_b300 import trajam
    return trajam


def draw_shape(rng):
    q = int(rng.integers(4, 200))
    m = int(rng.integers(1, 5))
    n = int(rng.integers(0, 40))
    B = int(rng.choice([1, 2, 7, 8, 9, 33, 150, 301]))
    pb = W.make_shape(int(rng.integers(0, 10 ** 6)), B=B, q=q, n=max(n, 1), m=m)
    if n == 0:
        pb = W.with_obstacles_removed(pb, v_max=2.0, a_max=2.0)
    return pb


def check(pb, state, rng, k=6):
    T = tj()
    st = T.split_state(state)
    idx = np.unique(rng.choice(pb["B"], size=min(pb["B"], k), replace=False))
    o, tol = coef_tolerance(dict(pb, init=pb["init"][idx], B=len(idx)), 10)
    for key in ("xi1", "xi2"):
        e = coef_err(st[key][idx], o[key])
        assert e.max() <= tol, (pb["q"], pb["m"], pb["n"], pb["B"], key, e.max(), tol)


@pytest.mark.parametrize("seed", range(12))
def test_random_shape_both_kernels(seed):
    T = tj()
    rng = np.random.default_rng(1000 + seed)
    pb = draw_shape(rng)
    for kernel in (T.AM_KERNEL_FUSED, T.AM_KERNEL_PLAIN):
        P = T.Problem(pb, kernel=kernel)
        P.solve(pb["init"].astype(np.float32), 10)
        state = P.state()
        P.close()
        check(pb, state, np.random.default_rng(seed))


@pytest.mark.parametrize("seed", range(3))
def test_random_group_mix(seed):
    T = tj()
    rng = np.random.default_rng(2000 + seed)
    pbs = []
    for _ in range(int(rng.integers(2, 9))):
        q = int(rng.choice([20, 50, 100, 150]))
        pbs.append(W.make_shape(int(rng.integers(0, 10 ** 6)), B=int(rng.choice([1, 5, 64, 300])), q=q,
                                n=int(rng.integers(1, 33)), m=int(rng.integers(1, 5))))
    probs = [T.Problem(pb).init_state(pb["init"].astype(np.float32)) for pb in pbs]
    G = T.Group(probs, threads=int(rng.choice([0, 128, 256, 384])))
    G.solve(10)
    for pb, P in zip(pbs, probs):
        check(pb, P.state(), rng, k=4)
    G.close()
    for P in probs:
        P.close()
