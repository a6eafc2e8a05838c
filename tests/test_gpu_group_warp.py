"""Grouped and served solves on the warp-pair kernels.

A problem whose handle selects AM_KERNEL_AUTO (or AM_KERNEL_WARP) runs in a
group on the warp-pair group kernels when its form and shape fit them (FP32,
default alpha form; two, three or four warps per trajectory for q <= 128,
192, 256), every other problem on the small-tile group kernels, all in one
launch.  A trajectory's arithmetic on the warp-pair
kernels does not depend on which CTA slot runs it, so each problem gives
the same bits in the group as alone with the kernel AM_KERNEL_AUTO picks
for it; the results also match the FP64 oracle (with the mix's widened
coefficient tolerance, see test_gpu_group).  A server whose scenes select
AM_KERNEL_AUTO serves a request alone and in a mixed round with the same
bits.
"""
import numpy as np
import pytest

from paper_2109_13030_b300 import workload as W

from test_gpu_group import check_oracle, mix, split_all

pytestmark = pytest.mark.gpu


def tj():
    from paper_2109_13030_b300 import trajam
    return trajam


def alone(pb, iters, kernel):
    T = tj()
    P = T.Problem(pb, kernel=kernel)
    P.solve(pb["init"].astype(np.float32), iters)
    out = split_all(P)
    out["state"] = P.state()
    P.close()
    return out


def group(pbs, iters, kernel, reps=1, stream=None):
    T = tj()
    probs = [T.Problem(pb, kernel=kernel).init_state(pb["init"].astype(np.float32), stream=stream) for pb in pbs]
    G = T.Group(probs)
    for _ in range(reps):
        G.solve(iters, stream=stream)
    outs = []
    for P in probs:
        o = split_all(P)
        o["state"] = P.state()
        outs.append(o)
    stats = G.stats()
    G.close()
    for P in probs:
        P.close()
    return outs, stats


def test_auto_group_equals_alone_bit_for_bit_and_oracle():
    """Ten mixed problems, q in {50, 100, 150}: the q <= 128 ones on the
    two-warp group kernels, the q = 150 ones on the three-warp kernels, one
    launch per (warps, circles) pair."""
    T = tj()
    pbs = mix(count=10, seed=8)
    assert {pb["q"] for pb in pbs} & {50, 100} and 150 in {pb["q"] for pb in pbs}
    outs, (launches, items) = group(pbs, 10, T.AM_KERNEL_AUTO)
    variants = {(2 if pb["q"] <= 128 else 3, pb["m"]) for pb in pbs}
    assert launches == len(variants)
    for pb, g in zip(pbs, outs):
        a = alone(pb, 10, T.AM_KERNEL_AUTO)
        np.testing.assert_array_equal(g["state"], a["state"])
        for k in ("res", "res_psi", "cost", "mind"):
            np.testing.assert_array_equal(g[k], a[k], err_msg=k)
        check_oracle(pb, g)


def test_autotune_picks_a_warp_slot_cap_and_every_cap_gives_the_same_bits():
    """The autotuner times caps on the warp-pair group kernels' trajectory
    slots per CTA and keeps one; since a trajectory's arithmetic does not
    depend on the CTA slot that runs it, every cap gives the same bits."""
    T = tj()
    pbs = mix(count=6, seed=12)
    states = {}
    for cap in (None, 0, 5, 3, 1):
        probs = [T.Problem(pb, kernel=T.AM_KERNEL_AUTO).init_state(pb["init"].astype(np.float32)) for pb in pbs]
        G = T.Group(probs)
        if cap is None:
            threads, ms = G.autotune(10)
            assert G.warp_slots() in (0, 7, 6, 5, 4, 3) and ms > 0
        else:
            T.am_group_set_option(G.g, T.AM_GOPT_WARP_SLOTS, cap)
            assert G.warp_slots() == cap
        G.solve(10)
        states[cap] = [P.state() for P in probs]
        G.close()
        for P in probs:
            P.close()
    for cap in (0, 5, 3, 1):
        for a, b in zip(states[cap], states[None]):
            np.testing.assert_array_equal(a, b)
    G = T.Group([T.Problem(pbs[0], kernel=T.AM_KERNEL_AUTO).init_state(pbs[0]["init"].astype(np.float32))])
    with pytest.raises(T.TrajamError):
        T.am_group_set_option(G.g, T.AM_GOPT_WARP_SLOTS, 9)
    G.close()


_MIX_ORACLE = {}


@pytest.mark.parametrize("kernel", ["auto", "small_tile"])
def test_full_size_uneven_mix_sampled_against_the_oracle(kernel):
    """The benchmark's uneven mix at full size (64 problems, B 128..2048, about
    70 k trajectories) in one grouped solve of 10 iterations; the first and
    the last trajectory of every problem (the first and last tiles) against
    the FP64 oracle, with the mix's noise-derived tolerance."""
    from test_gpu_group import coef_tolerance
    from test_gpu_parity import assert_coefs
    T = tj()
    k = T.AM_KERNEL_AUTO if kernel == "auto" else T.AM_KERNEL_FUSED
    pbs = W.make_uneven(0, count=64)
    assert sum(pb["B"] for pb in pbs) > 60000
    probs = [T.Problem(pb, kernel=k).init_state(pb["init"].astype(np.float32)) for pb in pbs]
    G = T.Group(probs)
    G.solve(10)
    for i, (pb, P) in enumerate(zip(pbs, probs)):
        st = T.split_state(P.state())
        idx = [0, pb["B"] - 1]
        if i not in _MIX_ORACLE:  # shared by both kernels' runs
            _MIX_ORACLE[i] = coef_tolerance(dict(pb, init=pb["init"][idx], B=len(idx)), 10)
        o, tol = _MIX_ORACLE[i]
        assert_coefs({key: st[key][idx] for key in ("xi1", "xi2")}, o, tol=tol)
    G.close()
    for P in probs:
        P.close()


def test_warp_group_equals_warp_alone():
    """Every problem selects AM_KERNEL_WARP: the same bits as lone warp-pair
    solves, also when the captured launch is replayed on a stream."""
    import torch
    T = tj()
    pbs = mix(count=6, seed=9)
    st = torch.cuda.Stream()
    outs, _ = group(pbs, 10, T.AM_KERNEL_WARP, reps=2, stream=st)
    for pb, g in zip(pbs, outs):
        # two group solves of 10 iterations from the cold start: the second
        # continues from the first, like one 10-iteration solve then a warm one
        P = T.Problem(pb, kernel=T.AM_KERNEL_WARP)
        P.solve(pb["init"].astype(np.float32), 10)
        P.solve(None, 10)
        ref = P.state()
        P.close()
        np.testing.assert_array_equal(g["state"], ref)


def test_server_auto_scene_alone_equals_in_mix():
    T = tj()
    pbs = W.make_uneven(21, count=4, scale=1.0 / 64)

    def serve(ks, start_after_submit):
        S = T.Server(8 << 30, 10)
        probs = []
        for pb in pbs:
            P = T.Problem(pb, kernel=T.AM_KERNEL_AUTO)
            S.add_scene(P, pb["init"].astype(np.float32))
            probs.append(P)
        if not start_after_submit:
            S.start()
        tickets = [S.submit(k) for k in ks]
        if start_after_submit:
            S.start()
        out = [S.wait(t) for t in tickets]
        S.close()
        for P in probs:
            P.close()
        return out

    first = serve([0], False)[0]
    mixed = serve(range(len(pbs)), True)
    assert first["status"] == 0 and all(r["status"] == 0 for r in mixed)
    assert all(r["batch"] == len(pbs) for r in mixed)
    np.testing.assert_array_equal(np.asarray(mixed[0]["coeffs"]), np.asarray(first["coeffs"]))


@pytest.mark.parametrize("case", ["paper", "q150", "q256", "literal", "tf32", "large"])
def test_auto_picks_the_kernel(case):
    """AM_KERNEL_AUTO solves with the large-batch kernel from B = 16384 on,
    else with the warp-pair kernel where it takes the problem, else with the
    small-tile kernel: the same bits as the explicit choice."""
    T = tj()
    flags, expect = {}, T.AM_KERNEL_WARP
    if case == "paper":
        pb = W.make_problem("paper", 0, B=64)
    elif case == "q150":
        pb = W.make_shape(11, 16, 150, 6, 3)
    elif case == "q256":
        pb = W.make_shape(12, 9, 256, 20, 2)
    elif case == "tf32":
        pb, flags, expect = W.make_problem("tiny", 0, B=16), dict(precision=T.AM_TF32), T.AM_KERNEL_FUSED
    elif case == "literal":
        pb, flags, expect = W.make_problem("tiny", 0, B=16), dict(alpha_mode=1), T.AM_KERNEL_FUSED
    else:
        pb, expect = W.make_problem("paper", 0, B=16384), T.AM_KERNEL_LARGE
    a = alone(dict(pb), 10, T.AM_KERNEL_AUTO) if not flags else None
    if flags:
        P = T.Problem(pb, kernel=T.AM_KERNEL_AUTO, **flags)
        P.solve(pb["init"].astype(np.float32), 10)
        a = {"state": P.state()}
        P.close()
        P = T.Problem(pb, kernel=expect, **flags)
        P.solve(pb["init"].astype(np.float32), 10)
        b = {"state": P.state()}
        P.close()
    else:
        b = alone(dict(pb), 10, expect)
    np.testing.assert_array_equal(a["state"], b["state"])
