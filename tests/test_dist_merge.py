"""Sharded batch on two CPU ranks (gloo): the cross-rank best merge returns
the same trajectory as a selection over the whole batch.

Each rank runs the FP64 oracle on its contiguous range of one problem's
samples (a stand-in for a GPU's solve; the merge sees only per-rank bests),
picks its local best by the lexicographic key (collision-free first, then
cost, then index), and the ranks merge.  The expected winner is the same key
taken over the oracle's results for the whole batch.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2109_13030_b300 import workload as W


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def local_best(o, lo):
    ok = o["mind"] >= 0.99
    cand = np.where(ok)[0] if ok.any() else np.arange(len(o["cost"]))
    i = cand[np.lexsort((cand, o["cost"][cand]))][0]
    coeffs = np.stack([o["xi1"][i, 0:11], o["xi1"][i, 22:33], o["xi2"][i]]).astype(np.float32)
    return (not ok.any()), float(o["cost"][i]), lo + int(i), coeffs


def worker(rank, world, port, pb, iters, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2109_13030_b300 import dist_best as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = D.shard_range(pb["B"], rank, world)
    sub = dict(pb, init=pb["init"][lo:hi], B=hi - lo)
    o = O.solve(sub, iters)
    collides, cost, gidx, coeffs = local_best(o, lo)
    best = D.merge_best(collides, cost, gidx, coeffs, torch.device("cpu"))
    # the device-side form on the same local bests (record: local index,
    # cost, residual, coefficients)
    rec = torch.tensor([gidx - lo, cost, 0.0, *coeffs.ravel()], dtype=torch.float32)
    win = D.merge_best_device(rec, torch.tensor([collides]), lo)
    out[rank] = (best["index"], best["cost"], best["collides"], best["rank"],
                 best["coeffs"].numpy().copy(), win.numpy().copy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_merge_matches_whole_batch(world):
    pb = W.make_problem("tiny", 2)
    iters = 20
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = free_port()
        procs = [ctx.Process(target=worker, args=(r, world, port, pb, iters, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    whole = O.solve(pb, iters)
    collides, cost, gidx, coeffs = local_best(whole, 0)
    for r in range(world):
        idx, c, col, owner, co, win = res[r]
        assert idx == gidx and col == collides
        assert c == pytest.approx(cost, rel=1e-12)
        np.testing.assert_array_equal(co, coeffs)
        # the device-side merge picks the same trajectory on every rank
        assert int(win[0]) == gidx and win[1] == np.float32(cost)
        np.testing.assert_array_equal(win[3:], coeffs.ravel())
    # the owner is the rank whose range holds the winner
    from paper_2109_13030_b300 import dist_best as D
    lo, hi = D.shard_range(pb["B"], res[0][3], world)
    assert lo <= gidx < hi


def test_shard_ranges_cover_batch():
    from paper_2109_13030_b300 import dist_best as D
    for B in (1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            spans = [D.shard_range(B, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == B
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))


def test_device_merge_order_single_rank_rules():
    """The device-side merge's ordering on one gloo rank (world 1): the
    record comes back with its index made global, and a non-finite cost is
    kept as it is."""
    import torch
    import torch.distributed as dist
    from paper_2109_13030_b300 import dist_best as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(free_port()))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        rec = torch.arange(36, dtype=torch.float32)
        win = D.merge_best_device(rec, torch.tensor([False]), 100)
        assert win[0] == 100 and torch.equal(win[1:], rec[1:])
        rec[1] = float("nan")
        win = D.merge_best_device(rec, torch.tensor([True]), 5)
        assert win[0] == 5 and torch.isnan(win[1])
    finally:
        dist.destroy_process_group()


def test_key_order():
    from paper_2109_13030_b300 import dist_best as D
    assert D.key_of(False, 5.0, 9) < D.key_of(True, 1.0, 0)
    assert D.key_of(False, 1.0, 9) < D.key_of(False, 2.0, 0)
    assert D.key_of(False, 1.0, 3) < D.key_of(False, 1.0, 4)


def rules_worker(rank, world, port, cases, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2109_13030_b300 import dist_best as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = []
    for case in cases:
        idx, cost, collides, offset = case[rank]
        rec = torch.zeros(36, dtype=torch.float32)
        rec[0], rec[1] = float(idx), float(cost)
        rec[3:] = float(rank + 1)  # coefficients tell the owner apart
        win = D.merge_best_device(rec, torch.tensor([collides]), offset)
        res.append((int(win[0]), float(win[3])))
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_device_merge_rules_on_two_ranks():
    """Equal costs go to the lower global index; a collision-free trajectory
    beats a cheaper colliding one; a non-finite cost ranks last."""
    cases = [
        [(3, 5.0, False, 0), (0, 5.0, False, 10)],              # tie: global 3 < 10
        [(2, 1.0, True, 0), (4, 9.0, False, 10)],               # collision-free first: global 14
        [(1, float("nan"), False, 0), (7, 50.0, True, 10)],     # non-finite last: global 17
        [(0, 2.0, False, 0), (0, 1.0, False, 10)],              # lower cost: global 10
    ]
    expect = [(3, 1.0), (14, 2.0), (17, 2.0), (10, 2.0)]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = free_port()
        procs = [ctx.Process(target=rules_worker, args=(r, 2, port, cases, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1] == expect
