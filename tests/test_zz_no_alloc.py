"""The allocation-free entry point against the allocating one.

am_solve_batch_noalloc serves callers that cannot allocate device memory at
solve time (a real-time re-planning step, a stream capture, an external
allocator): it runs the plain loop with its intermediates in a fixed area of
the library instead of memory obtained from cudaMalloc.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

from paper_2109_13030_b300 import workload as W

pytestmark = pytest.mark.gpu

COEF_TOL = 1e-4  # the coefficient tolerance of the parity tests


def cold_state(init: np.ndarray) -> np.ndarray:
    """B x 110 cold-start state: xi1 = (c_x, cos c_psi, c_y, sin c_psi), xi2 = c_psi."""
    B = init.shape[0]
    s = np.zeros((B, 110), dtype=np.float32)
    s[:, 0:11] = init[:, 0]
    s[:, 11:22] = np.cos(init[:, 2])
    s[:, 22:33] = init[:, 1]
    s[:, 33:44] = np.sin(init[:, 2])
    s[:, 44:55] = init[:, 2]
    return s


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    from paper_2109_13030_b300 import trajam as T
    pb = W.make_problem("paper", 7, B=256)
    B, iters = pb["B"], 20
    s0 = cold_state(pb["init"].astype(np.float32))

    # the existing entry point: plain loop, scratch from cudaMalloc
    P = T.Problem(pb, kernel=T.AM_KERNEL_PLAIN)
    T.am_set_state(P.h, B, s0)
    P.B = B
    P.solve(None, iters)
    ref_state = P.state()
    ref = P.results()

    stream = torch.cuda.current_stream()
    for call in range(2):
        state = torch.tensor(s0, device="cuda")
        outs = [torch.full((B,), float("nan"), device="cuda") for _ in range(4)]
        T.am_solve_batch_noalloc(P.h, B, state, *outs, iters, stream)
        torch.cuda.synchronize()
        st = state.cpu().numpy().astype(np.float64)
        err = np.max(np.abs(st - ref_state), axis=1) / np.maximum(np.max(np.abs(ref_state), axis=1), 1.0)
        assert err.max() <= COEF_TOL, (call, err.max())
        for name, o in zip(("res", "res_psi", "cost", "mind"), outs):
            v = o.cpu().numpy()
            assert np.all(np.isfinite(v)), (call, name)
            np.testing.assert_allclose(v, ref[name], rtol=1e-3, atol=5e-4, err_msg=f"{call} {name}")
    P.close()


def test_noalloc_rejects_batches_beyond_the_fixed_area():
    import torch
    from paper_2109_13030_b300 import trajam as T
    pb = W.make_problem("paper", 0, B=4)
    P = T.Problem(pb)
    B = 5000
    state = torch.zeros((B, 110), device="cuda")
    outs = [torch.zeros(B, device="cuda") for _ in range(4)]
    with pytest.raises(T.TrajamError) as e:
        T.am_solve_batch_noalloc(P.h, B, state, *outs, 10)
    assert e.value.code == T.AM_ERR_BUDGET
    assert "32 MiB" in str(e.value)
    P.close()


def test_noalloc_orders_itself_after_the_handles_stream():
    """The handle works on its own non-blocking stream and the caller solves on
    another: the call waits for what the handle's stream has queued (an event
    the handle owns, recorded there), so obstacles replaced just before the
    call are the ones the solve sees.  Checked against the allocating entry
    point solving the same scene after a full synchronisation."""
    import torch
    from paper_2109_13030_b300 import trajam as T
    pb = W.make_problem("paper", 8, B=128)
    other = W.make_problem("paper", 9, B=128)  # different obstacles
    B, iters = pb["B"], 20
    s0 = cold_state(pb["init"].astype(np.float32))
    obs = [np.ascontiguousarray(other[k], dtype=np.float32) for k in ("xo", "yo", "ao", "bo")]

    R = T.Problem(dict(pb, xo=other["xo"], yo=other["yo"], ao=other["ao"], bo=other["bo"]),
                  kernel=T.AM_KERNEL_PLAIN)
    T.am_set_state(R.h, B, s0)
    R.B = B
    R.solve(None, iters)
    ref_state, ref = R.state(), R.results()
    R.close()

    s_handle, s_call = torch.cuda.Stream(), torch.cuda.Stream()
    P = T.Problem(pb)
    state = torch.tensor(s0, device="cuda")
    outs = [torch.full((B,), float("nan"), device="cuda") for _ in range(4)]
    torch.cuda.synchronize()
    T.am_set_stream(P.h, s_handle)
    T.am_set_obstacles(P.h, other["n"], *obs)  # queued on the handle's stream
    T.am_solve_batch_noalloc(P.h, B, state, *outs, iters, s_call)
    s_call.synchronize()
    st = state.cpu().numpy().astype(np.float64)
    err = np.max(np.abs(st - ref_state), axis=1) / np.maximum(np.max(np.abs(ref_state), axis=1), 1.0)
    assert err.max() <= COEF_TOL, err.max()
    np.testing.assert_allclose(outs[2].cpu().numpy(), ref["cost"], rtol=1e-3)
    T.am_set_stream(P.h, None)
    P.close()
