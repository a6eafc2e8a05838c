"""Edge shapes on the GPU: the smallest solvable horizon, the largest shapes the
fused kernel holds in shared memory, the maximum shape (q = 256, m = 4,
n = 64) on the plain kernel, and the shapes that are rejected.

The fused kernel stages a problem's constants in shared memory; the largest
shapes (q = 256 with more than 45 obstacles) do not fit and are refused with
AM_ERR_ARG, naming the plain kernel, which runs any shape.
Tolerances against the oracle follow the mixed-problem rule (the larger of
1e-4 and three times the oracle's own movement under FP32-sized noise).
"""
import numpy as np
import pytest

from paper_2109_13030_b300 import workload as W

from test_gpu_group import coef_tolerance
from test_gpu_parity import assert_coefs

pytestmark = pytest.mark.gpu


def tj():
    from paper_2109_13030_b300 import trajam
    return trajam


def solve(pb, iters, kernel=0):
    T = tj()
    P = T.Problem(pb, kernel=kernel)
    P.solve(pb["init"].astype(np.float32), iters)
    out = T.split_state(P.state())
    out.update(P.results())
    P.close()
    return out


@pytest.mark.parametrize("kernel", [0, 1])
def test_smallest_solvable_horizon(kernel):
    pb = W.make_shape(3, B=5, q=6, n=2, m=1)
    o, tol = coef_tolerance(pb, 10)
    assert_coefs(solve(pb, 10, kernel), o, tol=tol)


def test_singular_horizon_rejected():
    """With q = 3 samples the position KKT matrix is singular (as in the oracle)."""
    T = tj()
    pb = W.make_shape(3, B=2, q=3, n=2, m=1)
    with pytest.raises(T.TrajamError) as e:
        T.Problem(pb)
    assert e.value.code == T.AM_ERR_ARG and "singular" in str(e.value)


@pytest.mark.parametrize("q,n,m", [(150, 64, 4), (200, 64, 4), (256, 32, 4), (256, 45, 2), (50, 64, 1)])
def test_largest_fused_shapes(q, n, m):
    pb = W.make_shape(5, B=6, q=q, n=n, m=m)
    o, tol = coef_tolerance(pb, 5)
    assert_coefs(solve(pb, 5, kernel=0), o, tol=tol)


def test_maximum_shape_runs_on_the_plain_kernel():
    T = tj()
    pb = W.make_shape(7, B=4, q=256, n=64, m=4)
    with pytest.raises(T.TrajamError) as e:
        solve(pb, 5, kernel=0)
    assert e.value.code == T.AM_ERR_ARG and "plain kernel" in str(e.value)
    o, tol = coef_tolerance(pb, 5)
    assert_coefs(solve(pb, 5, kernel=1), o, tol=tol)
    P = T.Problem(pb)
    P.init_state(pb["init"].astype(np.float32))
    with pytest.raises(T.TrajamError) as e:
        T.Group([P]).solve(5)
    assert e.value.code == T.AM_ERR_ARG
    P.close()


def test_single_obstacle_single_circle():
    pb = W.make_shape(9, B=3, q=40, n=1, m=1)
    o, tol = coef_tolerance(pb, 10)
    for kernel in (0, 1):
        assert_coefs(solve(pb, 10, kernel), o, tol=tol)
