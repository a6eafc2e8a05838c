"""Reduced-precision forms (AM_TF32, AM_BF16, AM_SPLIT_BF16) on the
4096-trajectory paper-shaped workload, against the FP64 oracle on sampled
trajectories.

In these forms the tensor-core contraction over the time grid, R = F^T (g -
F xi1), takes one product of operands rounded to TF32 (unit roundoff u =
2^-11) or BF16 (u = 2^-8), or three BF16 products of operands split into
hi + lo (split BF16, u = 2^-16); the position and heading steps stay FP32.
The error is a reported property of the form, not an FP32 parity bar: after
10 iterations the coefficients are measured within ~6 u (TF32), ~17 u (BF16)
and ~7 u (split BF16) of the oracle, and the cost within ~1 u, ~2 u and
~0.5 u.  The bounds below are 30 u on coefficients and 10 u on the cost; an
implementation mistake (a wrong fragment layout, a dropped term) gives
errors of order one.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_13030_b300 import workload as W

from test_gpu_parity import COEF_TOL, coef_err, sub_problem

pytestmark = pytest.mark.gpu

U = {1: 2.0 ** -11, 2: 2.0 ** -8, 3: 2.0 ** -16}


def tj():
    from paper_2109_13030_b300 import trajam
    return trajam


@pytest.fixture(scope="module")
def workload():
    pb = W.make_problem("precision", 0)
    idx = np.unique(np.concatenate([[0, 1, 4095], np.random.default_rng(3).choice(pb["B"], 21, replace=False)]))
    return pb, idx, O.solve(sub_problem(pb, idx), 10)


def solve(pb, precision, iters=10):
    T = tj()
    P = T.Problem(pb, precision=precision)
    P.solve(pb["init"].astype(np.float32), iters)
    out = T.split_state(P.state())
    out.update(P.results())
    P.close()
    return out


@pytest.mark.parametrize("precision", [1, 2, 3])
def test_reduced_precision_error_bound(workload, precision):
    pb, idx, o = workload
    g = solve(pb, precision)
    u = U[precision]
    for key in ("xi1", "xi2"):
        e = coef_err(g[key][idx], o[key])
        assert np.all(np.isfinite(e)) and e.max() <= 30 * u, (key, e.max())
    dc = np.abs(g["cost"][idx] - o["cost"]) / np.abs(o["cost"])
    assert dc.max() <= 10 * u, dc.max()


def test_fp32_form_on_the_same_workload(workload):
    pb, idx, o = workload
    g = solve(pb, 0)
    for key in ("xi1", "xi2"):
        assert coef_err(g[key][idx], o[key]).max() <= COEF_TOL


def test_reduced_precision_not_on_the_plain_kernel():
    T = tj()
    pb = W.make_problem("tiny", 0)
    P = T.Problem(pb, precision=T.AM_TF32, kernel=T.AM_KERNEL_PLAIN)
    with pytest.raises(T.TrajamError) as e:
        P.solve(pb["init"].astype(np.float32), 5)
    assert e.value.code == T.AM_ERR_ARG
    P.close()
