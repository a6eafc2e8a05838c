"""The CEM comparator (Sec. IV, Table IV) on the GPU, against its definition.

* The score J of given plans equals a numpy evaluation of the objective
  written out here (its own Bernstein basis and derivatives, inflated
  ellipses, circle centres, penetration and bound penalties).
* One iteration's samples have the documented starting mean and covariance
  (straight line; blockdiag(sigma_xy^2 C, sigma_xy^2 C, sigma_psi^2 C), C from
  ``workload.smoothness_covariance``) and standard normal whitened values.
* The refit equals numpy's on the same samples and scores: the K lowest
  (ties to the lower index), their mean and covariance (normalised by K),
  smoothing and the covariance floor.
* The best plan is the lowest score seen, and re-scoring it gives its score.
"""
from math import comb

import numpy as np
import pytest
from scipy import stats

from paper_2109_13030_b300 import workload as W

pytestmark = pytest.mark.gpu


def tj():
    from paper_2109_13030_b300 import trajam
    return trajam


def basis(q, T):
    """P, dP/dt, d2P/dt2 of the degree-10 Bernstein basis on t_k = k T / (q - 1)."""
    tau = np.linspace(0.0, 1.0, q)

    def b(n, k):
        return comb(n, k) * tau ** k * (1 - tau) ** (n - k) if 0 <= k <= n else np.zeros(q)

    P = np.stack([b(10, k) for k in range(11)], 1)
    Pd = np.stack([10 * (b(9, k - 1) - b(9, k)) for k in range(11)], 1) / T
    Pdd = np.stack([90 * (b(8, k - 2) - 2 * b(8, k - 1) + b(8, k)) for k in range(11)], 1) / T ** 2
    return P, Pd, Pdd


def objective(pb, c, w_coll, w_bound):
    """J and the smallest ellipse distance of one plan c = (c_x, c_y, c_psi)."""
    P, Pd, Pdd = basis(pb["q"], pb["T"])
    cx, cy, cp = (np.asarray(v, np.float64) for v in c)
    x, y, psi = P @ cx, P @ cy, P @ cp
    xd, yd = Pd @ cx, Pd @ cy
    xdd, ydd, pdd = Pdd @ cx, Pdd @ cy, Pdd @ cp
    J = np.sum(xdd ** 2 + ydd ** 2 + pdd ** 2)
    J += w_bound * np.sum(np.maximum(0, np.hypot(xd, yd) - pb["v_max"]) ** 2
                          + np.maximum(0, np.hypot(xdd, ydd) - pb["a_max"]) ** 2)
    a = pb["ao"] + pb["r_c"]
    b = pb["bo"] + pb["r_c"]
    dmin = np.inf
    for r in pb["r"]:
        X, Y = x + r * np.cos(psi), y + r * np.sin(psi)
        d = np.hypot((X[None, :] - pb["xo"]) / a[:, None], (Y[None, :] - pb["yo"]) / b[:, None])
        J += w_coll * np.sum(np.maximum(0, 1 - d) ** 2)
        dmin = min(dmin, d.min())
    return J, dmin


def end_points(bc, T):
    """Control points 0, 1, 2, 8, 9, 10 fixed by value, velocity, acceleration at both ends."""
    c0, c10 = bc[0], bc[3]
    c1 = c0 + T * bc[1] / 10
    c9 = c10 - T * bc[4] / 10
    c2 = 2 * c1 - c0 + T * T * bc[2] / 90
    c8 = 2 * c9 - c10 + T * T * bc[5] / 90
    return [c0, c1, c2], [c8, c9, c10]


def full_plans(pb, z):
    """Coefficients from boundary conditions and z (control points 3..7 of x, y, psi)."""
    out = np.zeros((z.shape[0], 3, 11))
    for blk, bc in enumerate((pb["x_bc"], pb["y_bc"], pb["psi_bc"])):
        lo, hi = end_points(bc, pb["T"])
        out[:, blk, :3] = lo
        out[:, blk, 8:] = hi
        out[:, blk, 3:8] = z[:, 5 * blk:5 * blk + 5]
    return out


@pytest.fixture(scope="module")
def paper():
    return W.make_problem("paper", 0, B=64)


def test_score_matches_the_objective(paper):
    T = tj()
    P = T.Problem(paper)
    c = paper["init"].copy()
    rng = np.random.default_rng(2)
    c[:, 2, 3:8] += rng.normal(0, 0.5, (paper["B"], 5))   # exercise the heading,
    c[:, 2, 8:] += rng.normal(0, 0.3, (paper["B"], 3))    # its last control points included
    for w_coll, w_bound in ((1e4, 1e2), (0.0, 0.0), (1.0, 0.0)):
        cost, md = T.am_cem_score(P.h, c.reshape(-1, 33).astype(np.float32), w_coll, w_bound)
        for l in range(paper["B"]):
            J, d = objective(paper, c[l].astype(np.float32), w_coll, w_bound)
            assert cost[l] == pytest.approx(J, rel=2e-4, abs=1e-3), (l, w_coll)
            assert md[l] == pytest.approx(d, rel=1e-5, abs=1e-5)
    assert np.any(md < 1.0) and np.any(md > 1.0)   # both colliding and free plans among them
    P.close()


@pytest.fixture(scope="module")
def one_iteration(paper):
    T = tj()
    P = T.Problem(paper)
    N, K, alpha, reg = 8192, 512, 0.7, 1e-3
    T.am_cem_solve(P.h, samples=N, elites=K, iters=1, sigma_xy=1.0, sigma_psi=0.3, alpha=alpha, reg=reg, seed=5)
    s = T.am_cem_get_samples(P.h, N)
    best = T.am_cem_get_best(P.h)
    cost_again, md_again = T.am_cem_score(P.h, full_plans(paper, s["z"].astype(np.float64))[:256]
                                          .reshape(-1, 33).astype(np.float32))
    P.close()
    return dict(s=s, N=N, K=K, alpha=alpha, reg=reg, best=best, cost_again=cost_again)


def start_distribution(pb):
    mu0 = np.zeros(15)
    for blk, bc in enumerate((pb["x_bc"], pb["y_bc"], pb["psi_bc"])):
        mu0[5 * blk:5 * blk + 5] = bc[0] + (bc[3] - bc[0]) * np.arange(1, 6) / 6.0
    C = W.smoothness_covariance()
    S0 = np.zeros((15, 15))
    for blk, s in enumerate((1.0, 1.0, 0.3)):
        S0[5 * blk:5 * blk + 5, 5 * blk:5 * blk + 5] = s * s * C
    return mu0, S0


def test_samples_have_the_start_distribution(paper, one_iteration):
    s = one_iteration["s"]
    z = s["z"].astype(np.float64)
    mu0, S0 = start_distribution(paper)
    n = z.shape[0]
    assert np.all(np.abs(z.mean(0) - mu0) <= 5 * np.sqrt(np.diag(S0)) / np.sqrt(n))
    assert np.abs(np.cov(z.T) - S0).max() <= 0.1
    w = np.linalg.solve(np.linalg.cholesky(S0), (z - mu0).T).ravel()
    assert stats.kstest(w, "norm").pvalue > 1e-4


def test_scores_of_samples_match_rescoring(one_iteration):
    c = one_iteration["cost_again"]
    np.testing.assert_allclose(c, one_iteration["s"]["cost"][:256], rtol=1e-5)


def test_refit_matches_the_definition(paper, one_iteration):
    o = one_iteration
    s = o["s"]
    z = s["z"].astype(np.float64)
    cost = s["cost"]
    order = np.lexsort((np.arange(o["N"]), cost))        # by score, ties to the lower index
    E = z[order[:o["K"]]]
    m = E.mean(0)
    cov = (E - m).T @ (E - m) / o["K"]
    mu0, S0 = start_distribution(paper)
    np.testing.assert_allclose(s["mu"], o["alpha"] * m + (1 - o["alpha"]) * mu0, atol=2e-5)
    np.testing.assert_allclose(s["sigma"], o["alpha"] * cov + (1 - o["alpha"]) * S0 + o["reg"] * np.eye(15),
                               atol=2e-5)
    assert o["best"]["cost"] == pytest.approx(float(cost[order[0]]), rel=1e-7)


def test_best_is_the_lowest_seen_and_collision_free(paper):
    T = tj()
    P = T.Problem(paper)
    T.am_cem_solve(P.h, seed=3)
    best = T.am_cem_get_best(P.h)
    last = T.am_cem_get_samples(P.h, 8000)["cost"]
    assert best["cost"] <= last.min() + 1e-3
    again, md = T.am_cem_score(P.h, best["coeffs"].reshape(1, 33))
    assert again[0] == pytest.approx(best["cost"], rel=1e-6)
    assert md[0] == pytest.approx(best["min_dist"], rel=1e-6)
    assert best["min_dist"] >= 0.99          # 10 moving ellipses: CEM finds a way through
    P.close()


def test_cem_argument_checks(paper):
    T = tj()
    P = T.Problem(paper)
    with pytest.raises(T.TrajamError) as e:
        T.am_cem_get_best(P.h)
    assert e.value.code == T.AM_ERR_STATE
    for bad in (dict(samples=8), dict(samples=9000), dict(elites=1), dict(elites=2000), dict(iters=0),
                dict(alpha=0.0), dict(reg=0.0), dict(sigma_xy=-1.0), dict(w_coll=float("nan"))):
        with pytest.raises(T.TrajamError) as e:
            T.am_cem_solve(P.h, **bad)
        assert e.value.code == T.AM_ERR_ARG, bad
    with pytest.raises(T.TrajamError):
        T.am_cem_solve(P.h, warm=np.zeros(33), warm_dt=-1.0)
    P.close()


def test_cem_reaches_the_free_space_optimum():
    """No obstacles, inactive bounds: J is the smoothness cost alone, whose
    minimum over control points 3..7 (the rest fixed by the boundary
    conditions) is a least-squares problem, solved here in numpy.  CEM's best
    plan must come within 1 % of it and never below it."""
    T = tj()
    pb = W.with_obstacles_removed(W.make_problem("paper", 0, B=8))
    P = T.Problem(pb)
    T.am_cem_solve(P.h, seed=11, iters=30)
    best = T.am_cem_get_best(P.h)
    _, _, Pdd = basis(pb["q"], pb["T"])
    H = Pdd.T @ Pdd
    J_star = 0.0
    for bc in (pb["x_bc"], pb["y_bc"], pb["psi_bc"]):
        lo, hi = end_points(bc, pb["T"])
        c_fixed = np.zeros(11)
        c_fixed[:3], c_fixed[8:] = lo, hi
        E = np.zeros((11, 5))
        E[3:8, :] = np.eye(5)
        z = -np.linalg.solve(E.T @ H @ E, E.T @ H @ c_fixed)
        c = c_fixed + E @ z
        J_star += c @ H @ c
    assert J_star * (1 - 1e-4) <= best["cost"] <= J_star * 1.01, (best["cost"], J_star)
    P.close()
