"""Single-step pins of the FP64 oracle: the position QP, the lambda update and
the lambda_psi update, each against an independent numpy statement.

Everything the checks need is rebuilt here from the paper's definitions, not
taken from the oracle:

* the basis from scipy's Bernstein evaluation (BPoly);
* F from the block structure printed after Eq. ine_1 (per side: A_v = Pd,
  A_a = Pdd, for every circle i and obstacle j the row block [P, r_i P], and
  [0, P] for the slack rows);
* g from the projections in their geometric form: a point outside an ellipse
  stays where it is and a point inside is pushed radially (in the
  ellipse-scaled frame) onto its boundary; velocity and acceleration are
  shortened to at most v_max and a_max (the d >= 1 and d in [0, 1] clips of
  Eq. compute_zeta_3 - compute_da);
* the slack boundary values from sympy's derivatives of cos(psi(t)) and
  sin(psi(t)).

The mutation tests at the end compile altered copies of the oracle (a
dropped rho, a flipped sign) on the CPU and check that the matching pin
fails, so the pins are known to see those mistakes.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import sympy as sp
from scipy.interpolate import BPoly

from oracle import oracle as O
from paper_2109_13030_b300 import workload as W


def basis(q, T, der, degree=10):
    t = np.linspace(0.0, T, q)
    M = np.zeros((q, degree + 1))
    for k in range(degree + 1):
        c = np.zeros((degree + 1, 1))
        c[k] = 1.0
        bp = BPoly(c, [0.0, T])
        M[:, k] = bp.derivative(der)(t) if der else bp(t)
    return M


def slack_bc(psi_bc):
    """(cos psi, d/dt cos psi, d2/dt2 cos psi) at t=0 and t=T and the same for
    sin, for a heading with the given value, rate and acceleration at the ends."""
    t = sp.symbols("t")
    out_c, out_s = [], []
    for e in range(2):
        p0, p1, p2 = (sp.Float(float(v), 30) for v in psi_bc[3 * e:3 * e + 3])
        psi = p0 + p1 * t + p2 * t**2 / 2
        for f, out in ((sp.cos(psi), out_c), (sp.sin(psi), out_s)):
            out.extend(float(sp.diff(f, t, k).subs(t, 0)) for k in range(3))
    return np.array(out_c), np.array(out_s)


def make_case(rho, rho_psi, seed=5, q=40, n=4, m=3, B=3):
    """Moving ellipses, three circles, a turning heading, random multipliers and
    a random start heading polynomial, so every term of the step is nonzero."""
    pb = W.make_shape(seed, B=B, q=q, n=n, m=m)
    pb["rho"], pb["rho_psi"] = rho, rho_psi
    pb["psi_bc"] = np.array([0.2, 0.15, -0.05, 0.9, -0.1, 0.02])
    rng = np.random.default_rng(seed + 100)
    xi1, xi2 = O.state_from_init(pb["init"])
    xi2 = xi2 + rng.normal(0.0, 0.3, xi2.shape)
    xi1[:, 11:22] = rng.normal(1.0, 0.1, (B, 11))
    xi1[:, 33:44] = rng.normal(0.0, 0.1, (B, 11))
    state = dict(xi1=xi1, xi2=xi2, lam=rng.normal(0.0, 2.0, (B, 44)),
                 lampsi=rng.normal(0.0, 1.0, (B, 11)))
    return pb, state


def build_F_side(pb, P, Pd, Pdd):
    """F of one side acting on (c_pos, c_slack): rows v, a, obstacle rows
    (circle-major, then obstacle, then step) and the slack rows."""
    q, m, n = pb["q"], pb["m"], pb["n"]
    Z = np.zeros_like(P)
    blocks = [np.hstack([Pd, Z]), np.hstack([Pdd, Z])]
    for i in range(m):
        for _ in range(n):
            blocks.append(np.hstack([P, pb["r"][i] * P]))
    blocks.append(np.hstack([Z, P]))
    return np.vstack(blocks)


def build_g(pb, x, xd, xdd, y, yd, ydd, psi):
    """g per side from the projections in geometric form (see the module text)."""
    q, m, n = pb["q"], pb["m"], pb["n"]
    gx, gy = [], []
    for (ux, uy), umax in (((xd, yd), pb["v_max"]), ((xdd, ydd), pb["a_max"])):
        norm = np.hypot(ux, uy)
        f = np.where(norm > umax, umax / np.where(norm > 0, norm, 1.0), 1.0)
        gx.append(ux * f)
        gy.append(uy * f)
    for i in range(m):
        for j in range(n):
            a = pb["ao"][j] + pb["r_c"]
            b = pb["bo"][j] + pb["r_c"]
            xt = x + pb["r"][i] * np.cos(psi) - pb["xo"][j]
            yt = y + pb["r"][i] * np.sin(psi) - pb["yo"][j]
            e = np.sqrt(xt**2 / a**2 + yt**2 / b**2)
            f = np.maximum(1.0, 1.0 / e)
            gx.append(pb["xo"][j] + xt * f)
            gy.append(pb["yo"][j] + yt * f)
    gx.append(np.cos(psi))
    gy.append(np.sin(psi))
    return np.concatenate(gx), np.concatenate(gy)


def kkt_parts(pb):
    q, T, rho = pb["q"], pb["T"], pb["rho"]
    P, Pd, Pdd = (basis(q, T, d) for d in (0, 1, 2))
    Fs = build_F_side(pb, P, Pd, Pdd)
    H = Pdd.T @ Pdd
    Qbar = np.zeros((44, 44))
    for blk in range(4):
        Qbar[11 * blk:11 * blk + 11, 11 * blk:11 * blk + 11] = H
    FtF = Fs.T @ Fs
    Qbar[0:22, 0:22] += rho * FtF
    Qbar[22:44, 22:44] += rho * FtF
    A = np.vstack([P[0], Pd[0], Pdd[0], P[-1], Pd[-1], Pdd[-1]])
    Aeq = np.zeros((24, 44))
    for e in range(4):
        Aeq[6 * e:6 * e + 6, 11 * e:11 * e + 11] = A
    cbc, sbc = slack_bc(pb["psi_bc"])
    beq = np.concatenate([pb["x_bc"], cbc, pb["y_bc"], sbc])
    return P, Pd, Pdd, Fs, Qbar, Aeq, beq


def g_of(pb, xi1, xi2, P, Pd, Pdd):
    cx, cy = xi1[0:11], xi1[22:33]
    return build_g(pb, P @ cx, Pd @ cx, Pdd @ cx, P @ cy, Pd @ cy, Pdd @ cy, P @ xi2)


# ---------------------------------------------------------------- the pins


def check_position_step(rho):
    """Eq. zeta_1_sepration_1 with Eq. zeta_1_sepration_3 and Eq. over_2: from
    the given (xi1, xi2, lam), one iteration's xi1 is the minimiser of
    1/2 xi^T Qbar xi + qbar^T xi s.t. Aeq xi = beq with Qbar = Q + rho F^T F and
    qbar = -lam - rho F^T g0, g0 from the given trajectory and heading."""
    pb, st = make_case(rho, 0.7)
    out = O.solve(pb, 1, state=st)
    P, Pd, Pdd, Fs, Qbar, Aeq, beq = kkt_parts(pb)
    K = np.block([[Qbar, Aeq.T], [Aeq, np.zeros((24, 24))]])
    for l in range(pb["B"]):
        gx, gy = g_of(pb, st["xi1"][l], st["xi2"][l], P, Pd, Pdd)
        Ftg = np.concatenate([Fs.T @ gx, Fs.T @ gy])
        lin = st["lam"][l] + rho * Ftg                        # -qbar
        xi_np = np.linalg.solve(K, np.concatenate([lin, beq]))[:44]
        xi = out["xi1"][l]
        scale = np.linalg.norm(Qbar, np.inf) * np.max(np.abs(xi)) + np.max(np.abs(lin))
        # stationarity: Qbar xi - lin + Aeq^T mu = 0 for some mu
        r = lin - Qbar @ xi
        mu = np.linalg.lstsq(Aeq.T, r, rcond=None)[0]
        assert np.max(np.abs(Aeq.T @ mu - r)) <= 1e-10 * scale
        assert np.max(np.abs(Aeq @ xi - beq)) <= 1e-10 * max(1.0, np.max(np.abs(beq)))
        np.testing.assert_allclose(xi, xi_np, rtol=0, atol=1e-10 * max(1.0, np.max(np.abs(xi_np))))


def check_lambda_update(rho):
    """Eq. update_lambda_1: lam' = lam - rho F^T (F xi1' - g'), with xi1' the
    step's new position coefficients and g' rebuilt from xi1' and the new
    heading xi2'."""
    pb, st = make_case(rho, 0.7)
    out = O.solve(pb, 1, state=st)
    P, Pd, Pdd, Fs, *_ = kkt_parts(pb)
    for l in range(pb["B"]):
        xi1, xi2 = out["xi1"][l], out["xi2"][l]
        gx, gy = g_of(pb, xi1, xi2, P, Pd, Pdd)
        rx, ry = Fs @ xi1[0:22] - gx, Fs @ xi1[22:44] - gy
        lam = st["lam"][l] - rho * np.concatenate([Fs.T @ rx, Fs.T @ ry])
        scale = max(1.0, np.max(np.abs(lam)))
        np.testing.assert_allclose(out["lam"][l], lam, rtol=0, atol=1e-11 * scale)
        # the residual reported is the norm of the same vector
        assert out["res"][l] == pytest.approx(np.sqrt(np.sum(rx**2) + np.sum(ry**2)), rel=1e-9)


def check_lambda_psi_update(rho, rho_psi, dual_sign):
    """Eq. update_lambda_psi in the reading that matches the lambda update
    (lam_psi' = lam_psi - rho_psi P^T (P xi2' - psi_t)); dual_sign = 1 is the
    printed sign (lam_psi' = lam_psi + rho_psi P^T (P xi2' - psi_t)).  psi_t is
    atan2(s, c) of the new slacks unwrapped against the previous heading."""
    pb, st = make_case(rho, rho_psi)
    out = O.solve(pb, 1, state=st, psi_dual_sign=dual_sign)
    P = basis(pb["q"], pb["T"], 0)
    sgn = -1.0 if dual_sign else 1.0
    for l in range(pb["B"]):
        psi0 = P @ st["xi2"][l]
        c, s = P @ out["xi1"][l, 11:22], P @ out["xi1"][l, 33:44]
        psit = psi0 + np.angle(np.exp(1j * (np.arctan2(s, c) - psi0)))
        v = P @ out["xi2"][l] - psit
        lp = st["lampsi"][l] - sgn * rho_psi * (P.T @ v)
        np.testing.assert_allclose(out["lampsi"][l], lp, rtol=0, atol=1e-10 * max(1.0, np.max(np.abs(lp))))
        assert out["res_psi"][l] == pytest.approx(np.linalg.norm(v), rel=1e-9)


@pytest.mark.parametrize("rho", [0.5, 3.0])
def test_position_step_solves_its_kkt_system(rho):
    check_position_step(rho)


@pytest.mark.parametrize("rho", [0.5, 3.0])
def test_lambda_update(rho):
    check_lambda_update(rho)


@pytest.mark.parametrize("rho,rho_psi,sign", [(0.5, 0.7, 0), (3.0, 0.7, 0), (0.5, 1.9, 1)])
def test_lambda_psi_update(rho, rho_psi, sign):
    check_lambda_psi_update(rho, rho_psi, sign)


# ------------------------------------------------------------ mutations

# (name, text in am_oracle.c, replacement, pins expected to fail)
MUTATIONS = [
    ("rho dropped on F^T F", "S->K1[a * n1 + b] += pb->rho * s;", "S->K1[a * n1 + b] += s;",
     ["position"]),
    ("rho dropped on F^T g", "lam[a] + pb->rho * w->Ftv[a]", "lam[a] + w->Ftv[a]", ["position"]),
    ("lambda sign flipped in the position step", "w->rhs1[a] = lam[a] + pb->rho",
     "w->rhs1[a] = -lam[a] + pb->rho", ["position"]),
    ("rho dropped in the lambda update", "lam[a] -= pb->rho * w->Ftv[a];", "lam[a] -= w->Ftv[a];",
     ["lambda"]),
    ("lambda update sign flipped", "lam[a] -= pb->rho * w->Ftv[a];", "lam[a] += pb->rho * w->Ftv[a];",
     ["lambda"]),
    ("rho_psi dropped", "lampsi[a] -= sgn * pb->rho_psi * w->rhsp[a];", "lampsi[a] -= sgn * w->rhsp[a];",
     ["lambda_psi"]),
    ("rho in place of rho_psi", "lampsi[a] -= sgn * pb->rho_psi * w->rhsp[a];",
     "lampsi[a] -= sgn * pb->rho * w->rhsp[a];", ["lambda_psi"]),
    ("lambda_psi sign flipped", "lampsi[a] -= sgn * pb->rho_psi * w->rhsp[a];",
     "lampsi[a] += sgn * pb->rho_psi * w->rhsp[a];", ["lambda_psi"]),
]

CHECKS = {
    "position": lambda: [check_position_step(r) for r in (0.5, 3.0)],
    "lambda": lambda: [check_lambda_update(r) for r in (0.5, 3.0)],
    "lambda_psi": lambda: [check_lambda_psi_update(0.5, 0.7, s) for s in (0, 1)],
}


def _load(path):
    lib = ctypes.CDLL(path)
    lib.or_solve.restype = ctypes.c_int
    lib.or_dense_solve.restype = ctypes.c_int
    lib.or_rows_per_side.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("name,old,new,fails", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistakes(tmp_path, monkeypatch, name, old, new, fails):
    src = open(O.SRC).read()
    assert src.count(old) == 1, name
    d = tmp_path / "mut"
    d.mkdir()
    shutil.copy(os.path.join(O.HERE, "am_oracle.h"), d / "am_oracle.h")
    (d / "am_oracle.c").write_text(src.replace(old, new))
    so = str(d / "libmut.so")
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
                           "-o", so, str(d / "am_oracle.c"), "-lm"])
    monkeypatch.setattr(O, "_lib", _load(so))
    for key, check in CHECKS.items():
        if key in fails:
            with pytest.raises(AssertionError):
                check()
        else:
            check()  # the other pins still hold
