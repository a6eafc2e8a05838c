"""The fused kernels' atan2 for the heading target (octant reduction and a
degree-8 polynomial in a^2), replayed step by step in float32 on the CPU and
checked against FP64 arctan2: every octant, both axes, signed zeros, tiny and
huge magnitudes, and atan2(0, 0) = 0.  The coefficients are read from the
kernels' shared header so the two cannot drift apart."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def coefficients():
    src = open(os.path.join(ROOT, "paper_2109_13030_b300", "csrc", "am_heading.cuh")).read()
    body = re.search(r"kAtanPoly\[9\] = \{([^}]*)\}", src).group(1)
    return np.array([float(v.strip().rstrip("f")) for v in body.split(",")], dtype=np.float32)


def atan2_f32(y, x):
    y = np.asarray(y, dtype=np.float32)
    x = np.asarray(x, dtype=np.float32)
    c = coefficients()
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    with np.errstate(invalid="ignore", divide="ignore"):
        a = np.where(mx > 0, mn / np.where(mx > 0, mx, 1), 0).astype(np.float32)
    s = (a * a).astype(np.float32)
    p = np.full_like(s, c[8])
    for k in range(7, -1, -1):
        p = (p * s + c[k]).astype(np.float32)   # one rounding per step, as fmaf
    r = (a * p).astype(np.float32)
    r = np.where(ay > ax, np.float32(1.57079637) - r, r).astype(np.float32)
    r = np.where(x < 0, np.float32(3.14159274) - r, r).astype(np.float32)
    return np.copysign(r, y).astype(np.float32)


def test_polynomial_fit_error():
    c = coefficients().astype(np.float64)
    a = np.linspace(1e-6, 1, 200001)
    approx = a * np.polyval(c[::-1], a * a)
    assert np.max(np.abs(approx - np.arctan(a)) / np.arctan(a)) < 5e-8


def test_all_octants_against_fp64():
    rng = np.random.default_rng(0)
    ang = rng.uniform(-np.pi, np.pi, 400000)
    rad = 10.0 ** rng.uniform(-6, 3, ang.size)
    y = (rad * np.sin(ang)).astype(np.float32)
    x = (rad * np.cos(ang)).astype(np.float32)
    got = atan2_f32(y, x).astype(np.float64)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    err = np.abs(got - ref)
    # a few float32 ulp of pi at most (the quotient a carries one rounding here,
    # two ulp with the device's approximate division)
    assert err.max() < 1.5e-6, err.max()
    assert np.median(err) < 1e-7


def test_axes_and_special_values():
    y = np.array([0, 0, 1, -1, 0.0, -0.0, 1, 1, -1, -1, 1e-30, 3e30], dtype=np.float32)
    x = np.array([0, 1, 0, 0, -1, -1, 1, -1, 1, -1, 1e-30, -3e30], dtype=np.float32)
    got = atan2_f32(y, x).astype(np.float64)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    ref[0] = 0.0  # atan2(0, 0) = 0
    assert np.all(np.abs(got - ref) < 1e-6), (got, ref)
