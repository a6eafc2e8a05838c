"""Writes bernstein_deg10.txt: exact Bernstein basis values and derivatives.

Eq. param of the paper parametrises x(t) = P c_x with a polynomial basis; this
build uses the degree-10 Bernstein basis B_k(tau) = C(10,k) tau^k (1-tau)^(10-k)
on tau = t / T.  The values are computed in exact rational arithmetic from that
definition (expanding the polynomial and differentiating term by term), so they
depend on no code under test.  Columns: tau, k, B_k, dB_k/dtau, d2B_k/dtau2.
"""
from fractions import Fraction as Fr
from math import comb
import os

N = 10
TAUS = [Fr(0), Fr(1, 7), Fr(1, 3), Fr(1, 2), Fr(9, 10), Fr(1)]


def poly_coeffs(k):
    # C(N,k) tau^k (1-tau)^(N-k) = C(N,k) sum_j C(N-k,j) (-1)^j tau^(k+j)
    c = [Fr(0)] * (N + 1)
    for j in range(N - k + 1):
        c[k + j] += comb(N, k) * comb(N - k, j) * (-1) ** j
    return c


def ev(c, tau, der):
    s = Fr(0)
    for p, a in enumerate(c):
        if p < der or a == 0:
            continue
        f = 1
        for r in range(der):
            f *= (p - r)
        s += a * f * tau ** (p - der)
    return s


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bernstein_deg10.txt")
    with open(out, "w") as fh:
        fh.write("# Exact degree-10 Bernstein basis (Eq. param), tau k B dB/dtau d2B/dtau2\n")
        for tau in TAUS:
            for k in range(N + 1):
                c = poly_coeffs(k)
                fh.write(f"{float(tau)!r} {k} {float(ev(c, tau, 0))!r} {float(ev(c, tau, 1))!r} "
                         f"{float(ev(c, tau, 2))!r}\n")
