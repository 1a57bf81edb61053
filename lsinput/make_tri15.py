"""Write ``tri15.txt``: the 15-node fully symmetric interpolation/quadrature rule.

The paper discretises each curved triangle with a Vioreanu-Rokhlin rule of
interpolation degree p (n_q = (p+1)(p+2)/2 interior nodes whose degree of
exactness exceeds p; Section 3).  Those tables are not reproduced here: this
script computes its own p = 4 rule (15 nodes) on the reference triangle
{(x, y): x, y >= 0, x + y <= 1} with the orbit structure 3 x S21 + 1 x S111
(3*3 + 6 = 15 nodes).  The 9 orbit parameters are fitted by nonlinear least
squares to the moments of every monomial of total degree <= 7, which the fit
meets to round-off: a one-parameter family of degree-7 rules.  The member kept
has its S111 orbit at smallest barycentric coordinate 0.04 (the most interior
member with well-separated positive weights), reached by continuation from a
seeded starting point.

Run:  python -m lsinput.make_tri15      (rewrites lsinput/tri15.txt)
"""
import itertools
import os
from math import factorial

import numpy as np
from scipy.optimize import least_squares

DEGREE = 7
C_S111 = 0.04
_MONOS = [(i, d - i) for d in range(DEGREE + 1) for i in range(d + 1)]
_EXACT = np.array([factorial(i) * factorial(j) / factorial(i + j + 2) for i, j in _MONOS])


def _expand(a, b, c, w):
    pts, wts = [], []
    for ai, wi in zip(a, w[:3]):
        for lam in [(ai, ai, 1 - 2 * ai), (ai, 1 - 2 * ai, ai), (1 - 2 * ai, ai, ai)]:
            pts.append(lam)
            wts.append(wi)
    bary = (b, c, 1 - b - c)
    for perm in itertools.permutations(range(3)):
        pts.append(tuple(bary[k] for k in perm))
        wts.append(w[3])
    lam = np.array(pts)
    return lam[:, 1], lam[:, 2], np.array(wts)


def _residual(q, c):
    x, y, w = _expand(q[0:3], q[3], c, q[4:8])
    return np.array([np.sum(w * x**i * y**j) for i, j in _MONOS]) - _EXACT


def solve_rule():
    # Seeded start on the degree-7 family (found by a random multistart search).
    q = np.array([0.41632373, 0.16812755, 0.05617228, 0.66355879,
                  0.06104687, 0.03826279, 0.02018902, 0.023584])
    c0 = 1.0 - 0.66355879 - 0.31267409
    for c in np.linspace(c0, C_S111, 20):
        r = least_squares(_residual, q, args=(c,), xtol=1e-15, ftol=1e-15, gtol=1e-15)
        q = r.x
    assert np.max(np.abs(_residual(q, C_S111))) < 1e-15
    return _expand(q[0:3], q[3], C_S111, q[4:8])


def main():
    x, y, w = solve_rule()
    path = os.path.join(os.path.dirname(__file__), "tri15.txt")
    with open(path, "w") as f:
        f.write("# 15-node symmetric rule on the triangle (0,0),(1,0),(0,1); degree of exactness 7\n")
        f.write("# columns: x y weight (weights sum to 1/2); written by lsinput/make_tri15.py\n")
        for xi, yi, wi in zip(x, y, w):
            f.write(f"{xi:.17e} {yi:.17e} {wi:.17e}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
