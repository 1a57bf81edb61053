"""Write dd_consts.h: double-double constants of the device correction setup.

Each constant c is stored as the pair (hi, lo) of doubles with hi = round(c) and
lo = round(c - hi), i.e. about 106 significant bits: pi, pi/2, 2/pi, Euler's
gamma, ln 2, the reciprocal factorials 1/n! (n = 0..30) used by the Taylor series
of exp, sin and cos, and for the ascending Bessel series (Abramowitz & Stegun
9.1.10-9.1.13) the reciprocals 1/k^2 and 1/(k (k + 1)) and the harmonic numbers
H_k and H_k + H_{k+1} (k = 0..DD_NSERIES).  Values from mpmath at 60 digits.

Run:  python paper_2608_17615_b300/csrc/gen_dd_consts.py
"""
import os

import mpmath

mpmath.mp.dps = 60
NFACT = 31
NSERIES = 96


def split(x):
    x = mpmath.mpf(x)
    hi = float(x)
    lo = float(x - mpmath.mpf(hi))
    return hi, lo


def fmt(name, x):
    hi, lo = split(x)
    return f"#define {name} {{{hi!r}, {lo!r}}}"


def table(name, vals):
    body = ",\n    ".join("{%r, %r}" % split(v) for v in vals)
    return f"static __device__ __constant__ DD {name}[{len(vals)}] = {{\n    {body}}};"


def main():
    out = ["// Generated by gen_dd_consts.py -- do not edit.", "#pragma once",
           f"#define DD_NFACT {NFACT}", f"#define DD_NSERIES {NSERIES}",
           fmt("DD_PI", mpmath.pi), fmt("DD_PI_2", mpmath.pi / 2), fmt("DD_2_PI", 2 / mpmath.pi),
           fmt("DD_EULER", mpmath.euler), fmt("DD_LN2", mpmath.log(2))]
    out.append(table("dd_inv_fact", [1 / mpmath.factorial(n) for n in range(NFACT)]))
    rk2 = [0] + [mpmath.mpf(1) / (k * k) for k in range(1, NSERIES + 1)]
    rkk1 = [0] + [mpmath.mpf(1) / (k * (k + 1)) for k in range(1, NSERIES + 1)]
    H = [mpmath.mpf(0)]
    for k in range(1, NSERIES + 2):
        H.append(H[-1] + mpmath.mpf(1) / k)
    out.append(table("dd_rk2", rk2))
    out.append(table("dd_rkk1", rkk1))
    out.append(table("dd_hk", H[: NSERIES + 1]))
    out.append(table("dd_hh", [H[k] + H[k + 1] for k in range(NSERIES + 1)]))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dd_consts.h")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
