"""Bessel and Hankel functions of orders 0 and 1 for real z > 0.

Written from the textbook definitions (Abramowitz & Stegun, ch. 9), not from
any library's constants:

* z <= 4: ascending series (A&S 9.1.10, 9.1.11 with 9.1.13 for Y0, Y1);
* 4 < z <= 25: Miller's backward recurrence for J_n normalised by
  J0 + 2 sum_k J_2k = 1 (A&S 9.1.46 / 9.12), then the Neumann series
  Y0 = (2/pi)[(ln(z/2) + gamma) J0 - 2 sum_k (-1)^k J_2k / k] (A&S 9.1.88) and its
  derivative for Y1 = -Y0';
* z > 25: Hankel's asymptotic expansion with P, Q in powers of 1/(8z)
  (A&S 9.2.5-9.2.10), summed until the terms drop below the working epsilon.

The routines work in the dtype of their argument: float64 for the pair sums
and numpy.longdouble (x86 80-bit, 64-bit mantissa) for the correction setup.
Used for the Green's function G(x, y) = (i/4) H0^(1)(k|x - y|) (Section 2).
"""
import numpy as np

_PI_S = "3.14159265358979323846264338327950288419716939937510"
_GAMMA_S = "0.57721566490153286060651209008240243104215933593992"


def _consts(dt):
    return dt.type(_PI_S), dt.type(_GAMMA_S)


def _series(z):
    dt = z.dtype
    one = dt.type(1)
    PI, EG = _consts(dt)
    q = -(z * z) / 4
    j0 = np.ones_like(z)
    j1 = np.ones_like(z)           # J1 = (z/2) sum_k q^k / (k! (k+1)!)
    t0 = np.ones_like(z)
    t1 = np.ones_like(z)
    hk = np.zeros_like(z)          # harmonic number H_k
    sy0 = np.zeros_like(z)         # sum_{k>=1} (-1)^{k+1} H_k (z^2/4)^k / (k!)^2
    sy1 = np.ones_like(z)          # sum_k (H_k + H_{k+1}) q^k / (k! (k+1)!), k = 0 term is 1
    for kk in range(1, 45):
        t0 = t0 * q / (kk * kk)
        t1 = t1 * q / (kk * (kk + 1))
        j0 = j0 + t0
        j1 = j1 + t1
        hk = hk + one / kk
        sy0 = sy0 - hk * t0        # (-1)^{k+1} (z^2/4)^k = -q^k
        sy1 = sy1 + (hk + hk + one / (kk + 1)) * t1
    j1 = j1 * (z / 2)
    L = np.log(z / 2) + EG
    y0 = (2 / PI) * (L * j0 + sy0)
    y1 = (-2 / (PI * z)) + (2 / PI) * L * j1 - (z / (2 * PI)) * sy1       # A&S 9.1.11, n = 1
    return j0, j1, y0, y1


def _miller(z):
    """Normalised J0, J1 by backward recurrence, Y0 and Y1 by Neumann series."""
    dt = z.dtype
    PI, EG = _consts(dt)
    nstart = int(2 * ((int(np.max(z)) + 44) // 2))
    J = np.zeros((nstart + 2,) + z.shape, dtype=dt)
    J[nstart] = dt.type("1e-200")
    for n in range(nstart, 0, -1):
        J[n - 1] = (2 * n / z) * J[n] - J[n + 1]
        big = np.abs(J[n - 1]) > dt.type("1e200")
        if np.any(big):
            J[n - 1:] = J[n - 1:] * np.where(big, dt.type("1e-200"), dt.type(1))
    norm = J[0] + 2 * np.sum(J[2:nstart + 1:2], axis=0)
    J = J / norm
    ks = np.arange(1, nstart // 2 + 1)
    coef = ((-1.0) ** ks).astype(dt) / ks.astype(dt)
    s0 = np.tensordot(coef, J[2 * ks], axes=(0, 0))
    # Y1 = -(Y0)' = (2/pi)[-J0/z + (ln(z/2)+gamma) J1 + sum_k (-1)^k (J_{2k-1} - J_{2k+1}) / k]
    s1 = np.tensordot(coef, J[2 * ks - 1] - J[2 * ks + 1], axes=(0, 0))
    L = np.log(z / 2) + EG
    j0, j1 = J[0], J[1]
    y0 = (2 / PI) * (L * j0 - 2 * s0)
    y1 = (2 / PI) * (-j0 / z + L * j1 + s1)
    return j0, j1, y0, y1


def _asymptotic(z):
    dt = z.dtype
    PI, _ = _consts(dt)
    eps = np.finfo(dt).eps / 16
    cz, sz = np.cos(z), np.sin(z)
    r2 = np.sqrt(dt.type(0.5))
    amp = np.sqrt(2 / (PI * z))
    out = []
    for nu in (0, 1):
        mu = 4 * nu * nu
        P = np.ones_like(z)
        Q = np.zeros_like(z)
        term = np.ones_like(z)
        for kk in range(1, 80):
            term = term * (mu - (2 * kk - 1) ** 2) / (kk * 8 * z)
            if kk % 2 == 1:
                Q = Q + ((-1) ** ((kk - 1) // 2)) * term
            else:
                P = P + ((-1) ** (kk // 2)) * term
            if np.max(np.abs(term)) < eps:
                break
        # cos/sin of chi = z - (nu/2 + 1/4) pi from cos z, sin z (no rounding of chi)
        if nu == 0:
            c, s = r2 * (cz + sz), r2 * (sz - cz)
        else:
            c, s = r2 * (sz - cz), -r2 * (sz + cz)
        out.append(amp * (P * c - Q * s))
        out.append(amp * (P * s + Q * c))
    j0, y0, j1, y1 = out
    return j0, j1, y0, y1


def bessel01(z):
    """(J0, J1, Y0, Y1) at real z > 0, any shape; float64 unless z is longdouble."""
    z = np.asarray(z)
    if z.dtype != np.longdouble:
        z = z.astype(np.float64)
    shape = z.shape
    z = z.ravel()
    if np.any(z <= 0):
        raise ValueError("bessel01 needs z > 0")
    res = [np.empty_like(z) for _ in range(4)]
    for mask, fn in ((z <= 4, _series), ((z > 4) & (z <= 25), _miller), (z > 25, _asymptotic)):
        if np.any(mask):
            vals = fn(z[mask])
            for r, v in zip(res, vals):
                r[mask] = v
    return tuple(r.reshape(shape) for r in res)


def hankel01(z):
    """(H0^(1)(z), H1^(1)(z)) = (J0 + i Y0, J1 + i Y1) at real z > 0."""
    j0, j1, y0, y1 = bessel01(z)
    return j0 + 1j * y0, j1 + 1j * y1


def green(k, r):
    """Helmholtz Green's function (i/4) H0^(1)(k r), r > 0 (Section 2)."""
    h0, _ = hankel01(k * np.asarray(r))
    return 0.25j * h0
