"""Pins of the oracle's purely Cartesian solver (Section 6, comparison with a purely
Cartesian discretization; Table struct_vs_fitted).

* The FFT convolution of V^(C) equals the plain double sum over the grid (a ragged,
  non-square grid, so that a transposed axis or a wrong padding fails).
* On the constant-contrast disk (eta = 1.25, k = 5) with k h_C = 0.125 on [-2, 2]^2:
  the S^(C)-preconditioned GMRES takes few iterations (the paper: 6) against many
  unpreconditioned (the paper: 28), and the error against the Mie series at the interior
  grid nodes stalls at the 1e-2 level (the paper: 2.1e-2) because the grid cannot resolve
  the jump of the contrast across the circle.
"""
import numpy as np

from oracle.cartesian import CartesianLS
from oracle.farfield import mie_interior
from oracle.precond import Grid


def _disk_grid(k, hk=0.125, half=2.0):
    h = hk / k
    n = int(round(2 * half / h)) + 1
    g = Grid((-half, half, -half, half), n, n)
    pts = g.points()
    inside = np.hypot(pts[:, 0], pts[:, 1]) < 1.0
    return g, pts, inside


def test_fft_convolution_matches_plain_sum():
    g = Grid((-0.5, 0.5, -0.6, 0.6), 11, 13)
    m = np.ones(g.n, np.complex128)
    C = CartesianLS(g, 7.0, m)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(g.n) + 1j * rng.standard_normal(g.n)
    a, b = C.potential(f), C.potential_dense(f)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(b))


def test_structured_disk_iterations_and_accuracy():
    k, n_opt = 5.0, 1.5
    g, pts, inside = _disk_grid(k)
    m = np.where(inside, 1 - n_opt**2, 0.0).astype(np.complex128)
    C = CartesianLS(g, k, m)
    b = np.exp(1j * k * pts[:, 0])
    u, hist, it_p = C.solve(b, tol=1e-8)
    _, _, it_u = C.solve(b, tol=1e-8, precond=False)
    ref = mie_interior(pts[inside], k, n_opt)
    err = np.max(np.abs(u[inside] - ref)) / np.max(np.abs(ref))
    print("structured disk k=5: iterations", it_p, "unpreconditioned", it_u, "max error", err)
    assert it_p <= 10 and it_u >= 2 * it_p
    assert 1e-3 < err < 0.2
