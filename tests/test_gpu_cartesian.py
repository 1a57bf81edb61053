"""Purely Cartesian operator (ls_cartesian_create) against the oracle's CartesianLS:
L^(C) by FFT convolution and S^(C) applies to the FP64 matvec bar 1e-11 on a ragged,
non-square grid, and the preconditioned solve of the structured disk to the GMRES
tolerance times a condition factor, with the same iteration count."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_17615_b300 as L
from lsinput.workloads import random_density
from oracle.cartesian import CartesianLS
from oracle.precond import Grid


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_cartesian_apply_parity():
    box, nx, ny, k = (-1.0, 1.0, -0.9, 0.9), 41, 37, 9.0
    g = Grid(box, nx, ny)
    pts = g.points()
    m = np.where(np.hypot(pts[:, 0], pts[:, 1]) < 0.7, 1 - 1.5**2, 0.0).astype(np.complex128)
    ora = CartesianLS(g, k, m)
    op = L.CartesianOperator(k, m, box=box, nx=nx, ny=ny)
    x = random_density(g.n, 90)
    assert _rel(op.apply(x), ora.apply(x)) < 1e-11
    assert _rel(op.apply_precond(x), ora.S(x)) < 1e-11
    # L^T: V^(C) is symmetric, so L^T x = x + k^2 m V x
    assert _rel(op.apply_transpose(x), x + k**2 * m * ora.potential(x)) < 1e-11


def test_cartesian_disk_solve():
    k, n_opt, hk = 5.0, 1.5, 0.125
    h = hk / k
    n = int(round(4.0 / h)) + 1
    box = (-2.0, 2.0, -2.0, 2.0)
    g = Grid(box, n, n)
    pts = g.points()
    m = np.where(np.hypot(pts[:, 0], pts[:, 1]) < 1.0, 1 - n_opt**2, 0.0).astype(np.complex128)
    op = L.CartesianOperator(k, m, box=box, nx=n, ny=n, tol=1e-8)
    u, _, _, it, st = op.solve([0.0])
    ora = CartesianLS(g, k, m)
    uo, _, ito = ora.solve(np.exp(1j * k * pts[:, 0]), tol=1e-8)
    print("structured disk k=5 iterations GPU / oracle", it[0], ito)
    assert st == L.LS_OK and abs(int(it[0]) - ito) <= 1
    assert _rel(u[0], uo) < 1e-7
