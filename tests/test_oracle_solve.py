"""Pins of the oracle's operator, GMRES and far field: dense LU, the Mie series,
convergence under refinement, the energy balance (Eq. dissipativity_identity)."""
import numpy as np
import pytest

from lsinput.workloads import constant_disk
from oracle.farfield import far_field, mie_far_field, mie_interior
from oracle.gmres import gmres
from oracle.operator import Operator, plane_wave


@pytest.fixture(scope="module")
def disk_solutions():
    out = {}
    for nr in (2, 3):
        wl = constant_disk(k=5.0, n_rings=nr)
        op = Operator(wl.mesh, wl.k, wl.m, kappa=3.0)
        b = plane_wave(wl.mesh.nodes, wl.k, 0.0)
        u, hist, it = gmres(op.apply, b, tol=1e-12)
        out[nr] = (wl, op, b, u, hist, it)
    return out


def test_gmres_matches_dense_lu(disk_solutions):
    wl, op, b, u, hist, it = disk_solutions[2]
    ud = np.linalg.solve(op.dense(), b)
    assert np.max(np.abs(u - ud)) < 1e-10 * np.max(np.abs(ud))
    assert hist[-1] <= 1e-12 and it < 100
    # the Givens estimate is the true residual
    assert np.linalg.norm(b - op.apply(u)) / np.linalg.norm(b) < 1e-11


def test_mie_and_refinement(disk_solutions):
    errs = []
    for nr in (2, 3):
        wl, op, b, u, _, _ = disk_solutions[nr]
        ref = mie_interior(wl.mesh.nodes, wl.k, 1.5)
        errs.append(np.max(np.abs(u - ref)) / np.max(np.abs(ref)))
    assert errs[1] < 5e-4
    # h ratio 3/2; order p + 3 = 7 expected (Section 3); demand at least 6
    assert errs[0] / errs[1] > 1.5**6


def test_far_field_vs_mie(disk_solutions):
    wl, op, b, u, _, _ = disk_solutions[3]
    uinf = far_field(wl.mesh.nodes, wl.mesh.weights, wl.m, u, wl.k, wl.ff_angles)
    ref = mie_far_field(wl.ff_angles, wl.k, 1.5)
    assert np.max(np.abs(uinf - ref)) / np.max(np.abs(ref)) < 5e-4


def test_mie_energy_balance():
    # lossless disk: Im int conj(m u) u_inc = (1/k) ||u_inf||^2 (Eq. dissipativity_identity);
    # both sides from the Mie series alone, integrated by a fine polar rule
    k, n_opt = 5.0, 1.5
    rr, wr = np.polynomial.legendre.leggauss(80)
    rr, wr = (rr + 1) / 2, wr / 2
    th = 2 * np.pi * np.arange(256) / 256
    R, T = np.meshgrid(rr, th, indexing="ij")
    pts = np.stack([(R * np.cos(T)).ravel(), (R * np.sin(T)).ravel()], 1)
    w = (np.outer(wr * rr, np.full(256, 2 * np.pi / 256))).ravel()
    u = mie_interior(pts, k, n_opt)
    m = 1 - n_opt**2
    lhs = np.imag(np.sum(w * np.conj(m * u) * np.exp(1j * k * pts[:, 0])))
    uinf = mie_far_field(th, k, n_opt)
    rhs = np.sum(np.abs(uinf) ** 2) * 2 * np.pi / 256 / k
    assert abs(lhs - rhs) < 1e-12 * rhs


def test_discrete_energy_balance(disk_solutions):
    wl, op, b, u, _, _ = disk_solutions[3]
    uinf = far_field(wl.mesh.nodes, wl.mesh.weights, wl.m, u, wl.k, wl.ff_angles)
    lhs = np.imag(np.sum(wl.mesh.weights * np.conj(wl.m * u) * b))
    rhs = np.sum(np.abs(uinf) ** 2) * 2 * np.pi / len(wl.ff_angles) / wl.k
    assert abs(lhs - rhs) < 1e-4 * rhs
