"""Pins of the oracle's diagnostics (Section 6 and the appendix on invertibility).

* Ritz values: a full Arnoldi process on a small system reproduces the spectrum of the
  matrix; and, as Figure ritz_spectrum shows, the preconditioned Ritz values cluster
  around 1 more tightly than the unpreconditioned ones.
* rho sampling (Eq. rho_def): for a constant contrast the imaginary part of
  rho(w) = <S^(C) w, w>_D / ||w||_D^2 over w in the range of the round trip R_II carries
  the sign of the contrast m0 = 1 - n0 (the appendix: below zero for n0 > 1, above for
  n0 < 1), at k = 10, k h_C = 1.
"""
import numpy as np

from lsinput.workloads import constant_disk
from oracle.diagnostics import rho_samples
from oracle.gmres import ritz_values
from oracle.operator import Operator, plane_wave
from oracle.precond import Grid, Preconditioner


def test_full_arnoldi_ritz_values_are_the_spectrum():
    wl = constant_disk(k=5.0, n_rings=1)
    op = Operator(wl.mesh, wl.k, wl.m)
    n = wl.mesh.n_nodes
    b = plane_wave(wl.mesh.nodes, wl.k, 0.0) + 0.3 * np.exp(1j * np.arange(n))
    rv = ritz_values(op.apply, b, n)
    ev = np.linalg.eigvals(op.dense())
    d = np.abs(rv[:, None] - ev[None, :]).min(axis=1)
    assert rv.size == n and np.max(d) < 1e-9 * np.max(np.abs(ev))


def test_preconditioned_ritz_values_cluster_at_one():
    wl = constant_disk(k=10.0, n_rings=3, nx=48, ny=48)
    op = Operator(wl.mesh, wl.k, wl.m)
    P = Preconditioner(Grid(wl.box, wl.nx, wl.ny), wl.mesh.nodes, wl.k, wl.m_grid)
    b = plane_wave(wl.mesh.nodes, wl.k, 0.0)
    r_u = ritz_values(op.apply, b, 30)
    r_p = ritz_values(op.apply, b, 30, apply_P=P.apply)
    spread_u, spread_p = np.median(np.abs(r_u - 1)), np.median(np.abs(r_p - 1))
    print("median |ritz - 1|: unpreconditioned", spread_u, "preconditioned", spread_p)
    assert spread_p < 0.5 * spread_u


def test_rho_imaginary_part_carries_the_contrast_sign():
    for n0, sign in ((1.5**2, -1.0), (0.8, 1.0)):
        wl = constant_disk(k=10.0, n_opt=np.sqrt(n0), n_rings=6, nx=25, ny=25)
        rho = rho_samples(Grid(wl.box, wl.nx, wl.ny), wl.mesh.nodes, wl.k, wl.m_grid, 200, seed=5)
        assert np.all(sign * rho.imag > 0), (n0, rho.imag.min(), rho.imag.max())
