"""Diagnostics on the GPU against the oracle: Ritz values of the GMRES Hessenberg
(ls_op_ritz) and the rho sampling of the Approach II preconditioner (ls_precond_rho_dev).

Ritz values: the library's Arnoldi (classical Gram-Schmidt twice) and the oracle's (modified
Gram-Schmidt, two passes) span the same Krylov space, so after the same 30 steps their
Ritz values agree up to the rounding of the two orthogonalisations (bar 1e-8 of the
spectral radius, each library value matched to its nearest oracle value); the
preconditioned values cluster around 1 (Figure ritz_spectrum).  rho: same vectors, same
formula, so the FP64 bar 1e-11."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_17615_b300 as L
from lsinput.workloads import constant_disk
from oracle.gmres import ritz_values
from oracle.operator import Operator, plane_wave
from oracle.precond import Grid, Preconditioner


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_ritz_values_match_oracle():
    wl = constant_disk(k=10.0, n_rings=3, nx=48, ny=48)
    M = L.Mesh(wl.mesh)
    b = plane_wave(wl.mesh.nodes, wl.k, 0.0)
    ora = Operator(wl.mesh, wl.k, wl.m)
    P = Preconditioner(Grid(wl.box, wl.nx, wl.ny), wl.mesh.nodes, wl.k, wl.m_grid)
    spreads = {}
    for prec in (0, 1):
        op = L.Operator(M, wl.k, wl.m, wl.m_grid, nx=48, ny=48, use_precond=prec, tol=1e-15, max_iter=30)
        op.solve([0.0])
        rl = op.ritz()
        ro = ritz_values(ora.apply, b, 30, apply_P=P.apply if prec else None)
        assert rl.size == ro.size == 30
        d = np.abs(rl[:, None] - ro[None, :]).min(axis=1)
        assert np.max(d) < 1e-8 * np.max(np.abs(ro))
        spreads[prec] = np.median(np.abs(rl - 1))
    assert spreads[1] < 0.5 * spreads[0]


def test_rho_matches_oracle():
    wl = constant_disk(k=10.0, n_rings=6, nx=25, ny=25)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=25, ny=25)
    P = Preconditioner(Grid(wl.box, wl.nx, wl.ny), wl.mesh.nodes, wl.k, wl.m_grid)
    rng = np.random.default_rng(8)
    X = (rng.standard_normal((16, 625)) + 1j * rng.standard_normal((16, 625))) / np.sqrt(2)
    rho = op.precond_rho_dev(torch.from_numpy(X).cuda())
    for s in range(16):
        w = P.TQC @ (P.T @ X[s])
        Sw = P.lu.solve(P.A @ w)
        ref = np.sum(P.D * np.conj(Sw) * w) / np.sum(P.D * np.abs(w) ** 2)
        assert abs(rho[s] - ref) < 1e-11 * abs(ref)
    assert np.all(rho.imag < 0)          # contrast m = 1 - 1.5^2 < 0 (the appendix's sign)
