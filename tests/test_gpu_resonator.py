"""The open-cavity resonator (Section 6, more general examples) at small k on the GPU:
the preconditioned solve against the oracle's dense solve (GMRES tolerance x condition
factor), and the energy balance of Eq. dissipativity_identity for this lossless
(real) contrast, Im sum_j w_j conj(m_j u_j) b_j = ||u_inf||^2 / k, to the discretisation
level (the field is trapped in the cavity, so the balance is the check of the far field
and of the solution together)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_17615_b300 as L
from lsinput.workloads import open_resonator
from oracle.operator import Operator as OracleOp, plane_wave


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_open_resonator_solve():
    wl = open_resonator(k=10.0, n_s=2, n_theta=30, nx=64, ny=64)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=64, ny=64, tol=1e-10)
    ff = 2 * np.pi * np.arange(256) / 256
    u, uinf, _, it, st = op.solve(wl.directions, ff)
    print("open resonator k=10 preconditioned iterations", it[0])
    assert st == L.LS_OK
    b = plane_wave(wl.mesh.nodes, wl.k, np.pi)
    ud = np.linalg.solve(OracleOp(wl.mesh, wl.k, wl.m).dense(), b)
    assert np.linalg.norm(u[0] - ud) < 1e-8 * np.linalg.norm(ud)
    lhs = np.imag(np.sum(wl.mesh.weights * np.conj(wl.m * u[0]) * b))
    rhs = np.sum(np.abs(uinf[0]) ** 2) * 2 * np.pi / ff.size / wl.k
    assert abs(lhs - rhs) < 1e-3 * rhs
