"""The host-buffer and auxiliary calls of the C ABI against the oracle.

ls_solve with an explicit right-hand side, ls_apply_precond, ls_apply_transpose,
ls_solve_adjoint (host buffers), the explicit residual check of every GMRES solve
(ls_op_last_residual) against a full re-apply (ls_residual_dev), the device
contrast setter and the misfit reduction.  Bars: the FP64 matvec bar 1e-11 for
single applies, GMRES tolerance x a condition factor for solves, rounding for
the reductions.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_17615_b300 as L
from lsinput.workloads import constant_disk, random_density, two_material
from oracle.farfield import far_field
from oracle.operator import Operator as OracleOp, plane_wave
from oracle.precond import Grid, Preconditioner


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def tiny():
    wl = two_material("tiny", k=8.0, nx=48, ny=48)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=48, ny=48, tol=1e-10)
    ora = OracleOp(wl.mesh, wl.k, wl.m)
    return wl, op, ora


def test_solve_with_explicit_rhs(tiny):
    wl, op, ora = tiny
    b = plane_wave(wl.mesh.nodes, wl.k, 0.4)
    u1, f1, _, it1, st1 = op.solve([0.4], wl.ff_angles)
    u2, f2, _, it2, st2 = op.solve(b=b[None, :], ff_angles=wl.ff_angles)
    assert st1 == st2 == L.LS_OK and it1[0] == it2[0]
    assert _rel(u2[0], u1[0]) < 1e-12 and _rel(f2[0], f1[0]) < 1e-12
    # a non-plane-wave right-hand side against the oracle's dense solve
    g = random_density(wl.mesh.n_nodes, 31)
    u3, _, _, _, st3 = op.solve(b=g[None, :])
    assert st3 == L.LS_OK
    assert _rel(u3[0], np.linalg.solve(ora.dense(), g)) < 1e-8


def test_host_apply_precond_and_transpose(tiny):
    wl, op, ora = tiny
    x = random_density(wl.mesh.n_nodes, 32)
    P = Preconditioner(Grid(wl.box, wl.nx, wl.ny), wl.mesh.nodes, wl.k, wl.m_grid)
    assert _rel(op.apply_precond(x), P.apply(x)) < 1e-11
    assert _rel(op.apply_transpose(x), ora.dense().T @ x) < 1e-11


def test_host_adjoint_solve(tiny):
    wl, op, ora = tiny
    g = np.stack([random_density(wl.mesh.n_nodes, 40 + r) for r in range(2)])
    lam, iters, st = op.solve_adjoint(g)
    assert st == L.LS_OK
    At = ora.dense().T
    for r in range(2):
        assert _rel(lam[r], np.linalg.solve(At, g[r])) < 1e-8


def test_explicit_residual_check(tiny):
    wl, op, _ = tiny
    n = wl.mesh.n_nodes
    b = torch.from_numpy(plane_wave(wl.mesh.nodes, wl.k, 1.1)).cuda().view(1, -1)
    u = torch.empty_like(b)
    it, st = op.solve_dev(b, u)
    assert st == L.LS_OK
    r_exit = op.last_residual()
    r_full = op.residual_dev(b[0], u[0])
    print("explicit exit residual", r_exit, "full re-apply", r_full)
    assert 0 < r_exit <= 1e-9 and r_full <= 1e-9
    # both measure ||P(b - L u)|| / ||P b||; they differ only by the rounding of the products
    assert abs(r_exit - r_full) <= 1e-12


def test_contrast_from_device_and_misfit(tiny):
    wl, op, _ = tiny
    n = wl.mesh.n_nodes
    x = torch.from_numpy(random_density(n, 50)).cuda()
    y_host, y_dev = torch.empty_like(x), torch.empty_like(x)
    m2 = np.real(wl.m) * 0.9
    op.set_contrast(m2.astype(np.complex128))
    op.apply_dev(x, y_host)
    op.set_contrast_dev(torch.from_numpy(m2).cuda())
    op.apply_dev(x, y_dev)
    op.set_contrast(wl.m)
    assert torch.equal(y_host, y_dev)
    uinf = torch.from_numpy(np.stack([random_density(32, 60 + r) for r in range(3)])).cuda()
    tgt = torch.from_numpy(np.stack([random_density(32, 70 + r) for r in range(3)])).cuda()
    res = torch.empty_like(uinf)
    J = op.misfit_dev(uinf, tgt, res)
    d = (uinf - tgt).cpu().numpy()
    assert torch.equal(res, uinf - tgt)
    assert abs(J - 0.5 * np.sum(np.abs(d) ** 2)) <= 1e-14 * J


def test_double_float_preconditioner_blocks(tiny):
    """The FP32 and mixed forms apply P with the cyclic-reduction blocks in double-float
    (pairs of FP32, ~2^-44 per operation); against the oracle's P that stays within the
    a-priori bound cond_1(C) x 2^-44 ~ 1e-8 (cond_1(C) ~ 2e5), and the forms that take it
    cannot see it (FP32 operator error ~1e-7; the mixed form certifies with the
    double-float operator).  P of the FP64-accurate form keeps complex128 blocks."""
    wl, op, ora = tiny
    x = random_density(wl.mesh.n_nodes, 33)
    P = Preconditioner(Grid(wl.box, wl.nx, wl.ny), wl.mesh.nodes, wl.k, wl.m_grid)
    ref = P.apply(x)
    out = {}
    for mode in (2, 4):
        opm = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=48, ny=48, tol=1e-10, pairsum=mode)
        out[mode] = _rel(opm.apply_precond(x), ref)
    e64 = _rel(op.apply_precond(x), ref)
    print("P with double-float blocks vs oracle", out, "complex128 blocks", e64)
    assert e64 < 1e-11 and out[2] < 1e-9 and out[4] < 1e-9
