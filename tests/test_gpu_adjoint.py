"""GPU differentiation form: transposed operators, adjoint solve, misfit gradient.

Targets: transposed applies satisfy y^T (A x) = (A^T y)^T x to rounding; the
gradient matches the oracle's dense adjoint-state gradient and central finite
differences of the GPU misfit (h = 1e-6) to <= 1e-5 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_17615_b300 as L
from paper_2608_17615_b300.misfit import far_field_misfit
from lsinput.workloads import constant_disk, random_density, two_material
from oracle.adjoint import DenseMisfit, far_field_matrix
from oracle.operator import Operator as OracleOp, plane_wave


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex128)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bil(a, b):
    return torch.sum(a * b).item()


def test_transposes_are_transposes():
    wl = two_material("tiny", k=8.0, nx=48, ny=48)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=48, ny=48)
    n = wl.mesh.n_nodes
    x = _dev(random_density(n, 1))
    y = _dev(random_density(n, 2))
    for fwd, tr in ((op.apply_dev, op.apply_transpose_dev), (op.apply_precond_dev, op.apply_precond_transpose_dev)):
        ax = torch.empty_like(x)
        aty = torch.empty_like(y)
        fwd(x, ax)
        tr(y, aty)
        lhs, rhs = _bil(y, ax), _bil(aty, x)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # V^T against the oracle's dense potential matrix
    ora = OracleOp(wl.mesh, wl.k, wl.m)
    V = ora.naive_matrix() + ora.dV.toarray()
    vt = torch.empty_like(x)
    op.potential_transpose_dev(x, vt)
    ref = V.T @ x.cpu().numpy()
    assert np.linalg.norm(vt.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-11


def test_adjoint_solve_residual():
    wl = two_material("tiny", k=8.0, nx=48, ny=48)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=48, ny=48, tol=1e-10)
    g = _dev(random_density(wl.mesh.n_nodes, 3)).view(1, -1)
    lam = torch.empty_like(g)
    iters, st = op.solve_transpose_dev(g, lam)
    assert st == L.LS_OK
    r = torch.empty_like(lam[0])
    op.apply_transpose_dev(lam[0], r)
    assert (torch.linalg.norm(r - g[0]) / torch.linalg.norm(g[0])).item() < 1e-8


def _problem():
    wl = constant_disk(k=6.0, n_rings=2, nx=32, ny=32)      # 360 nodes
    x, y = wl.mesh.nodes[:, 0], wl.mesh.nodes[:, 1]
    m = 1 - (1.4 + 0.2 * np.exp(-(x**2 + y**2) / 0.2)) ** 2
    mg_pts = wl.grid_points
    rg = np.hypot(mg_pts[:, 0], mg_pts[:, 1])
    m_grid = np.where(rg < 1, 1 - (1.4 + 0.2 * np.exp(-rg**2 / 0.2)) ** 2, 0).astype(complex)
    ff = 2 * np.pi * np.arange(8) / 8
    dirs = [0.0, np.pi / 3]
    blob = 0.05 * np.exp(-((x + 0.3) ** 2 + (y + 0.2) ** 2) / 0.02)
    mt = 1 - (np.sqrt(1 - m) + blob) ** 2
    return wl, m, m_grid, ff, dirs, mt


def test_gradient_vs_oracle_and_fd():
    wl, m, m_grid, ff, dirs, mt = _problem()
    ora = OracleOp(wl.mesh, wl.k, m.astype(complex))
    V = ora.naive_matrix() + ora.dV.toarray()
    A = far_field_matrix(wl.mesh.nodes, wl.mesh.weights, wl.k, ff)
    b = [plane_wave(wl.mesh.nodes, wl.k, d) for d in dirs]
    Lt = np.eye(m.size) + wl.k**2 * V * mt[None, :]
    targets = np.stack([A @ (mt * np.linalg.solve(Lt, bb)) for bb in b])
    g_ref = DenseMisfit(V, wl.k, b, A, list(targets)).gradient(m)

    op = L.Operator(L.Mesh(wl.mesh), wl.k, m.astype(complex), m_grid, nx=32, ny=32, tol=1e-12)
    mt_t = torch.from_numpy(m).cuda().requires_grad_(True)
    tg = _dev(targets)
    J = far_field_misfit(mt_t, op, dirs, ff, tg)
    (grad,) = torch.autograd.grad(J, mt_t)
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-8

    # central differences of the GPU misfit on 20 seeded nodes
    rng = np.random.default_rng(7)
    idx = rng.choice(m.size, 20, replace=False)
    h = 1e-6
    errs = []
    for j in idx:
        e = np.zeros(m.size)
        e[j] = h
        jp = far_field_misfit(torch.from_numpy(m + e).cuda(), op, dirs, ff, tg).item()
        jm = far_field_misfit(torch.from_numpy(m - e).cuda(), op, dirs, ff, tg).item()
        errs.append(abs((jp - jm) / (2 * h) - g[j]))
    rel = max(errs) / np.max(np.abs(g))
    print("gradient: oracle rel", np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref), "FD rel", rel)
    assert rel < 1e-5


def test_batched_adjoint_solve_matches_single():
    """Lock-step transposed solves (FP32 batched pair sum) against the FP64 single solves."""
    wl = two_material("tiny", k=8.0, nx=48, ny=48)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=48, ny=48, tol=1e-10)
    n = wl.mesh.n_nodes
    g = _dev(np.stack([random_density(n, 10 + r) for r in range(5)]))
    lam = torch.empty_like(g)
    op.solve_transpose_dev(g, lam)
    lam_b = torch.empty_like(g)
    iters, st = op.solve_transpose_batch_dev(g, lam_b)
    assert st == L.LS_OK
    assert (iters > 0).all()
    err = (torch.linalg.norm(lam_b - lam, dim=1) / torch.linalg.norm(lam, dim=1)).max().item()
    print("batched adjoint: iterations", iters, "max rel err vs FP64", err)
    assert err < 1e-5


def test_batched_gradient_vs_oracle():
    """Precision form of the differentiation pipeline: batched forward and adjoint solves."""
    wl, m, m_grid, ff, dirs, mt = _problem()
    dirs = [0.0, np.pi / 3, np.pi / 2, 2.0, 4.0]
    ora = OracleOp(wl.mesh, wl.k, m.astype(complex))
    V = ora.naive_matrix() + ora.dV.toarray()
    A = far_field_matrix(wl.mesh.nodes, wl.mesh.weights, wl.k, ff)
    b = [plane_wave(wl.mesh.nodes, wl.k, d) for d in dirs]
    Lt = np.eye(m.size) + wl.k**2 * V * mt[None, :]
    targets = np.stack([A @ (mt * np.linalg.solve(Lt, bb)) for bb in b])
    g_ref = DenseMisfit(V, wl.k, b, A, list(targets)).gradient(m)

    op = L.Operator(L.Mesh(wl.mesh), wl.k, m.astype(complex), m_grid, nx=32, ny=32, tol=1e-10)
    mt_t = torch.from_numpy(m).cuda().requires_grad_(True)
    J = far_field_misfit(mt_t, op, dirs, ff, _dev(targets), batched=True)
    (grad,) = torch.autograd.grad(J, mt_t)
    rel = np.linalg.norm(grad.cpu().numpy() - g_ref) / np.linalg.norm(g_ref)
    J_ref = DenseMisfit(V, wl.k, b, A, list(targets)).value(m)
    print("batched gradient: rel err vs oracle", rel, "misfit rel err", abs(J.item() - J_ref) / J_ref)
    assert rel < 1e-5
    assert abs(J.item() - J_ref) <= 1e-5 * J_ref
