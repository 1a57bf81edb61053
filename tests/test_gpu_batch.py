"""GPU batching form: R right-hand sides per launch (FP32 table; CUDA-core kernel
or the tensor-core GEMM with iterative refinement, the default).

Target: <= 1e-6 relative solution error against the FP64 path (and the FP64
oracle on a small case); the CUDA-core batched pair sum matches the FP64 one to
~1e-7, the tensor-core one within its truncation bound (tests/test_gpu_tc.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_17615_b300 as L
from lsinput.workloads import constant_disk, random_density, star_scatterer, two_material
from oracle.operator import Operator as OracleOp, plane_wave


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex128)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("kind,bar", [(0, 5e-7), (1, 2e-6)])        # kind 1: run length 4, bound 5e-7 per stage run
def test_batched_pairsum_matches_fp64(kind, bar):
    wl = two_material("tiny", k=8.0)
    n = wl.mesh.n_nodes
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0)
    op.set_batch_kernel(kind)
    R = 13                                         # two RHS blocks, the second ragged
    F = _dev(np.stack([random_density(n, 100 + r) for r in range(R)]))
    Y = torch.empty_like(F)
    op.pairsum_batch_dev(F, Y)
    for r in (0, 7, 12):
        y1 = torch.empty_like(F[r])
        op.pairsum_dev(F[r].contiguous(), y1)
        err = (torch.linalg.norm(Y[r] - y1) / torch.linalg.norm(y1)).item()
        assert err < bar, (r, err)


def test_batched_solve_star():
    # a scatterer of the batched workload (star with an inner interface), 16 directions
    wl = star_scatterer(1, 6000, k=10.0, nx=96, ny=96)
    n = wl.mesh.n_nodes
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, box=wl.box, nx=wl.nx, ny=wl.ny, tol=1e-9)
    dirs = wl.directions[::4]
    B = torch.empty((dirs.size, n), dtype=torch.complex128, device="cuda")
    op.incident_dev(dirs, B)
    U = torch.empty_like(B)
    Uinf = torch.empty((dirs.size, wl.ff_angles.size), dtype=torch.complex128, device="cuda")
    iters, st = op.solve_batch_dev(B, U, wl.ff_angles, Uinf)
    assert st == L.LS_OK
    u1 = torch.empty_like(B[0])
    u32 = torch.empty_like(B[0])
    uinf1 = torch.empty((1, wl.ff_angles.size), dtype=torch.complex128, device="cuda")
    op32 = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, box=wl.box, nx=wl.nx, ny=wl.ny, tol=1e-9, pairsum=2)
    worst, worst32 = 0.0, 0.0
    for r in (0, 5, dirs.size - 1):
        it1, st1 = op.solve_dev(B[r].contiguous().view(1, -1), u1.view(1, -1), wl.ff_angles, uinf1)
        op32.solve_dev(B[r].contiguous().view(1, -1), u32.view(1, -1))
        worst = max(worst, (torch.linalg.norm(U[r] - u1) / torch.linalg.norm(u1)).item())
        worst32 = max(worst32, (torch.linalg.norm(u32 - u1) / torch.linalg.norm(u1)).item())
    print("batched star: iterations", iters.min(), iters.max(), "max rel err vs FP64", worst,
          "(single-RHS precision form:", worst32, ")")
    assert worst < 1e-6


def test_batched_solve_vs_oracle_small():
    wl = constant_disk(k=5.0, n_rings=3, nx=48, ny=48)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=48, ny=48, tol=1e-10)
    dirs = np.array([0.0, 1.0, 2.0])
    B = torch.empty((3, wl.mesh.n_nodes), dtype=torch.complex128, device="cuda")
    op.incident_dev(dirs, B)
    U = torch.empty_like(B)
    iters, st = op.solve_batch_dev(B, U)
    assert st == L.LS_OK
    Ld = OracleOp(wl.mesh, wl.k, wl.m).dense()
    for r, d in enumerate(dirs):
        ud = np.linalg.solve(Ld, plane_wave(wl.mesh.nodes, wl.k, d))
        assert np.linalg.norm(U[r].cpu().numpy() - ud) / np.linalg.norm(ud) < 1e-6


@pytest.mark.parametrize("kind", [0, 1])
def test_multi_scatterer_persistent(kind):
    # three stars of uneven size and different k in one lock-step solve; each must
    # match its own batched solve (same arithmetic per unit, different launch form)
    R = 8
    ops, B, U = [], [], []
    for s, nn, kk in ((0, 2000, 8.0), (1, 5000, 10.0), (2, 9000, 12.0)):
        wl = star_scatterer(s, nn, k=kk, nx=64, ny=64)
        op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, box=wl.box, nx=wl.nx, ny=wl.ny, tol=1e-8)
        op.set_batch_kernel(kind)                  # 0: CUDA-core persistent kernel, 1: tensor cores
        b = torch.empty((R, wl.mesh.n_nodes), dtype=torch.complex128, device="cuda")
        op.incident_dev(wl.directions[:: wl.directions.size // R][:R], b)
        ops.append(op)
        B.append(b)
        U.append(torch.empty_like(b))
    iters, st = L.solve_multi_dev(ops, B, U)
    assert st == L.LS_OK
    for op, b, u in zip(ops, B, U):
        u1 = torch.empty_like(b)
        it1, st1 = op.solve_batch_dev(b, u1)
        assert st1 == L.LS_OK
        err = (torch.linalg.norm(u - u1) / torch.linalg.norm(u1)).item()
        assert err < 1e-12, err
    print("multi-scatterer iterations per scatterer:", [list(i) for i in iters])
