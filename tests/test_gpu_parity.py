"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 matvec <= 1e-11 relative L2 (the target for the FP64 form);
device Hankel <= 5e-14 relative (the series branch near z = 6 loses about two
digits to cancellation); solutions agree to the GMRES tolerance times a
condition factor.  Sizes span many pair-sum tiles and chunks with ragged tails
(3,240 / 1,800 / 40,200 nodes against tiles of 128 targets and 256 sources).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_17615_b300 as L
from lsinput.mesh import disk_mesh
from lsinput.workloads import constant_disk, random_density, two_material
from oracle.bessel import hankel01
from oracle.farfield import far_field, mie_far_field, mie_interior
from oracle.gmres import gmres
from oracle.nystrom import naive_apply
from oracle.operator import Operator as OracleOp, plane_wave
from oracle.precond import Grid, Preconditioner


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex128)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_device_hankel():
    z = np.concatenate([np.logspace(-6, 2.3, 20000), np.linspace(5.9, 6.1, 2001), np.linspace(0.5, 60, 5000)])
    zt = torch.from_numpy(z).cuda()
    out = torch.empty(z.size, dtype=torch.complex128, device="cuda")
    L.hankel0_dev(zt, out)
    h = out.cpu().numpy()
    ref, _ = hankel01(z)
    err = np.abs(h - ref) / np.abs(ref)
    assert err.max() < 5e-14, (err.max(), z[err.argmax()])


@pytest.mark.parametrize("mode", [0, 1, 3])
def test_pairsum_parity_disk(mode):
    # mode 0: tabulated H0(k sqrt(t)); 1: direct series / modulus-phase evaluation;
    # 3: the same table evaluated in double-float arithmetic on the FP32 pipe
    wl = constant_disk(k=5.0, n_rings=3)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0, pairsum=mode)
    f = random_density(wl.mesh.n_nodes, 3)
    y = torch.empty(wl.mesh.n_nodes, dtype=torch.complex128, device="cuda")
    op.pairsum_dev(_dev(f), y)
    ref = naive_apply(wl.mesh.nodes, wl.mesh.weights, wl.k, f)
    assert _rel(y.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("case", ["disk", "two_material"])
def test_apply_parity_full(case):
    if case == "disk":
        wl = constant_disk(k=5.0, n_rings=2)
    else:
        wl = two_material("tiny", k=8.0)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0)
    x = random_density(wl.mesh.n_nodes, 5)
    y = torch.empty(wl.mesh.n_nodes, dtype=torch.complex128, device="cuda")
    op.apply_dev(_dev(x), y)
    ref = OracleOp(wl.mesh, wl.k, wl.m).apply(x)
    assert _rel(y.cpu().numpy(), ref) < 1e-11
    # host-buffer entry point gives the same numbers
    assert np.array_equal(op.apply(x), y.cpu().numpy())


@pytest.fixture(scope="module")
def tm40k():
    # 40,200 nodes, k = 20, 256^2 grid; the FP64-pipe table form, the reference the other
    # arithmetics are compared with
    wl = two_material("small")
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, tol=1e-8, pairsum=0)
    return wl, op


def test_apply_parity_two_material_full_size(tm40k):
    wl, op = tm40k
    n = wl.mesh.n_nodes
    x = random_density(n, 11)
    y = torch.empty(n, dtype=torch.complex128, device="cuda")
    op.apply_dev(_dev(x), y)
    rows = np.concatenate([np.arange(0, n, 997), [n - 1]])
    ref = OracleOp(wl.mesh, wl.k, wl.m, rows_only=True).apply_rows(x, rows)
    assert _rel(y.cpu().numpy()[rows], ref) < 1e-11


def test_pairsum_table_vs_direct_full_size(tm40k):
    wl, op = tm40k
    n = wl.mesh.n_nodes
    opd = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0, pairsum=1)
    f = _dev(random_density(n, 17))
    y0 = torch.empty_like(f)
    y1 = torch.empty_like(f)
    op.pairsum_dev(f, y0)
    opd.pairsum_dev(f, y1)
    assert (torch.linalg.norm(y0 - y1) / torch.linalg.norm(y1)).item() < 1e-13


def test_double_float_form_full_size(tm40k):
    # pairsum = 3 must meet the FP64 bar: pair sum within 1e-13 of the FP64 table
    # kernel and the L apply within 1e-11 of the oracle on sampled rows
    wl, op = tm40k
    n = wl.mesh.n_nodes
    opd = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0, pairsum=3)
    f = _dev(random_density(n, 23))
    y0 = torch.empty_like(f)
    y1 = torch.empty_like(f)
    op.pairsum_dev(f, y0)
    opd.pairsum_dev(f, y1)
    e_ps = (torch.linalg.norm(y1 - y0) / torch.linalg.norm(y0)).item()
    x = random_density(n, 11)
    y = torch.empty(n, dtype=torch.complex128, device="cuda")
    opd.apply_dev(_dev(x), y)
    rows = np.concatenate([np.arange(0, n, 1999), [n - 1]])
    ref = OracleOp(wl.mesh, wl.k, wl.m, rows_only=True).apply_rows(x, rows)
    e_ap = _rel(y.cpu().numpy()[rows], ref)
    print("double-float form: pair sum vs FP64", e_ps, "apply vs oracle", e_ap)
    assert e_ps < 1e-13 and e_ap < 1e-11


@pytest.mark.parametrize("case", ["two_material_tiny", "disk", "two_material_small"])
def test_symmetric_double_float_pair_sum(case, tm40k):
    # k_pairsum_dfs (one Hankel evaluation per unordered pair, rows and columns) against
    # k_pairsum_df (every ordered pair): bitwise the same H (the coordinate differences are
    # negated exactly), the products summed in another order in double-float (48-bit
    # significand: 3.6e-15 per operation over ~100 accumulations per output), so they agree
    # within the pair-sum parity bar of 1e-13; repeated launches are bitwise identical (no
    # atomics).  Block counts: 15 (odd), 26 (even: the distance nb/2 handled once), 315.
    if case == "two_material_tiny":
        wl = two_material("tiny", k=8.0)
    elif case == "disk":
        wl = constant_disk(k=5.0)
    else:
        wl = tm40k[0]
    n = wl.mesh.n_nodes
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0, pairsum=3)
    f = _dev(random_density(n, 77))
    ys, ys2, yo = torch.empty_like(f), torch.empty_like(f), torch.empty_like(f)
    op.pairsum_dev(f, ys)
    op.pairsum_dev(f, ys2)
    op.set_pair_symmetry(False)
    op.pairsum_dev(f, yo)
    op.set_pair_symmetry(True)
    e = (torch.linalg.norm(ys - yo) / torch.linalg.norm(yo)).item()
    ref = naive_apply(wl.mesh.nodes, wl.mesh.weights, wl.k, random_density(n, 77)) if n < 5000 else None
    e_or = _rel(ys.cpu().numpy(), ref) if ref is not None else None
    print(case, n, "symmetric vs ordered pair sum", e, "vs oracle naive sum", e_or)
    assert torch.equal(ys, ys2)
    assert e < 1e-13
    if ref is not None:
        assert e_or < 1e-13


def test_pairsum_precision_form_full_size(tm40k):
    # FP32 table (2e-8), FP32 strengths (6e-8), Kahan-compensated sums: ~1e-7 expected, for
    # the unordered-pair kernel (default) and the ordered-pair one alike
    wl, op = tm40k
    n = wl.mesh.n_nodes
    op32 = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0, pairsum=2)
    f = _dev(random_density(n, 19))
    y0 = torch.empty_like(f)
    y1 = torch.empty_like(f)
    y2 = torch.empty_like(f)
    op.pairsum_dev(f, y0)
    op32.pairsum_dev(f, y1)
    op32.set_pair_symmetry(False)
    op32.pairsum_dev(f, y2)
    err = (torch.linalg.norm(y1 - y0) / torch.linalg.norm(y0)).item()
    err_o = (torch.linalg.norm(y2 - y0) / torch.linalg.norm(y0)).item()
    print("precision-form pair sum rel err: unordered pairs", err, "ordered pairs", err_o)
    assert err < 5e-7 and err_o < 5e-7


def test_precision_form_solutions(tm40k):
    # target of the precision form: <= 1e-6 relative solution error vs FP64
    wl = two_material("tiny", k=8.0, nx=64, ny=64)
    op32 = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=64, ny=64, tol=1e-10, pairsum=2)
    u, _, _, _, st = op32.solve([np.pi / 4])
    b = plane_wave(wl.mesh.nodes, wl.k, np.pi / 4)
    ud = np.linalg.solve(OracleOp(wl.mesh, wl.k, wl.m).dense(), b)
    e_small = _rel(u[0], ud)
    wl2, op64 = tm40k
    op2 = L.Operator(L.Mesh(wl2.mesh), wl2.k, wl2.m, wl2.m_grid, tol=1e-10, pairsum=2)
    u32, _, _, it32, st32 = op2.solve([np.pi / 4])
    op64b = L.Operator(L.Mesh(wl2.mesh), wl2.k, wl2.m, wl2.m_grid, tol=1e-10)
    u64, _, _, it64, st64 = op64b.solve([np.pi / 4])
    e_full = _rel(u32[0], u64[0])
    print("precision form: small vs oracle", e_small, "full vs FP64 path", e_full, "iters", it32, it64)
    assert st == st32 == st64 == L.LS_OK
    assert e_small < 1e-6 and e_full < 1e-6


def test_mixed_form_solutions(tm40k):
    # pairsum = 4: FP32 GMRES refined against the double-float operator.  The refinement
    # stops on the accurate operator's residual, so the solution meets the FP64 solve's
    # tolerance times the condition factor, far inside the 1e-6 precision-form target.
    wl = two_material("tiny", k=8.0, nx=64, ny=64)
    op4 = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=64, ny=64, tol=1e-10, pairsum=4)
    u, _, _, it, st = op4.solve([np.pi / 4])
    A = OracleOp(wl.mesh, wl.k, wl.m).dense()
    b = plane_wave(wl.mesh.nodes, wl.k, np.pi / 4)
    e_small = _rel(u[0], np.linalg.solve(A, b))
    res_small = op4.last_residual()
    # the refinement's residual (updated with FP32 products of the corrections) against a full
    # re-apply of the double-float operator: they differ by ~eps32 ||k^2 V M|| ||d|| ~ 1e-13 ||b||
    # (times ||P|| in the preconditioned norm), asserted within a tenth of tol
    res_full = op4.residual_dev(_dev(b), _dev(u[0]))
    # the adjoint solve takes the same refinement (transposed operators)
    g = random_density(wl.mesh.n_nodes, 41)[None, :]
    lam, _, st_a = op4.solve_adjoint(g)
    e_adj = _rel(lam[0], np.linalg.solve(A.T, g[0]))
    # single applies use the accurate operator: identical to the double-float form
    op3 = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=64, ny=64, tol=1e-10, pairsum=3)
    x = _dev(random_density(wl.mesh.n_nodes, 42))
    y3, y4 = torch.empty_like(x), torch.empty_like(x)
    op3.apply_dev(x, y3)
    op4.apply_dev(x, y4)
    wl2, _ = tm40k
    op2 = L.Operator(L.Mesh(wl2.mesh), wl2.k, wl2.m, wl2.m_grid, tol=1e-10, pairsum=4)
    u4, _, _, it4, st4 = op2.solve([np.pi / 4])
    res_big = op2.last_residual()
    op64 = L.Operator(L.Mesh(wl2.mesh), wl2.k, wl2.m, wl2.m_grid, tol=1e-10)
    u64, _, _, it64, st64 = op64.solve([np.pi / 4])
    e_full = _rel(u4[0], u64[0])
    print("mixed form: small vs oracle", e_small, "adjoint", e_adj, "full vs FP64 path", e_full,
          "exit residuals", res_small, res_big, "full re-apply", res_full, "iterations (all inner)", it, it4,
          "FP64", it64)
    assert st == st_a == st4 == st64 == L.LS_OK
    assert torch.equal(y3, y4)
    assert res_small <= 1e-10 and res_full <= 1e-10 and abs(res_full - res_small) <= 1e-11
    assert e_small < 1e-8 and e_adj < 1e-8 and e_full < 1e-8


def test_precond_parity_small():
    wl = constant_disk(k=5.0, n_rings=3, nx=48, ny=48)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, wl.m_grid, nx=48, ny=48)
    x = random_density(wl.mesh.n_nodes, 7)
    y = torch.empty(wl.mesh.n_nodes, dtype=torch.complex128, device="cuda")
    op.apply_precond_dev(_dev(x), y)
    P = Preconditioner(Grid(wl.box, wl.nx, wl.ny), wl.mesh.nodes, wl.k, wl.m_grid)
    assert _rel(y.cpu().numpy(), P.apply(x)) < 1e-11


def test_precond_parity_full_size(tm40k):
    # The library and the oracle build C = A L^(C) independently (entries agree to 4.7e-14
    # of max |C|) and cond_1(C) ~ 2.6e5 on this 256^2 grid (scipy onenormest), so the
    # worst case for C^{-1} t is ~1e-8; measured 4.0e-13 with the cyclic-reduction solve,
    # and the bar is the FP64 matvec bar 1e-11.
    wl, op = tm40k
    n = wl.mesh.n_nodes
    x = random_density(n, 13)
    y = torch.empty(n, dtype=torch.complex128, device="cuda")
    op.apply_precond_dev(_dev(x), y)
    P = Preconditioner(Grid(wl.box, wl.nx, wl.ny), wl.mesh.nodes, wl.k, wl.m_grid)
    err = _rel(y.cpu().numpy(), P.apply(x))
    print("precond full-size rel err", err)
    assert err < 1e-11


def test_solve_matches_oracle_small_disk():
    wl = constant_disk(k=5.0, n_rings=3)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0, tol=1e-12)
    u, uinf, hist, iters, st = op.solve([0.0], wl.ff_angles)
    assert st == L.LS_OK and hist[0, iters[0]] <= 1e-12
    ora = OracleOp(wl.mesh, wl.k, wl.m)
    b = plane_wave(wl.mesh.nodes, wl.k, 0.0)
    ud = np.linalg.solve(ora.dense(), b)
    assert _rel(u[0], ud) < 1e-9
    ff = far_field(wl.mesh.nodes, wl.mesh.weights, wl.m, u[0], wl.k, wl.ff_angles)
    assert _rel(uinf[0], ff) < 1e-12


def test_solve_disk_mie_and_energy():
    wl = constant_disk(k=5.0, n_rings=6)      # 216 triangles, 3,240 nodes
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0, tol=1e-10)
    u, uinf, hist, iters, st = op.solve([0.0], wl.ff_angles)
    assert st == L.LS_OK
    ref = mie_interior(wl.mesh.nodes, wl.k, 1.5)
    e_int = np.max(np.abs(u[0] - ref)) / np.max(np.abs(ref))
    e_ff = np.max(np.abs(uinf[0] - mie_far_field(wl.ff_angles, wl.k, 1.5)))
    b = plane_wave(wl.mesh.nodes, wl.k, 0.0)
    lhs = np.imag(np.sum(wl.mesh.weights * np.conj(wl.m * u[0]) * b))
    rhs = np.sum(np.abs(uinf[0]) ** 2) * 2 * np.pi / len(wl.ff_angles) / wl.k
    print("disk iters", iters[0], "Mie e_int", e_int, "far-field err", e_ff, "energy", lhs, rhs)
    assert e_int < 1e-5 and e_ff < 1e-5
    assert abs(lhs - rhs) < 1e-5 * rhs


def test_preconditioned_solve_two_material():
    wl = two_material("tiny", k=8.0, nx=64, ny=64)
    mesh = L.Mesh(wl.mesh)
    opu = L.Operator(mesh, wl.k, wl.m, use_precond=0, tol=1e-10)
    opp = L.Operator(mesh, wl.k, wl.m, wl.m_grid, nx=64, ny=64, tol=1e-10)
    uu, _, _, iu, su = opu.solve([np.pi / 4])
    up, _, _, ip, sp = opp.solve([np.pi / 4])
    assert su == sp == L.LS_OK
    assert ip[0] < iu[0]
    assert _rel(up[0], uu[0]) < 1e-8
    b = plane_wave(wl.mesh.nodes, wl.k, np.pi / 4)
    ud = np.linalg.solve(OracleOp(wl.mesh, wl.k, wl.m).dense(), b)
    assert _rel(up[0], ud) < 1e-8


def test_two_material_full_size_solve(tm40k):
    wl, op = tm40k
    u, uinf, hist, iters, st = op.solve([np.pi / 4], wl.ff_angles)
    print("two-material preconditioned iterations", iters[0])
    assert st == L.LS_OK and iters[0] < 100
    # the true residual of the returned solution, with the library's own L and P
    n = wl.mesh.n_nodes
    ud = _dev(u[0])
    Lu = torch.empty(n, dtype=torch.complex128, device="cuda")
    op.apply_dev(ud, Lu)
    b = _dev(plane_wave(wl.mesh.nodes, wl.k, np.pi / 4))
    r = torch.empty_like(Lu)
    pb = torch.empty_like(Lu)
    op.apply_precond_dev(b - Lu, r)
    op.apply_precond_dev(b, pb)
    assert (torch.linalg.norm(r) / torch.linalg.norm(pb)).item() < 2e-8
    # the same solution through the oracle's operator on 48 sampled rows: the residual
    # b - L u the oracle computes matches the library's to the matvec bar (1e-11 of L u)
    # and is itself small (GMRES tolerance 1e-8 on the preconditioned residual)
    rows = np.sort(np.random.default_rng(5).choice(n, 48, replace=False))
    Lu_rows = OracleOp(wl.mesh, wl.k, wl.m, rows_only=True).apply_rows(u[0], rows)
    bh = b.cpu().numpy()
    r_oracle = bh[rows] - Lu_rows
    r_lib = (b - Lu).cpu().numpy()[rows]
    assert np.linalg.norm(r_oracle - r_lib) <= 1e-11 * np.linalg.norm(Lu_rows)
    assert np.linalg.norm(r_oracle) <= 1e-6 * np.linalg.norm(bh[rows])


def test_solve_dev_and_enoconv():
    wl = constant_disk(k=5.0, n_rings=2)
    mesh = L.Mesh(wl.mesh)
    op = L.Operator(mesh, wl.k, wl.m, use_precond=0, tol=1e-12)
    b = plane_wave(wl.mesh.nodes, wl.k, 0.3)
    bd = _dev(np.stack([b, 2 * b]))
    ud = torch.empty_like(bd)
    iters, st = op.solve_dev(bd, ud)
    assert st == L.LS_OK
    u = ud.cpu().numpy()
    assert _rel(u[1], 2 * u[0]) < 1e-12
    op3 = L.Operator(mesh, wl.k, wl.m, use_precond=0, tol=1e-12, max_iter=3)
    _, _, _, it3, st3 = op3.solve([0.3])
    assert st3 == L.LS_ENOCONV and it3[0] == 3


def test_bad_device_arguments():
    wl = constant_disk(k=5.0, n_rings=1)
    op = L.Operator(L.Mesh(wl.mesh), wl.k, wl.m, use_precond=0)
    x = torch.zeros(wl.mesh.n_nodes, dtype=torch.complex128, device="cuda")
    with pytest.raises(L.LsError):
        op.apply_dev(x, x)                     # aliasing is rejected
    with pytest.raises(L.LsError):
        op.apply_precond_dev(x, torch.empty_like(x))   # no preconditioner built
