"""CPU-side checks of the C-ABI library: it loads, exports every declared
symbol, validates inputs, and its host setup of the VDIM correction agrees with
the oracle's (both in extended precision, independently written), as does its
host setup of the preconditioner's stencils and banded C."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.sparse as sps

import paper_2608_17615_b300 as L
from lsinput.mesh import disk_mesh
from lsinput.workloads import two_material
from oracle import vdim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lsgpu.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ls_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(L.LIB_PATH)
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.EXPORTED) == names


def test_params_default():
    p = L.params_default()
    assert p.tol == 1e-8 and p.max_iter == 600 and p.use_precond == 1 and p.kappa == 3.0
    assert list(p.box) == [-1.2, 1.2, -1.2, 1.2] and p.nx == 256 and p.ny == 256
    assert p.prec == L.LS_PREC_FP64_DF and p.approach == 2 and p.setup_on_device == 1


def test_mesh_rejects_clockwise_element():
    m = disk_mesh(1)
    m.tris = m.tris.copy()
    m.tris[0] = m.tris[0][::-1]
    with pytest.raises(L.LsError) as e:
        L.Mesh(m)
    assert e.value.status == L.LS_EINVAL


def test_mesh_rejects_out_of_range_vertex():
    m = disk_mesh(1)
    m.tris = m.tris.copy()
    m.tris[2, 1] = 10_000
    with pytest.raises(L.LsError):
        L.Mesh(m)


def test_correction_rejects_bad_k():
    M = L.Mesh(disk_mesh(1))
    with pytest.raises(L.LsError):
        L.correction_host(M, -1.0)


def _csr(mesh, rp, ci, va):
    return sps.csr_matrix((va, ci, rp), shape=(mesh.n_nodes, mesh.n_nodes))


def test_correction_matches_oracle_disk():
    mesh = disk_mesh(2)
    k = 5.0
    A = _csr(mesh, *L.correction_host(L.Mesh(mesh), k, 3.0))
    B = vdim.correction_matrix(mesh, k, 3.0)
    assert (A != 0).nnz == (B != 0).nnz == 15 * mesh.n_nodes
    assert abs(A - B).max() < 1e-13 * abs(B).max()


def test_correction_matches_oracle_two_materials():
    # tiny two-material mesh: rows with a second (foreign-subdomain) block
    wl = two_material("tiny", k=8.0)
    mesh = wl.mesh
    A = _csr(mesh, *L.correction_host(L.Mesh(mesh), wl.k, 3.0))
    rows = np.arange(0, mesh.n_nodes, 7)
    B = vdim.correction_matrix(mesh, wl.k, 3.0, rows=rows)
    Ar = A[rows]
    assert np.array_equal(Ar.indptr, B.indptr)
    assert np.max(np.diff(B.indptr)) == 30          # some rows carry a foreign block
    assert abs(Ar - B).max() < 1e-13 * abs(B).max()


def _phase_align(a, b):
    """b rotated by the unit complex factor that best matches it to a."""
    z = np.vdot(b, a)
    return b * (z / abs(z)) if abs(z) > 0 else b


@pytest.mark.parametrize("k, nx", [(5.0, 24), (10.0, 36)])
def test_grid_host_matches_oracle(k, nx):
    """The library's host setup of the sparsifying stencils (one per row class, on the
    truncated neighbourhoods) and of C = A L^(C) on the 3x3 pattern against the oracle's
    (independent SVD-based construction).  Stencils are unit vectors fixed up to a phase,
    which C's rows share."""
    from lsinput.workloads import constant_disk
    from oracle.precond import Grid, Preconditioner, STENCIL, row_class

    wl = constant_disk(k=k, n_rings=2, nx=nx, ny=nx)
    g = Grid(wl.box, wl.nx, wl.ny)
    P = Preconditioner(g, wl.mesh.nodes, wl.k, wl.m_grid)
    st, cb = L.grid_host(L.Mesh(wl.mesh), wl.k, wl.box, wl.nx, wl.ny, wl.m_grid)
    phase = np.ones(9, complex)
    for c in range(9):
        ca = (0, nx // 2, nx - 1)[c % 3]
        cb_ = (0, nx // 2, nx - 1)[c // 3]
        outside = [s for s, (da, db) in enumerate(STENCIL) if not (0 <= ca + da < nx and 0 <= cb_ + db < nx)]
        assert np.all(st[c, outside] == 0)
        assert abs(np.linalg.norm(st[c]) - 1) < 1e-13
        v = _phase_align(st[c], P.v[c])
        assert np.linalg.norm(st[c] - v) < 1e-8, c
        z = np.vdot(P.v[c], st[c])
        phase[c] = z / abs(z)
    C = P.C.tocsr()
    worst, scale = 0.0, abs(C).max()
    for b in range(nx):
        for a in range(nx):
            j = a + nx * b
            ph = phase[row_class(g, a, b)]
            for da, db in STENCIL:
                la, lb = a + da, b + db
                if not (0 <= la < nx and 0 <= lb < nx):
                    continue
                worst = max(worst, abs(cb[b, db + 1, da + 1, a] - ph * C[j, la + nx * lb]))
    assert worst < 1e-8 * scale, worst / scale


@pytest.mark.parametrize("approach", [1, 2])
def test_transfer_host_matches_oracle(approach):
    """The library's host T_Q^C (both approaches) against the oracle's, on the curved
    two-material mesh (curved elements on both sides of the interface)."""
    from oracle.precond import Grid, transfer_CQ, transfer_QC_I, transfer_QC_II
    wl = two_material("tiny", k=8.0)
    box, nx = (-1.2, 1.2, -1.2, 1.2), 41
    rp, ci, va, nint = L.transfer_host(L.Mesh(wl.mesh), box, nx, nx, approach)
    A = sps.csr_matrix((va, ci, rp), shape=(nx * nx, wl.mesh.n_nodes))
    g = Grid(box, nx, nx)
    if approach == 1:
        B, owner = transfer_QC_I(g, wl.mesh)
        assert nint == int((owner >= 0).sum())
    else:
        B, _ = transfer_QC_II(transfer_CQ(g, wl.mesh.nodes))
    assert (A != 0).nnz == (B != 0).nnz
    assert abs(A - B).max() < 1e-13 * abs(B).max()


def test_hessenberg_eigenvalues_match_numpy():
    """The library's host QR iteration (Ritz values) against LAPACK through numpy, on random
    complex upper Hessenberg matrices and on one with a nearly repeated cluster at 1 (the
    preconditioned spectrum's shape)."""
    rng = np.random.default_rng(11)
    for n in (1, 2, 7, 40, 120):
        H = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), -1)
        e = np.sort_complex(L.hessenberg_eigenvalues(H))
        ref = np.sort_complex(np.linalg.eigvals(H))
        assert np.max(np.abs(e - ref)) < 1e-9 * max(1.0, np.max(np.abs(ref)))
    n = 60
    Q = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(1 + 0.05 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))) @ Q.conj().T
    import scipy.linalg as sl
    Hh = sl.hessenberg(A)
    e = L.hessenberg_eigenvalues(Hh)
    ref = np.linalg.eigvals(A)
    d = np.abs(e[:, None] - ref[None, :]).min(axis=1)
    assert np.max(d) < 1e-10


def test_correction_size_query_plans_only():
    """The size query of both correction builds (null output arrays) only plans the patches:
    it runs without a GPU and gives the nnz of the full host build (15 entries per
    target-patch block)."""
    import ctypes
    wl = two_material("tiny", k=8.0)
    mesh = L.Mesh(wl.mesh)
    nnz_d, nnz_h = ctypes.c_int64(), ctypes.c_int64()
    st = L._lib.ls_correction_dev(mesh.handle, 8.0, 3.0, None, ctypes.byref(nnz_d), None, None, None, None)
    assert st == L.LS_OK
    assert L._lib.ls_correction_host(mesh.handle, 8.0, 3.0, ctypes.byref(nnz_h), None, None, None) == L.LS_OK
    rp, ci, va = L.correction_host(mesh, 8.0, 3.0)
    assert nnz_d.value == nnz_h.value == ci.size and nnz_d.value % 15 == 0
