"""Pins of the oracle's preconditioner (Section 4): transfer-operator identities,
the round trip of Approach II (Lemma approachII_gram), exterior columns of
S - I (Eq. S_minus_I), the stencil minimisation (Eq. sparsifying_min) and
invertibility of P (Lemma well_poss_P)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from lsinput.workloads import constant_disk
from oracle.gmres import gmres
from oracle.operator import Operator, plane_wave
from oracle.precond import Grid, Preconditioner, cartesian_kernel, row_class, STENCIL


@pytest.fixture(scope="module")
def small():
    wl = constant_disk(k=5.0, n_rings=2, nx=24, ny=24)
    g = Grid(wl.box, wl.nx, wl.ny)
    P = Preconditioner(g, wl.mesh.nodes, wl.k, wl.m_grid)
    return wl, g, P


def test_bilinear_rows_sum_to_one(small):
    wl, g, P = small
    assert np.max(np.abs(np.asarray(P.T.sum(1)).ravel() - 1)) < 1e-14
    assert P.T.getnnz(axis=1).max() <= 4
    # reproduces linear fields exactly (bilinear interpolation)
    z = g.points()
    assert np.max(np.abs(P.T @ (2 * z[:, 0] - 3 * z[:, 1]) - (2 * wl.mesh.nodes[:, 0] - 3 * wl.mesh.nodes[:, 1]))) < 1e-13


def test_approach_II_round_trip(small):
    wl, g, P = small
    R = (P.TQC @ P.T).toarray()
    pix = np.asarray(P.T.sum(0)).ravel() > 0
    rs = R.sum(1)
    assert np.max(np.abs(rs[pix] - 1)) < 1e-13 and np.max(np.abs(rs[~pix])) == 0
    DR = np.diag(P.D) @ R
    assert np.max(np.abs(DR - DR.T)) < 1e-14            # D R_II = T^T T is symmetric
    Dh = np.sqrt(P.D)
    ev = np.linalg.eigvalsh((Dh[:, None] * R) / Dh[None, :])
    assert ev.min() > -1e-12 and ev.max() < 1 + 1e-12  # eigenvalues in [0, 1]


def test_exterior_columns_vanish(small):
    wl, g, P = small
    ext = np.nonzero(wl.m_grid == 0)[0]
    worst = 0.0
    for j in ext[::7]:
        e = np.zeros(g.n, complex)
        e[j] = 1
        worst = max(worst, np.max(np.abs(P.S_minus_I(e))))
    assert worst < 1e-13


def test_stencil_minimises(small):
    wl, g, P = small
    A, B = np.meshgrid(np.arange(g.nx), np.arange(g.ny))
    A, B = A.ravel(), B.ravel()
    for c in range(9):
        ca = (0, g.nx // 2, g.nx - 1)[c % 3]
        cb = (0, g.ny // 2, g.ny - 1)[c // 3]
        assert row_class(g, ca, cb) == c
        v = P.v[c]
        assert abs(np.linalg.norm(v) - 1) < 1e-14
        offs = [s for s, (da, db) in enumerate(STENCIL) if 0 <= ca + da < g.nx and 0 <= cb + db < g.ny]
        assert len(offs) == (9 if c == 4 else (4 if c in (0, 2, 6, 8) else 6))
        assert np.all(v[[s for s in range(9) if s not in offs]] == 0)
        # v B has norm sigma_min; the truncated neighbourhoods are also nearly rank deficient
        keep = ~((np.abs(A - ca) <= 1) & (np.abs(B - cb) <= 1))
        Bm = np.stack([cartesian_kernel(wl.k, g.h, A[keep] - (ca + STENCIL[s][0]), B[keep] - (cb + STENCIL[s][1]))
                       for s in offs])
        sv = P.sv[c]
        assert abs(np.linalg.norm(v[offs] @ Bm) - sv[-1]) < 1e-12 * sv[0]
        assert sv[-1] < (1e-3 if c == 4 else 5e-2) * sv[0]


def test_sparsifying_preconditioner_cartesian_iterations():
    """S^(C) is an approximate inverse of L^(C) (Eq. LC_def): on the Cartesian problem of the
    constant disk the preconditioned GMRES needs a handful of iterations, nearly independent
    of k (the behaviour the sparsifying preconditioner is cited for), far fewer than
    the unpreconditioned count."""
    counts = []
    for k, nx in ((5.0, 24), (10.0, 40)):
        g = Grid((-1.2, 1.2, -1.2, 1.2), nx, nx)
        z = g.points()
        m = np.where(np.hypot(z[:, 0], z[:, 1]) < 1, -1.25, 0).astype(complex)
        P = Preconditioner(g, np.zeros((1, 2)), k, m)
        A, B = np.meshgrid(np.arange(nx), np.arange(nx))
        A, B = A.ravel(), B.ravel()
        V = cartesian_kernel(k, g.h, A[:, None] - A[None, :], B[:, None] - B[None, :])
        Lc = np.eye(g.n) + k * k * V * m[None, :]
        b = np.exp(1j * k * z[:, 0])
        _, _, it_u = gmres(lambda x: Lc @ x, b, tol=1e-8)
        _, _, it_p = gmres(lambda x: Lc @ x, b, tol=1e-8, apply_P=lambda x: P.lu.solve(P.A @ x))
        counts.append((it_u, it_p))
    for it_u, it_p in counts:
        assert it_p <= 10 and it_p < it_u / 3, counts


def test_P_invertible_and_reduces_iterations():
    wl = constant_disk(k=5.0, n_rings=3, nx=48, ny=48)
    g = Grid(wl.box, wl.nx, wl.ny)
    P = Preconditioner(g, wl.mesh.nodes, wl.k, wl.m_grid)
    n = wl.mesh.n_nodes
    Pd = np.stack([P.apply(c) for c in np.eye(n, dtype=complex)], 1)
    assert np.linalg.svd(Pd, compute_uv=False).min() > 1e-3
    op = Operator(wl.mesh, wl.k, wl.m)
    b = plane_wave(wl.mesh.nodes, wl.k, 0.0)
    u0, _, i0 = gmres(op.apply, b, tol=1e-10)
    u1, _, i1 = gmres(op.apply, b, tol=1e-10, apply_P=P.apply)
    assert i1 < i0
    assert np.max(np.abs(u0 - u1)) < 1e-8 * np.max(np.abs(u0))
