"""Cartesian-grid preconditioner P = I + T_C^Q (S - I) T_Q^C (Eq. preconditioner_factored).

* Grid (Section 4): n_x x n_y nodes z_(a,b) = (x0 + a h_C, y0 + b h_C), endpoints
  included, index a + n_x b.
* T_C^Q (Eq. psi_def): bilinear interpolation from the four corners of the
  cell containing each quadrature node; rows sum to one.
* T_Q^C, Approach II (Eq. T_H^C_def, Eq. D_def): D^{-1} (T_C^Q)^T with D the
  column sums at pixelation nodes and 1 elsewhere.
* V^(C) (Eq. LS_eq_on_cartesian_points): G(z_i - z_l) h_C^2 off the diagonal.
  Reading: the Duan-Rokhlin corrected weights are not available, the diagonal
  is the integral of G over the disc of area h_C^2,
  (i pi a H1(k a)) / (2k) - 1/k^2 with pi a^2 = h_C^2.
* Stencil (Eq. sparsifying_min, Eq. cart_neighbors_LS): the neighbourhood
  N(j) = {i : |i - j|_inf <= 1, z_i in D} is the 3x3 block truncated to the
  grid, so a row's stencil depends on its class c = ca + 3 cb (ca = 0 at the
  first column, 1 inside, 2 at the last column; cb likewise for rows): interior
  (9 points), edge (6) or corner (4).  By translation invariance one
  representative per class suffices (the grid centre, the middle of an edge, the
  corner itself): B = V^(C)(N(j), N(j)^c) against every other grid node,
  v = conj of the left singular vector of the smallest singular value.
  A(j, N(j)) = v_c(j) on every row.
* C (Eq. LC_def): A L^(C) kept on the 3x3 pattern of each row, with
  L^(C) = I + k^2 V^(C) M^(C), M^(C) = diag(m(z_j)).  S = C^{-1} A, applied
  with a sparse LU (SuperLU from scipy).
"""
import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla
import scipy.special as sp

from .bessel import hankel01

STENCIL = [(da, db) for db in (-1, 0, 1) for da in (-1, 0, 1)]


class Grid:
    def __init__(self, box, nx, ny):
        self.box, self.nx, self.ny = box, nx, ny
        x0, x1, y0, y1 = box
        self.h = (x1 - x0) / (nx - 1)
        if abs((y1 - y0) / (ny - 1) - self.h) > 1e-14 * self.h:
            raise ValueError("grid must have a uniform step in x and y")
        self.x0, self.y0 = x0, y0

    @property
    def n(self):
        return self.nx * self.ny

    def points(self):
        a = np.arange(self.nx)
        b = np.arange(self.ny)
        A, B = np.meshgrid(a, b)
        return np.stack([self.x0 + A.ravel() * self.h, self.y0 + B.ravel() * self.h], axis=1)


def transfer_CQ(grid, nodes):
    """Sparse T_C^Q (N_Q x N_C) of bilinear weights psi_j(y_q)."""
    fx = (nodes[:, 0] - grid.x0) / grid.h
    fy = (nodes[:, 1] - grid.y0) / grid.h
    a = np.clip(np.floor(fx).astype(np.int64), 0, grid.nx - 2)
    b = np.clip(np.floor(fy).astype(np.int64), 0, grid.ny - 2)
    rows, cols, vals = [], [], []
    q = np.arange(nodes.shape[0])
    for da in (0, 1):
        for db in (0, 1):
            zx = grid.x0 + (a + da) * grid.h
            zy = grid.y0 + (b + db) * grid.h
            psi = (1 - np.abs(nodes[:, 0] - zx) / grid.h) * (1 - np.abs(nodes[:, 1] - zy) / grid.h)
            rows.append(q)
            cols.append((a + da) + grid.nx * (b + db))
            vals.append(psi)
    return sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(nodes.shape[0], grid.n))


def transfer_QC_II(T):
    """Approach II: D^{-1} T^T with D = column sums (1 where the column is empty)."""
    colsum = np.asarray(T.sum(axis=0)).ravel()
    D = np.where(colsum > 0, colsum, 1.0)
    return sps.diags(1.0 / D) @ T.T.tocsr(), D


def cartesian_kernel(k, h, da, db):
    """V^(C) entry for grid offset (da, db) (arrays)."""
    r = h * np.sqrt(np.asarray(da, float) ** 2 + np.asarray(db, float) ** 2)
    out = np.empty(r.shape, dtype=np.complex128)
    nz = r > 0
    h0, _ = hankel01(k * r[nz])
    out[nz] = 0.25j * h0 * h * h
    a = h / np.sqrt(np.pi)
    out[~nz] = 1j * np.pi * a * sp.hankel1(1, k * a) / (2 * k) - 1 / k**2
    return out


def row_class(grid, a, b):
    """Class of grid row (a, b): ca + 3 cb with 0 / 1 / 2 = first / inner / last index."""
    ca = 0 if a == 0 else (2 if a == grid.nx - 1 else 1)
    cb = 0 if b == 0 else (2 if b == grid.ny - 1 else 1)
    return ca + 3 * cb


def stencil_vectors(grid, k):
    """v[c] (9 entries in STENCIL order, zero outside the grid) minimising
    ||v V^(C)(N(j), N(j)^c)||, ||v|| = 1, at the representative node j of each
    class c; also the singular values of each B."""
    A, B = np.meshgrid(np.arange(grid.nx), np.arange(grid.ny))
    A, B = A.ravel(), B.ravel()
    rep_a = (0, grid.nx // 2, grid.nx - 1)
    rep_b = (0, grid.ny // 2, grid.ny - 1)
    vs, svs = np.zeros((9, 9), np.complex128), []
    for c in range(9):
        ca, cb = rep_a[c % 3], rep_b[c // 3]
        offs = [s for s, (da, db) in enumerate(STENCIL)
                if 0 <= ca + da < grid.nx and 0 <= cb + db < grid.ny]
        keep = ~((np.abs(A - ca) <= 1) & (np.abs(B - cb) <= 1))
        rows = [cartesian_kernel(k, grid.h, A[keep] - (ca + STENCIL[s][0]), B[keep] - (cb + STENCIL[s][1]))
                for s in offs]
        U, sv, _ = np.linalg.svd(np.stack(rows, axis=0), full_matrices=False)
        vs[c, offs] = np.conj(U[:, -1])
        svs.append(sv)
    return vs, svs


class Preconditioner:
    def __init__(self, grid, nodes, k, m_grid):
        self.grid, self.k = grid, float(k)
        self.T = transfer_CQ(grid, nodes)
        self.TQC, self.D = transfer_QC_II(self.T)
        self.v, self.sv = stencil_vectors(grid, k)
        self.m_grid = np.asarray(m_grid, np.complex128)
        self.A, self.C = self._assemble()
        self.lu = spla.splu(self.C.tocsc())

    def _assemble(self):
        g, k, v = self.grid, self.k, self.v
        nx, ny = g.nx, g.ny
        Ar, Ac, Av, Cr, Cc, Cv = [], [], [], [], [], []
        # V^(C) on offsets [-2, 2]^2 for the C entries
        off = {(da, db): cartesian_kernel(k, g.h, np.array([da]), np.array([db]))[0]
               for da in range(-2, 3) for db in range(-2, 3)}
        for b in range(ny):
            for a in range(nx):
                j = a + nx * b
                vc = v[row_class(g, a, b)]
                arow = {}
                for s, (da, db) in enumerate(STENCIL):
                    if 0 <= a + da < nx and 0 <= b + db < ny:
                        arow[(a + da, b + db)] = vc[s]
                for (ia, ib), av in arow.items():
                    Ar.append(j); Ac.append(ia + nx * ib); Av.append(av)
                # C_jl = sum_i A_ji (delta_il + k^2 V^(C)_il m_l), l in the 3x3 pattern of j
                for da, db in STENCIL:
                    la, lb = a + da, b + db
                    if not (0 <= la < nx and 0 <= lb < ny):
                        continue
                    l = la + nx * lb
                    acc = arow.get((la, lb), 0.0)
                    ml = self.m_grid[l]
                    if ml != 0:
                        acc = acc + k * k * ml * sum(av * off[(ia - la, ib - lb)] for (ia, ib), av in arow.items())
                    Cr.append(j); Cc.append(l); Cv.append(acc)
        n = g.n
        return (sps.csr_matrix((Av, (Ar, Ac)), shape=(n, n)),
                sps.csr_matrix((np.array(Cv, dtype=np.complex128), (Cr, Cc)), shape=(n, n)))

    def S_minus_I(self, gvec):
        return self.lu.solve(self.A @ gvec) - gvec

    def apply(self, x):
        """P x = x + T_C^Q (S - I) T_Q^C x."""
        return x + self.T @ self.S_minus_I(self.TQC @ x)
