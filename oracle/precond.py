"""Cartesian-grid preconditioner P = I + T_C^Q (S - I) T_Q^C (Eq. preconditioner_factored).

* Grid (Section 4): n_x x n_y nodes z_(a,b) = (x0 + a h_C, y0 + b h_C), endpoints
  included, index a + n_x b.
* T_C^Q (Eq. psi_def): bilinear interpolation from the four corners of the
  cell containing each quadrature node; rows sum to one.
* T_Q^C, Approach II (Eq. T_H^C_def, Eq. D_def): D^{-1} (T_C^Q)^T with D the
  column sums at pixelation nodes and 1 elsewhere.  Approach I (Eq. T_HC_proj_def):
  the element-wise L^2 projection onto P1, evaluated at the interior grid nodes
  (transfer_QC_I below).
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


def _element_map_and_jacobian(mesh, t, xi, eta):
    """Physical point of reference point (xi, eta) in element t and the Jacobian of the
    element map (complex-step derivatives of the geometry map)."""
    from lsinput.mesh import _element_map
    V = mesh.vertices[mesh.tris[t]]
    curve, t0, t1, e = None, 0.0, 0.0, -1
    for ee in range(3):
        if mesh.edge_curve[t, ee] >= 0:
            curve = mesh.curves[mesh.edge_curve[t, ee]]
            t0, t1 = mesh.edge_theta[t, ee]
            e = ee
    hs = 1e-30
    x, y = _element_map(V, curve, t0, t1, e, xi, eta)
    xa, ya = _element_map(V, curve, t0, t1, e, xi + 1j * hs, eta + 0j)
    xb, yb = _element_map(V, curve, t0, t1, e, xi + 0j, eta + 1j * hs)
    J = np.array([[np.imag(xa) / hs, np.imag(xb) / hs], [np.imag(ya) / hs, np.imag(yb) / hs]])
    return np.real(x), np.real(y), J


def locate_points(mesh, pts, tol=1e-12):
    """Element containing each point (-1 if none): the point is in element t when the
    inverse of t's (curved) map, found by Newton's method from the affine guess, lies in
    the closed reference triangle; of several such elements the lowest index is taken."""
    owner = np.full(len(pts), -1, dtype=np.int64)
    for t in range(mesh.n_elem):
        V = mesh.vertices[mesh.tris[t]]
        # bounding box of the element, the curved edge's bulge included (edge points
        # strictly between the vertices, where the blending map is defined, plus the vertices)
        s_ = (np.arange(32) + 0.5) / 32
        with np.errstate(invalid="ignore", divide="ignore"):
            xs, ys = _element_map_and_jacobian(mesh, t, s_, np.zeros(32))[:2]
            xs2, ys2 = _element_map_and_jacobian(mesh, t, np.zeros(32), s_)[:2]
            xs3, ys3 = _element_map_and_jacobian(mesh, t, 1 - s_, s_)[:2]
        X = np.concatenate([xs, xs2, xs3, V[:, 0]]); Y = np.concatenate([ys, ys2, ys3, V[:, 1]])
        pad = 1e-9 * (1 + np.ptp(X) + np.ptp(Y))
        cand = np.nonzero((owner < 0) & (pts[:, 0] >= X.min() - pad) & (pts[:, 0] <= X.max() + pad)
                          & (pts[:, 1] >= Y.min() - pad) & (pts[:, 1] <= Y.max() + pad))[0]
        for j in cand:
            A = np.array([[V[1, 0] - V[0, 0], V[2, 0] - V[0, 0]], [V[1, 1] - V[0, 1], V[2, 1] - V[0, 1]]])
            ref = np.linalg.solve(A, pts[j] - V[0])
            with np.errstate(invalid="ignore", divide="ignore"):
                for _ in range(40):
                    x, y, J = _element_map_and_jacobian(mesh, t, np.array([ref[0]]), np.array([ref[1]]))
                    r = np.array([x[0] - pts[j, 0], y[0] - pts[j, 1]])
                    if not (np.all(np.isfinite(r)) and np.all(np.isfinite(J))):
                        break          # at a vertex of a curved element the blending is affine
                    step = np.linalg.solve(J[:, :, 0], r)
                    ref = ref - step
                    if np.max(np.abs(step)) < 1e-15:
                        break
            if np.all(np.isfinite(ref)) and ref[0] >= -tol and ref[1] >= -tol and ref[0] + ref[1] <= 1 + tol:
                owner[j] = t
    return owner


def barycentric(V, p):
    """Barycentric coordinates of points p [n, 2] in the straight triangle V [3, 2]."""
    A = np.array([[V[1, 0] - V[0, 0], V[2, 0] - V[0, 0]], [V[1, 1] - V[0, 1], V[2, 1] - V[0, 1]]])
    lam12 = np.linalg.solve(A, (p - V[0]).T).T
    return np.stack([1 - lam12[:, 0] - lam12[:, 1], lam12[:, 0], lam12[:, 1]], axis=1)


def transfer_QC_I(grid, mesh):
    """Approach I (Eq. T_HC_proj_def, Eq. T_HC_I_block): row j of an interior grid node
    z_j in element tau is E_C (M^tri)^{-1} E_Q^T W restricted to tau,
        T[j, q] = w_q sum_{i, i'} phi_i(z_j) (M^tau)^{-1}_{i i'} phi_i'(y_q),  y_q in tau,
    with phi_i the P1 Lagrange basis of tau's vertices (barycentric coordinates of the
    straight triangle through them, evaluated at the physical points) and the
    straight-triangle mass inverse of Eq. mass_closed_form,
    (M^tau)^{-1} = (3/|tau|) [[3, -1, -1], [-1, 3, -1], [-1, -1, 3]]; exterior rows zero.
    Returns the sparse matrix and the element of every grid node (-1 exterior)."""
    pts = grid.points()
    owner = locate_points(mesh, pts)
    Minv_unit = np.array([[3.0, -1.0, -1.0], [-1.0, 3.0, -1.0], [-1.0, -1.0, 3.0]])
    rows, cols, vals = [], [], []
    for j in np.nonzero(owner >= 0)[0]:
        t = owner[j]
        V = mesh.vertices[mesh.tris[t]]
        area = 0.5 * abs((V[1, 0] - V[0, 0]) * (V[2, 1] - V[0, 1]) - (V[2, 0] - V[0, 0]) * (V[1, 1] - V[0, 1]))
        q = np.arange(t * 15, (t + 1) * 15)
        phz = barycentric(V, pts[j:j + 1])[0]
        phq = barycentric(V, mesh.nodes[q])
        row = mesh.weights[q] * (phq @ ((3.0 / area) * Minv_unit) @ phz)
        rows.append(np.full(15, j)); cols.append(q); vals.append(row)
    T = sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(grid.n, mesh.n_nodes))
    return T, owner


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
    def __init__(self, grid, nodes, k, m_grid, approach=2, mesh=None):
        self.grid, self.k = grid, float(k)
        self.T = transfer_CQ(grid, nodes)
        self.TQC, self.D = transfer_QC_II(self.T)
        if approach == 1:
            self.TQC, self.owner = transfer_QC_I(grid, mesh)
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
