"""VDIM near/self correction of the naive pair sum (Eq. DIM_decomp).

The paper (Section 3) evaluates V_{Omega_l}[f](x) for a target x in triangle
tau(x) as V[f - F](x) + B[F](x): F is the degree-p interpolant of f on tau,
Phi a polynomial with (Delta + k^2) Phi = F, and B[F](x) collects single- and
double-layer potentials of Phi on the boundary plus the local value -Phi(x)
(Green's third identity).  V[f - F] is left to the plain quadrature.

Reading taken here (VDIM's own code is not available): the identity is applied
on a *local patch* P(x) of elements of the subdomain around the target, and the
plain quadrature covers the rest of the subdomain.  For target node x_j with
element tau and F = sum_q f_q L_q (L_q the Lagrange basis of tau's 15 nodes):

    V_h[f](x_j) = sum_{n != j} G w_n f_n + sum_q dV_jq f_q,
    dV_jq = E_jq - N_jq,
    E_jq  = -chi(x_j) Phi_q(x_j) + int_{dP} [G dPhi_q/dn - Phi_q dG/dn_y] ds_y,
    N_jq  = sum_{n in P, n != j} G(x_j, y_n) w_n L_q(y_n),

with Phi_q = L_q/k^2 - Delta L_q/k^4 + Delta^2 L_q/k^6 (exact for degree 4)
and the outward normal of P.  E_jq is the exact integral of G L_q over P.  The
same is done, with chi = 0 and the element of that subdomain nearest to x_j,
for every other subdomain that has elements within the patch radius of x_j.

Patch rule (shared definition with the CUDA library, restated there):
element t belongs to the patch of target j in subdomain l iff domain(t) = l and
|c_t - x_j|^2 < kappa^2 h_j^2, where c_t = ((v0 + v1) + v2)/3 is the vertex
centroid and h_j^2 the largest squared vertex distance of the target's own
element; the target's own element always belongs to its own patch.
kappa = inf gives the global form of Eq. DIM_decomp (patch = whole subdomain).

Boundary integrals: adaptive bisection with Gauss-Legendre 16 vs 32 points on
every panel (accept when the two agree), edges parametrised exactly (straight
segments or the polar-curve arcs of the mesh).

Precision: dV_jq is a small difference of two large numbers (E and N grow with
the Lagrange polynomials across the patch while dV is O(h^2 log h)), so all of
this module's arithmetic runs in numpy.longdouble (64-bit mantissa) and only
the final dV is rounded to complex128.  The patch membership test is done in
float64 exactly as written above.
"""
import numpy as np

from .bessel import hankel01

P_DEG = 4
EXPS = [(i, d - i) for d in range(P_DEG + 1) for i in range(d, -1, -1)]   # (a, b) of s1^a s2^b
N_Q = 15
LD = np.longdouble


def _gauss_legendre_ld(n):
    """Gauss-Legendre nodes/weights on [-1, 1] in long double (Newton on P_n
    from the float64 nodes, weights 2 / ((1 - x^2) P_n'(x)^2))."""
    x = np.polynomial.legendre.leggauss(n)[0].astype(LD)
    for _ in range(3):
        p0, p1 = np.ones_like(x), x.copy()
        for m in range(2, n + 1):
            p0, p1 = p1, ((2 * m - 1) * x * p1 - (m - 1) * p0) / m
        dp = n * (x * p1 - p0) / (x * x - 1)
        x = x - p1 / dp
    p0, p1 = np.ones_like(x), x.copy()
    for m in range(2, n + 1):
        p0, p1 = p1, ((2 * m - 1) * x * p1 - (m - 1) * p0) / m
    dp = n * (x * p1 - p0) / (x * x - 1)
    return x, 2 / ((1 - x * x) * dp * dp)


_GL16 = _gauss_legendre_ld(16)
_GL32 = _gauss_legendre_ld(32)


def _inverse_ld(A):
    """Inverse of a small square long-double matrix (Gauss-Jordan, partial pivoting)."""
    n = A.shape[0]
    M = np.concatenate([A.astype(LD), np.eye(n, dtype=LD)], axis=1)
    for c in range(n):
        p = c + int(np.argmax(np.abs(M[c:, c])))
        if p != c:
            M[[c, p]] = M[[p, c]]
        M[c] = M[c] / M[c, c]
        f = M[:, c].copy()
        f[c] = 0
        M = M - f[:, None] * M[c][None, :]
    return M[:, n:]


def element_geometry(mesh):
    V = mesh.vertices[mesh.tris]
    cen = ((V[:, 0] + V[:, 1]) + V[:, 2]) / 3.0
    d01 = ((V[:, 0] - V[:, 1]) ** 2).sum(1)
    d12 = ((V[:, 1] - V[:, 2]) ** 2).sum(1)
    d20 = ((V[:, 2] - V[:, 0]) ** 2).sum(1)
    h2 = np.maximum(np.maximum(d01, d12), d20)
    return cen, h2


def _mono(s1, s2):
    return np.stack([s1**a * s2**b for a, b in EXPS], axis=-1)


def _mono_grad(s1, s2, h):
    d1 = np.stack([(a * s1 ** max(a - 1, 0) * s2**b if a > 0 else 0 * s1) for a, b in EXPS], axis=-1) / h
    d2 = np.stack([(b * s1**a * s2 ** max(b - 1, 0) if b > 0 else 0 * s1) for a, b in EXPS], axis=-1) / h
    return d1, d2


def _laplacian_matrix(h):
    """Matrix D with lap(sum_a c_a m_a) = sum_a (D c)_a m_a in scaled monomials."""
    D = np.zeros((N_Q, N_Q), dtype=LD)
    idx = {e: i for i, e in enumerate(EXPS)}
    for col, (a, b) in enumerate(EXPS):
        if a >= 2:
            D[idx[(a - 2, b)], col] += a * (a - 1) / h**2
        if b >= 2:
            D[idx[(a, b - 2)], col] += b * (b - 1) / h**2
    return D


def lagrange_and_phi(nodes_tau, c, h, k):
    """Coefficients (15 monomials x 15 basis functions) of L_q and Phi_q."""
    s = (nodes_tau.astype(LD) - c) / h
    Vm = _mono(s[:, 0], s[:, 1])               # [node q, monomial a]
    C = _inverse_ld(Vm)                        # L_q = sum_a mono_a C[a, q]
    D = _laplacian_matrix(h)
    k2 = LD(k) * LD(k)
    Phi = C / k2 - (D @ C) / k2**2 + (D @ (D @ C)) / k2**3
    return C, Phi


def _edge_descriptors(mesh, edges):
    """Per edge: start/end vertex, curve parameters (or NaN for straight)."""
    T = np.array([t for t, _ in edges], dtype=np.int64)
    E = np.array([e for _, e in edges], dtype=np.int64)
    va = mesh.vertices[mesh.tris[T, E]].astype(LD)
    vb = mesh.vertices[mesh.tris[T, (E + 1) % 3]].astype(LD)
    cid = mesh.edge_curve[T, E]
    curv = np.where(cid[:, None] >= 0, mesh.curves[np.maximum(cid, 0)], np.nan).astype(LD)
    th = mesh.edge_theta[T, E].astype(LD)
    return va, vb, cid >= 0, curv, th


def _edge_points(desc, ei, tt):
    """Points y(t) and derivatives y'(t) on edges ei (per panel) at params tt [P, n]."""
    va, vb, is_curved, curv, th = desc
    va, vb, cflag, cv, th = va[ei], vb[ei], is_curved[ei], curv[ei], th[ei]
    y = va[:, None, :] + tt[:, :, None] * (vb - va)[:, None, :]
    dy = np.broadcast_to((vb - va)[:, None, :], y.shape).copy()
    if np.any(cflag):
        c = np.nonzero(cflag)[0]
        cx, cy, R, a, m, phi = (cv[c, i][:, None] for i in range(6))
        th0, th1 = th[c, 0][:, None], th[c, 1][:, None]
        t = th0 + tt[c] * (th1 - th0)
        r = R * (1.0 + a * np.cos(m * t + phi))
        dr = -R * a * m * np.sin(m * t + phi)
        co, si = np.cos(t), np.sin(t)
        y[c, :, 0] = cx + r * co
        y[c, :, 1] = cy + r * si
        dy[c, :, 0] = (dr * co - r * si) * (th1 - th0)
        dy[c, :, 1] = (dr * si + r * co) * (th1 - th0)
    return y, dy


def _boundary_integrand(x, y, dy, k, Phi, c, h):
    """[npts, 15] values of (G dPhi/dn - Phi dG/dn) |y'| at points y."""
    nx, ny = dy[:, 1], -dy[:, 0]                  # outward normal times |y'|
    rx, ry = y[:, 0] - x[0], y[:, 1] - x[1]
    r = np.sqrt(rx * rx + ry * ry)
    h0, h1 = hankel01(k * r)
    G = 1j * h0 / 4
    dGdn = 1j * (-k * h1) * ((rx * nx + ry * ny) / r) / 4
    s1, s2 = (y[:, 0] - c[0]) / h, (y[:, 1] - c[1]) / h
    M = _mono(s1, s2)
    g1, g2 = _mono_grad(s1, s2, h)
    phi = M @ Phi
    dphidn = (g1 * nx[:, None] + g2 * ny[:, None]) @ Phi
    return G[:, None] * dphidn - dGdn[:, None] * phi


def _gl(nodes_w, a, b):
    xg, wg = nodes_w
    return a[:, None] + (b - a)[:, None] * (xg[None, :] + 1) / 2, (b - a)[:, None] * wg[None, :] / 2


def boundary_integral(mesh, edges, x, k, Phi, c, h, rtol=1e-18, max_level=60):
    """Sum over edges (element, edge index) of the layer integrals, [15] complex.

    Adaptive bisection of every edge's parameter interval: a panel is accepted
    when its 16- and 32-point Gauss-Legendre values agree to rtol relative to
    the size of the whole integral."""
    desc = _edge_descriptors(mesh, edges)
    ei = np.arange(len(edges))
    A = np.zeros(len(edges), dtype=LD)
    B = np.ones(len(edges), dtype=LD)
    lev = np.zeros(len(edges), dtype=np.int64)
    total = np.zeros(N_Q, dtype=np.clongdouble)
    scale = None
    while ei.size:
        vals = {}
        for name, rule in (("g16", _GL16), ("g32", _GL32)):
            tt, ww = _gl(rule, A, B)
            y, dy = _edge_points(desc, ei, tt)
            f = _boundary_integrand(x, y.reshape(-1, 2), dy.reshape(-1, 2), k, Phi, c, h)
            vals[name] = np.einsum("pn,pnq->pq", ww, f.reshape(ei.size, -1, N_Q))
        i32 = vals["g32"]
        err = np.max(np.abs(i32 - vals["g16"]), axis=1)
        if scale is None:
            scale = max(np.max(np.abs(i32.sum(0))), np.max(np.abs(i32)))
        ok = (err <= rtol * scale * 8) | (lev >= max_level)
        total += i32[ok].sum(0)
        bad = ~ok
        mid = 0.5 * (A[bad] + B[bad])
        ei = np.concatenate([ei[bad], ei[bad]])
        A, B = np.concatenate([A[bad], mid]), np.concatenate([mid, B[bad]])
        lev = np.concatenate([lev[bad], lev[bad]]) + 1
    return total


def patch_elements(cen, h2j, xj, dom, domain_l, kappa):
    d2 = ((cen - xj[None, :]) ** 2).sum(1)
    return np.nonzero((dom == domain_l) & (d2 < kappa * kappa * h2j))[0], d2


def patch_boundary_edges(mesh, elems):
    count = {}
    for t in elems:
        for e in range(3):
            a, b = mesh.tris[t, e], mesh.tris[t, (e + 1) % 3]
            key = (min(a, b), max(a, b))
            count[key] = count.get(key, 0) + 1
    out = []
    for t in elems:
        for e in range(3):
            a, b = mesh.tris[t, e], mesh.tris[t, (e + 1) % 3]
            if count[(min(a, b), max(a, b))] == 1:
                out.append((int(t), e))
    return out


def correction_block(mesh, j, k, elems, tau, own, geom=None):
    """dV_{j, tau nodes} (15 values) for patch `elems` and interpolation element tau."""
    cen, h2 = geom if geom is not None else element_geometry(mesh)
    x = mesh.nodes[j].astype(LD)
    k = LD(k)
    nodes_tau = mesh.nodes[tau * N_Q:(tau + 1) * N_Q]
    V = mesh.vertices[mesh.tris[tau]].astype(LD)
    c = ((V[0] + V[1]) + V[2]) / 3            # centre and scale of the local monomials
    h = np.sqrt(np.max([((V[a] - V[b]) ** 2).sum() for a, b in ((0, 1), (1, 2), (2, 0))]))
    C, Phi = lagrange_and_phi(nodes_tau, c, h, k)
    # E: Green's identity on the patch
    edges = patch_boundary_edges(mesh, elems)
    E = boundary_integral(mesh, edges, x, k, Phi, c, h)
    if own:
        s = (x - c) / h
        E = E - (_mono(np.array([s[0]]), np.array([s[1]])) @ Phi)[0]
    # N: plain quadrature of G L_q over the patch nodes (self node excluded)
    idx = (elems[:, None] * N_Q + np.arange(N_Q)[None, :]).ravel()
    idx = idx[idx != j]
    y = mesh.nodes[idx].astype(LD)
    r = np.sqrt(((y - x[None, :]) ** 2).sum(1))
    h0, _ = hankel01(k * r)
    G = 1j * h0 / 4
    s = (y - c[None, :]) / h
    L = _mono(s[:, 0], s[:, 1]) @ C
    N = (G * mesh.weights[idx].astype(LD)) @ L
    return (E - N).astype(np.complex128)


def correction_row(mesh, j, k, kappa=3.0, geom=None):
    """Column indices and values of row j of the sparse correction dV."""
    geom = geom if geom is not None else element_geometry(mesh)
    cen, h2 = geom
    tau_j = j // N_Q
    dom = mesh.domain
    l = dom[tau_j]
    x = mesh.nodes[j]
    cols, vals = [], []
    for lp in np.unique(dom):
        elems, d2 = patch_elements(cen, h2[tau_j], x, dom, lp, kappa)
        if lp == l:
            if tau_j not in elems:
                elems = np.sort(np.append(elems, tau_j))
            tau = tau_j
        else:
            if elems.size == 0:
                continue
            tau = int(elems[np.argmin(d2[elems])])
        v = correction_block(mesh, j, k, elems, tau, own=(lp == l), geom=geom)
        cols.append(np.arange(tau * N_Q, (tau + 1) * N_Q))
        vals.append(v)
    return np.concatenate(cols), np.concatenate(vals)


def correction_matrix(mesh, k, kappa=3.0, rows=None):
    """scipy CSR of dV for the given rows (all rows by default)."""
    import scipy.sparse as sps
    geom = element_geometry(mesh)
    n = mesh.n_nodes
    rows = np.arange(n) if rows is None else np.asarray(rows)
    indptr, indices, data = [0], [], []
    for j in rows:
        c, v = correction_row(mesh, int(j), k, kappa, geom)
        indices.append(c)
        data.append(v)
        indptr.append(indptr[-1] + c.size)
    return sps.csr_matrix((np.concatenate(data), np.concatenate(indices), np.array(indptr)),
                          shape=(rows.size, n))
