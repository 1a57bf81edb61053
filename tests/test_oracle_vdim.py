"""Pins of the oracle's VDIM correction (Eq. DIM_decomp, local-patch reading)."""
import numpy as np
import pytest
import scipy.special as sp

from lsinput.mesh import disk_mesh, _element_map, load_rule, N_Q
from oracle import vdim
from oracle.nystrom import naive_apply, naive_rows


def _v1_disk(k, r):
    """V[1] inside the unit disk: -1/k^2 + (i pi H1(k) / (2k)) J0(k r)  (closed form)."""
    return -1 / k**2 + (1j * np.pi * sp.hankel1(1, k) / (2 * k)) * sp.j0(k * r)


@pytest.mark.parametrize("kappa", [np.inf, 3.0])
def test_constant_density_exact_on_small_disk(kappa):
    # For f = 1 the interpolant is exact (F = f), so with the patch covering the
    # whole subdomain V_h[1] equals the exact potential up to rounding.
    k = 5.0
    mesh = disk_mesh(2)
    f = np.ones(mesh.n_nodes, complex)
    dV = vdim.correction_matrix(mesh, k, kappa)
    v = naive_apply(mesh.nodes, mesh.weights, k, f) + dV @ f
    ex = _v1_disk(k, np.hypot(mesh.nodes[:, 0], mesh.nodes[:, 1]))
    assert np.max(np.abs(v - ex)) / np.max(np.abs(ex)) < 5e-13
    assert dV.nnz == 15 * mesh.n_nodes


def test_constant_density_local_patch_accuracy():
    # Local patches: the remainder is the plain quadrature outside the patch.
    k = 5.0
    mesh = disk_mesh(4)
    rows = np.arange(0, mesh.n_nodes, 37)
    f = np.ones(mesh.n_nodes, complex)
    dV = vdim.correction_matrix(mesh, k, 3.0, rows=rows)
    v = naive_rows(mesh.nodes, mesh.weights, k, f, rows) + dV @ f
    ex = _v1_disk(k, np.hypot(mesh.nodes[rows, 0], mesh.nodes[rows, 1]))
    assert np.max(np.abs(v - ex)) / np.max(np.abs(ex)) < 1e-8


def _lagrange_values(nodes_tau, y):
    """Lagrange basis of the 15 nodes evaluated at y, via a plain monomial solve."""
    c = nodes_tau.mean(0)
    def mono(p):
        s = p - c
        return np.stack([s[:, 0] ** a * s[:, 1] ** (d - a) for d in range(5) for a in range(d + 1)], 1)
    return mono(y) @ np.linalg.inv(mono(nodes_tau))


def _gl01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1) / 2, w / 2


def _element_points(mesh, t, xi, eta):
    V = mesh.vertices[mesh.tris[t]]
    curve, t0, t1, e = None, 0.0, 0.0, -1
    for ee in range(3):
        if mesh.edge_curve[t, ee] >= 0:
            curve = mesh.curves[mesh.edge_curve[t, ee]]
            t0, t1 = mesh.edge_theta[t, ee]
            e = ee
    x, y = _element_map(V, curve, t0, t1, e, xi, eta)
    hs = 1e-30
    xa, ya = _element_map(V, curve, t0, t1, e, xi + 1j * hs, eta + 0j)
    xb, yb = _element_map(V, curve, t0, t1, e, xi + 0j, eta + 1j * hs)
    J = (xa.imag * yb.imag - xb.imag * ya.imag) / hs**2
    return np.stack([np.real(x), np.real(y)], 1), J


def _duffy(P, n_u, graded):
    """Points/weights of the reference sub-triangle P[0], P[1], P[2] collapsed at P[0]."""
    us, uw = [], []
    edges = [0.0] + [2.0 ** (-m) for m in range(40, 0, -1)] + [1.0] if graded else [0.0, 1.0]
    xg, wg = _gl01(n_u)
    for a, b in zip(edges[:-1], edges[1:]):
        us.append(a + (b - a) * xg)
        uw.append((b - a) * wg)
    u, wu = np.concatenate(us), np.concatenate(uw)
    v, wv = _gl01(n_u)
    U, Vv = np.meshgrid(u, v, indexing="ij")
    W = np.outer(wu, wv) * U
    pts = P[0] + U[..., None] * ((1 - Vv)[..., None] * (P[1] - P[0]) + Vv[..., None] * (P[2] - P[0]))
    area2 = abs((P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[1, 1] - P[0, 1]) * (P[2, 0] - P[0, 0]))
    return pts.reshape(-1, 2), (W * area2).ravel()


def _brute_element(mesh, t, x, xref, fvals):
    """int over element t of G(x, y) L(y) dy by singularity-adapted tensor rules."""
    ref = [np.array([0.0, 0.0]), np.array([1.0, 0.0]), np.array([0.0, 1.0])]
    pieces = []
    if xref is not None:                   # target inside: split at the target, Duffy + grading
        for a in range(3):
            pieces.append(_duffy(np.array([xref, ref[a], ref[(a + 1) % 3]]), 24, True))
    else:                                  # 4^3 sub-triangles, each collapsed at a corner
        tris = [np.array(ref)]
        for _ in range(3):
            new = []
            for T in tris:
                m01, m12, m20 = (T[0] + T[1]) / 2, (T[1] + T[2]) / 2, (T[2] + T[0]) / 2
                new += [np.array([T[0], m01, m20]), np.array([m01, T[1], m12]),
                        np.array([m20, m12, T[2]]), np.array([m01, m12, m20])]
            tris = new
        for T in tris:
            pieces.append(_duffy(T, 24, False))
    total = 0
    for pts, w in pieces:
        y, J = _element_points(mesh, t, pts[:, 0], pts[:, 1])
        r = np.hypot(y[:, 0] - x[0], y[:, 1] - x[1])
        g = 0.25j * sp.hankel1(0, 5.0 * r)
        total = total + (w * J * g) @ fvals(y)
    return total


def test_green_identity_vs_brute_force():
    # E_jq = int_patch G L_q (Green's identity, boundary integrals) equals a
    # direct 2-D singular quadrature of G L_q over the patch elements.
    k = 5.0
    mesh = disk_mesh(1)          # 6 curved triangles
    rx, ry, _ = load_rule()
    j = 4                        # node 4 of element 0
    tau = j // N_Q
    elems = np.arange(mesh.n_elem)
    dV = vdim.correction_block(mesh, j, k, elems, tau, own=True)
    nodes_tau = mesh.nodes[tau * N_Q:(tau + 1) * N_Q]
    x = mesh.nodes[j]
    idx = np.array([i for i in range(mesh.n_nodes) if i != j])
    r = np.hypot(mesh.nodes[idx, 0] - x[0], mesh.nodes[idx, 1] - x[1])
    N = (0.25j * sp.hankel1(0, k * r) * mesh.weights[idx]) @ _lagrange_values(nodes_tau, mesh.nodes[idx])
    E_identity = dV + N
    fv = lambda y: _lagrange_values(nodes_tau, y)
    E_brute = sum(_brute_element(mesh, t, x, np.array([rx[4], ry[4]]) if t == tau else None, fv) for t in elems)
    assert np.max(np.abs(E_identity - E_brute)) < 1e-10 * np.max(np.abs(E_brute))
