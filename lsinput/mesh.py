"""Synthetic curved, interface-conforming triangle meshes with 15-node quadrature.

Seeded input generation shared by the oracle, the tests and the benchmark.  It
holds geometry and quadrature only, none of the solver's arithmetic.

Geometry (Section 3 of the paper: a conforming curved triangulation of every
subdomain on which the contrast is smooth; exact curved elements for the disk,
Section 6.1; meshes of different subdomains need not match across an interface):

* every element is a triangle (v0, v1, v2) in counter-clockwise order; edge e
  runs from v_e to v_{(e+1) % 3};
* an edge is either straight or an arc of a *polar curve*
  gamma(theta) = c + R (1 + a cos(m theta + phi)) (cos theta, sin theta)
  (a = 0 gives a circle), traversed from theta_start to theta_end;
* an element has at most one curved edge; its map from the reference triangle
  is the affine map plus a smooth edge-bubble blending term that moves that
  edge onto the curve and keeps the other two edges straight, so neighbouring
  elements of one subdomain share their edges exactly;
* quadrature nodes are the images of the 15 reference nodes and the weights are
  the reference weights times |det DF| (DF from a complex-step derivative, exact
  to round-off for these analytic maps).
"""
from dataclasses import dataclass, field
import os

import numpy as np

N_Q = 15


def load_rule():
    """Reference 15-node rule (x, y, w) on the triangle (0,0),(1,0),(0,1)."""
    path = os.path.join(os.path.dirname(__file__), "tri15.txt")
    data = np.loadtxt(path)
    return data[:, 0].copy(), data[:, 1].copy(), data[:, 2].copy()


def curve_point(curve, theta):
    """gamma(theta) for curve = (cx, cy, R, a, m, phi); theta may be complex."""
    cx, cy, R, a, m, phi = curve
    r = R * (1.0 + a * np.cos(m * theta + phi))
    return cx + r * np.cos(theta), cy + r * np.sin(theta)


@dataclass
class Mesh:
    vertices: np.ndarray            # [NV, 2] float64
    tris: np.ndarray                # [NT, 3] int32, counter-clockwise
    domain: np.ndarray              # [NT] int32 subdomain id
    edge_curve: np.ndarray          # [NT, 3] int32, -1 straight else curve id
    edge_theta: np.ndarray          # [NT, 3, 2] float64 (theta_start, theta_end)
    curves: np.ndarray              # [NC, 6] float64 (cx, cy, R, a, m, phi)
    nodes: np.ndarray = field(default=None)    # [NQ, 2]
    weights: np.ndarray = field(default=None)  # [NQ]

    @property
    def n_elem(self):
        return int(self.tris.shape[0])

    @property
    def n_nodes(self):
        return int(self.n_elem * N_Q)

    @property
    def node_domain(self):
        return np.repeat(self.domain, N_Q)


class _Builder:
    def __init__(self):
        self.verts, self.tris, self.dom, self.ecurve, self.etheta = [], [], [], [], []

    def add_vertex(self, x, y):
        self.verts.append((float(x), float(y)))
        return len(self.verts) - 1

    def add_tri(self, v, domain, curved=None):
        """curved = (edge index, curve id, theta_start, theta_end) or None."""
        P = np.array([self.verts[i] for i in v])
        area2 = (P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[1, 1] - P[0, 1]) * (P[2, 0] - P[0, 0])
        if area2 <= 0:
            raise ValueError("clockwise or degenerate triangle")
        ec = [-1, -1, -1]
        et = [[0.0, 0.0], [0.0, 0.0], [0.0, 0.0]]
        if curved is not None:
            e, cid, t0, t1 = curved
            ec[e] = cid
            et[e] = [t0, t1]
        self.tris.append(tuple(v))
        self.dom.append(domain)
        self.ecurve.append(ec)
        self.etheta.append(et)


def _hex_disk(b, curve_id, curve, n_rings, domain):
    """Star-shaped region {c + rho r(theta) e_theta : rho <= 1} meshed by 6 n^2
    triangles: ring i (i = 1..n) holds 6 i vertices at rho = i / n."""
    cx, cy = curve[0], curve[1]

    def place(rho, th):
        if rho == 0.0:
            return b.add_vertex(cx, cy)
        if rho == 1.0:
            x, y = curve_point(curve, th)
            return b.add_vertex(x, y)
        x, y = curve_point(curve, th)
        return b.add_vertex(cx + rho * (x - cx), cy + rho * (y - cy))

    rings = [[place(0.0, 0.0)]]
    angles = [[0.0]]
    for i in range(1, n_rings + 1):
        n = 6 * i
        th = [2.0 * np.pi * j / n for j in range(n)]
        rings.append([place(i / n_rings, t) for t in th])
        angles.append(th)
    for i in range(1, n_rings + 1):
        inner, outer = rings[i - 1], rings[i]
        nb = len(outer)
        outermost = i == n_rings

        def tri_outer(a_idx, jb):
            jn = (jb + 1) % nb
            v = (inner[a_idx], outer[jb], outer[jn])
            curved = None
            if outermost:
                t0 = angles[i][jb]
                t1 = angles[i][jn] if jn != 0 else 2.0 * np.pi
                curved = (1, curve_id, t0, t1)
            b.add_tri(v, domain, curved)

        if i == 1:
            for jb in range(nb):
                tri_outer(0, jb)
            continue
        na = len(inner)
        ia = ib = 0
        while ia < na or ib < nb:
            ta_next = 2.0 * np.pi * (ia + 1) / na
            tb_next = 2.0 * np.pi * (ib + 1) / nb
            if ib < nb and (ia == na or tb_next <= ta_next + 1e-13):
                tri_outer(ia % na, ib)
                ib += 1
            else:
                b.add_tri((inner[ia % na], outer[ib % nb], inner[(ia + 1) % na]), domain)
                ia += 1


def _blend_annulus(b, inner_id, inner, outer_id, outer, n_s, n_theta, domain):
    """Region between two polar curves sharing the parameter theta, meshed on
    the (s, theta) grid of B(s, theta) = (1-s) gamma_in + s gamma_out."""
    idx = np.zeros((n_s + 1, n_theta), dtype=np.int64)
    for i in range(n_s + 1):
        s = i / n_s
        for j in range(n_theta):
            th = 2.0 * np.pi * j / n_theta
            xi, yi = curve_point(inner, th)
            xo, yo = curve_point(outer, th)
            if i == 0:
                idx[i, j] = b.add_vertex(xi, yi)
            elif i == n_s:
                idx[i, j] = b.add_vertex(xo, yo)
            else:
                idx[i, j] = b.add_vertex((1 - s) * xi + s * xo, (1 - s) * yi + s * yo)
    for i in range(n_s):
        for j in range(n_theta):
            jn = (j + 1) % n_theta
            t0 = 2.0 * np.pi * j / n_theta
            t1 = 2.0 * np.pi * (j + 1) / n_theta
            # lower-right triangle: (i,j) -> (i+1,j) -> (i+1,j+1)
            curved = (1, outer_id, t0, t1) if i + 1 == n_s else None
            b.add_tri((idx[i, j], idx[i + 1, j], idx[i + 1, jn]), domain, curved)
            # upper-left triangle: (i,j) -> (i+1,j+1) -> (i,j+1)
            curved = (2, inner_id, t1, t0) if i == 0 else None
            b.add_tri((idx[i, j], idx[i + 1, jn], idx[i, jn]), domain, curved)


def _element_map(V, curve, t0, t1, e, xi, eta):
    """Physical point of reference point (xi, eta) (arrays; may be complex)."""
    lam = [1.0 - xi - eta, xi, eta]
    x = lam[0] * V[0, 0] + lam[1] * V[1, 0] + lam[2] * V[2, 0]
    y = lam[0] * V[0, 1] + lam[1] * V[1, 1] + lam[2] * V[2, 1]
    if curve is None:
        return x, y
    i, j = e, (e + 1) % 3
    li, lj = lam[i], lam[j]
    # Smooth edge-bubble blending: 4 li lj d(t), t = (1 + lj - li) / 2, with
    # d(t) = (gamma(theta(t)) - chord(t)) / (4 t (1 - t)); on the curved edge
    # (li + lj = 1) t = lj and the edge lands on the curve, and the other two
    # edges (li = 0 or lj = 0) stay straight.
    t = 0.5 * (1.0 + lj - li)
    gx, gy = curve_point(curve, t0 + t * (t1 - t0))
    den = 4.0 * t * (1.0 - t)
    dx = (gx - ((1 - t) * V[i, 0] + t * V[j, 0])) / den
    dy = (gy - ((1 - t) * V[i, 1] + t * V[j, 1])) / den
    x = x + 4.0 * li * lj * dx
    y = y + 4.0 * li * lj * dy
    return x, y


def map_nodes(mesh):
    """Fill mesh.nodes / mesh.weights (element-major, 15 nodes per element)."""
    rx, ry, rw = load_rule()
    NT = mesh.n_elem
    nodes = np.zeros((NT * N_Q, 2))
    weights = np.zeros(NT * N_Q)
    hstep = 1e-30
    for t in range(NT):
        V = mesh.vertices[mesh.tris[t]]
        curve, t0, t1, e = None, 0.0, 0.0, -1
        for ee in range(3):
            if mesh.edge_curve[t, ee] >= 0:
                curve = mesh.curves[mesh.edge_curve[t, ee]]
                t0, t1 = mesh.edge_theta[t, ee]
                e = ee
        x, y = _element_map(V, curve, t0, t1, e, rx, ry)
        xa, ya = _element_map(V, curve, t0, t1, e, rx + 1j * hstep, ry + 0j)
        xb, yb = _element_map(V, curve, t0, t1, e, rx + 0j, ry + 1j * hstep)
        J = (np.imag(xa) / hstep) * (np.imag(yb) / hstep) - (np.imag(xb) / hstep) * (np.imag(ya) / hstep)
        if np.any(J <= 0):
            raise ValueError(f"non-positive Jacobian in element {t}")
        nodes[t * N_Q:(t + 1) * N_Q, 0] = np.real(x)
        nodes[t * N_Q:(t + 1) * N_Q, 1] = np.real(y)
        weights[t * N_Q:(t + 1) * N_Q] = rw * J
    mesh.nodes, mesh.weights = nodes, weights
    return mesh


def _finish(b, curves):
    mesh = Mesh(vertices=np.array(b.verts, dtype=np.float64),
                tris=np.array(b.tris, dtype=np.int32),
                domain=np.array(b.dom, dtype=np.int32),
                edge_curve=np.array(b.ecurve, dtype=np.int32),
                edge_theta=np.array(b.etheta, dtype=np.float64),
                curves=np.array(curves, dtype=np.float64))
    return map_nodes(mesh)


def open_resonator_mesh(n_s, n_theta, r_in=0.8, r_out=1.0, theta0=np.pi / 9):
    """Truncated annulus {r_in < |x| < r_out, |theta| > theta0} (an open cavity whose
    aperture faces +x): the (s, theta) grid of the blend between the two circles over
    theta in [theta0, 2 pi - theta0], each cell split into two triangles; arcs exact,
    the two radial end edges straight."""
    inner = (0.0, 0.0, r_in, 0.0, 0.0, 0.0)
    outer = (0.0, 0.0, r_out, 0.0, 0.0, 0.0)
    b = _Builder()
    th = theta0 + (2 * np.pi - 2 * theta0) * np.arange(n_theta + 1) / n_theta
    idx = np.zeros((n_s + 1, n_theta + 1), dtype=np.int64)
    for i in range(n_s + 1):
        s_ = i / n_s
        for j in range(n_theta + 1):
            xi, yi = curve_point(inner, th[j])
            xo, yo = curve_point(outer, th[j])
            if i == 0:
                idx[i, j] = b.add_vertex(xi, yi)
            elif i == n_s:
                idx[i, j] = b.add_vertex(xo, yo)
            else:
                idx[i, j] = b.add_vertex((1 - s_) * xi + s_ * xo, (1 - s_) * yi + s_ * yo)
    for i in range(n_s):
        for j in range(n_theta):
            curved = (1, 1, th[j], th[j + 1]) if i + 1 == n_s else None
            b.add_tri((idx[i, j], idx[i + 1, j], idx[i + 1, j + 1]), 0, curved)
            curved = (2, 0, th[j + 1], th[j]) if i == 0 else None
            b.add_tri((idx[i, j], idx[i + 1, j + 1], idx[i, j + 1]), 0, curved)
    return _finish(b, [inner, outer])


def square_mesh(n, half=0.75):
    """Straight-edged mesh of the square [-half, half]^2: n x n cells, each split into
    two triangles (2 n^2 elements, one subdomain, no curved edges)."""
    g = np.linspace(-half, half, n + 1)
    X, Y = np.meshgrid(g, g)
    verts = np.stack([X.ravel(), Y.ravel()], axis=1)
    tris = []
    for b in range(n):
        for a in range(n):
            v0, v1, v2, v3 = b * (n + 1) + a, b * (n + 1) + a + 1, (b + 1) * (n + 1) + a + 1, (b + 1) * (n + 1) + a
            tris += [[v0, v1, v2], [v0, v2, v3]]
    nt = len(tris)
    mesh = Mesh(vertices=verts, tris=np.array(tris, dtype=np.int32), domain=np.zeros(nt, dtype=np.int32),
                edge_curve=np.full((nt, 3), -1, dtype=np.int32), edge_theta=np.zeros((nt, 3, 2)),
                curves=np.zeros((0, 6)))
    return map_nodes(mesh)


def disk_mesh(n_rings, radius=1.0, center=(0.0, 0.0)):
    """Single-subdomain disk: 6 n_rings^2 curved triangles (domain 0)."""
    curves = [(center[0], center[1], radius, 0.0, 0.0, 0.0)]
    b = _Builder()
    _hex_disk(b, 0, curves[0], n_rings, 0)
    return _finish(b, curves)


def inclusion_disk_mesh(n_rings_incl, n_s, n_theta, incl_center=(0.3, 0.1), incl_radius=0.3):
    """Unit disk with an off-centre circular inclusion: domain 0 is the disk
    minus the inclusion (blended annulus), domain 1 the inclusion (hex disk).
    The two meshes do not match across the interface."""
    curves = [(0.0, 0.0, 1.0, 0.0, 0.0, 0.0),
              (incl_center[0], incl_center[1], incl_radius, 0.0, 0.0, 0.0)]
    b = _Builder()
    _blend_annulus(b, 1, curves[1], 0, curves[0], n_s, n_theta, 0)
    _hex_disk(b, 1, curves[1], n_rings_incl, 1)
    return _finish(b, curves)


def star_mesh(phi, n_rings_inner, n_s, n_theta, R=1.0, amp=0.2, freq=5.0, inner_scale=0.5):
    """Star r(theta) = R (1 + amp cos(freq theta + phi)) with an inner interface
    at inner_scale * r(theta): domain 0 the outer shell, domain 1 the core."""
    curves = [(0.0, 0.0, R, amp, freq, phi),
              (0.0, 0.0, inner_scale * R, amp, freq, phi)]
    b = _Builder()
    _blend_annulus(b, 1, curves[1], 0, curves[0], n_s, n_theta, 0)
    _hex_disk(b, 1, curves[1], n_rings_inner, 1)
    return _finish(b, curves)
