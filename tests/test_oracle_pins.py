"""Pins of the oracle against closed forms and invariants of the continuous problem.

* Polynomial exactness (Eq. DIM_decomp, global form kappa = inf): for a density f
  that is a polynomial of degree <= p = 4 on the subdomain, the interpolant on
  every element equals f, so V_h[f](x_j) must equal the exact volume potential
  V[f](x_j) = int_Omega G(x_j, y) f(y) dy up to rounding.  The exact potential of
  a monomial on the unit disk is computed here independently of the oracle, by
  the Graf addition theorem G(x, y) = (i/4) sum_n J_n(k r_<) H_n(k r_>) e^{in(t_x - t_y)}:
  V[f](x) = (i pi / 2) sum_n e^{i n t_x} [H_n(k r) int_0^r J_n(k s) f_n(s) s ds
                                         + J_n(k r) int_r^R H_n(k s) f_n(s) s ds],
  f_n the Fourier modes of f, the radial integrals by Gauss-Legendre (scipy Bessel).
  Monomials of degree 2-4 exercise the Laplacian terms of Phi_q.
* Radial non-constant density f = J0(kappa |x|), kappa != k: (Delta + k^2) applied
  to -J0(kappa r) / (k^2 - kappa^2) gives -f, and matching at r = R with the Lommel
  integrals of J0 and H0 gives, for r < R,
  V[f](x) = -J0(kappa r)/(k^2 - kappa^2)
            + (i pi R / 2) [k H1(kR) J0(kappa R) - kappa H0(kR) J1(kappa R)] J0(k r) / (k^2 - kappa^2)
  (kappa -> 0 recovers the V[1] formula).  f is not a polynomial, so V_h[f] converges
  at the high order of the method (Section 3), measured here under refinement.
* Far-field reciprocity u_inf(xhat; d) = u_inf(-d; -xhat) of the continuous
  scattering problem (the far-field operator of a penetrable medium is symmetric):
  the oracle's discrete solutions reproduce it to discretisation error on the
  two-material workload, which has no symmetry that would make it hold trivially
  for the chosen angles; a sign error in the far-field phase breaks it at O(1).
"""
import numpy as np
import pytest
import scipy.special as sp

from lsinput.mesh import disk_mesh
from lsinput.workloads import two_material
from oracle import vdim
from oracle.farfield import far_field
from oracle.nystrom import naive_apply, naive_rows
from oracle.operator import Operator, plane_wave


def _gl(n, a, b):
    x, w = np.polynomial.legendre.leggauss(n)
    a = np.asarray(a, float)[:, None]
    b = np.asarray(b, float)[:, None]
    return a + (b - a) * (x[None, :] + 1) / 2, (b - a) * w[None, :] / 2


def _radial_integral(fun, a, b, n=40):
    """int_a^b fun(s) ds per row for arrays a <= b, on geometrically graded panels
    [a, 2a, 4a, ..., b] (fun may behave like s^m log s near 0)."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    total = np.zeros(a.shape, complex)
    lo = a.copy()
    while True:
        hi = np.minimum(np.maximum(2 * lo, lo + 1e-3), b)
        act = hi > lo
        if not np.any(act):
            break
        s, w = _gl(n, lo[act], hi[act])
        total[act] += np.sum(w * fun(s), axis=1)
        lo = np.where(act, hi, lo)
    return total


def exact_potential_monomial(a, b, k, pts, R=1.0):
    """V[x^a y^b](pts) on the disk of radius R (addition theorem, see module doc)."""
    d = a + b
    M = 32
    th = 2 * np.pi * np.arange(M) / M
    c = np.fft.fft(np.cos(th) ** a * np.sin(th) ** b) / M     # exact Fourier modes, |n| <= d
    r = np.hypot(pts[:, 0], pts[:, 1])
    tx = np.arctan2(pts[:, 1], pts[:, 0])
    out = np.zeros(len(pts), complex)
    for n in range(-d, d + 1):
        cn = c[n % M]
        if abs(cn) < 1e-14:
            continue
        s, w = _gl(60, np.zeros_like(r), r)
        inner = np.sum(w * sp.jv(n, k * s) * s ** (d + 1), axis=1)
        outer = _radial_integral(lambda s: sp.hankel1(n, k * s) * s ** (d + 1), r, np.full_like(r, R))
        # H_n(k r) times the inner integral vanishes as r -> 0 (the integral is O(r^(n+d+2)))
        hin = np.where(r > 0, sp.hankel1(n, k * np.where(r > 0, r, 1.0)) * inner, 0.0)
        out += cn * np.exp(1j * n * tx) * (1j * np.pi / 2) * (hin + sp.jv(n, k * r) * outer)
    return out


def exact_potential_j0(k, kap, r, R=1.0):
    """V[J0(kap |.|)] inside the disk of radius R (closed form, see module doc)."""
    c = (1j * np.pi * R / 2) * (k * sp.hankel1(1, k * R) * sp.j0(kap * R) - kap * sp.hankel1(0, k * R) * sp.j1(kap * R))
    return (-sp.j0(kap * r) + c * sp.j0(k * r)) / (k**2 - kap**2)


def test_reference_potential_reduces_to_constant_closed_form():
    # the addition-theorem reference itself, for f = 1, against V[1] (and J0 at kap -> 0)
    k = 5.0
    pts = np.array([[0.0, 0.0], [0.3, -0.2], [0.71, 0.5], [-0.05, 0.97]])
    r = np.hypot(pts[:, 0], pts[:, 1])
    v1 = -1 / k**2 + (1j * np.pi * sp.hankel1(1, k) / (2 * k)) * sp.j0(k * r)
    assert np.max(np.abs(exact_potential_monomial(0, 0, k, pts) - v1)) < 1e-12 * np.max(np.abs(v1))
    assert np.max(np.abs(exact_potential_j0(k, 1e-7, r) - v1)) < 1e-12


@pytest.fixture(scope="module")
def global_correction_disk():
    k = 5.0
    mesh = disk_mesh(2)
    return k, mesh, vdim.correction_matrix(mesh, k, np.inf)


@pytest.mark.parametrize("deg", [1, 2, 3, 4])
def test_polynomial_density_exact_global_form(global_correction_disk, deg):
    k, mesh, dV = global_correction_disk
    x, y = mesh.nodes[:, 0], mesh.nodes[:, 1]
    for a in range(deg, -1, -1):
        b = deg - a
        f = (x**a * y**b).astype(complex)
        vh = naive_apply(mesh.nodes, mesh.weights, k, f) + dV @ f
        ex = exact_potential_monomial(a, b, k, mesh.nodes)
        assert np.max(np.abs(vh - ex)) < 1e-12 * np.max(np.abs(ex)), (a, b)


def test_polynomial_pin_detects_dropped_bilaplacian_term(global_correction_disk, monkeypatch):
    # planted mistake in the oracle: Phi_q without its Delta^2 L_q / k^6 term is still
    # exact for degree <= 3 but must fail the degree-4 pin
    k, mesh, _ = global_correction_disk
    good = vdim.lagrange_and_phi

    def phi_without_bilaplacian(nodes_tau, c, h, kk):
        C, _ = good(nodes_tau, c, h, kk)
        D = vdim._laplacian_matrix(h)
        k2 = vdim.LD(kk) * vdim.LD(kk)
        return C, C / k2 - (D @ C) / k2**2

    monkeypatch.setattr(vdim, "lagrange_and_phi", phi_without_bilaplacian)
    rows = np.arange(0, mesh.n_nodes, 9)
    dV = vdim.correction_matrix(mesh, k, np.inf, rows=rows)
    x, y = mesh.nodes[:, 0], mesh.nodes[:, 1]
    f = (x**4).astype(complex)
    vh = naive_rows(mesh.nodes, mesh.weights, k, f, rows) + dV @ f
    ex = exact_potential_monomial(4, 0, k, mesh.nodes[rows])
    assert np.max(np.abs(vh - ex)) > 1e-6 * np.max(np.abs(ex))


def test_radial_bessel_density_closed_form_and_order():
    k, kap = 5.0, 3.0
    errs = []
    for nr in (3, 4):
        mesh = disk_mesh(nr)
        rows = np.arange(0, mesh.n_nodes, 7)
        r = np.hypot(mesh.nodes[:, 0], mesh.nodes[:, 1])
        f = sp.j0(kap * r).astype(complex)
        dV = vdim.correction_matrix(mesh, k, 3.0, rows=rows)
        vh = naive_rows(mesh.nodes, mesh.weights, k, f, rows) + dV @ f
        ex = exact_potential_j0(k, kap, r[rows])
        errs.append(np.max(np.abs(vh - ex)) / np.max(np.abs(ex)))
    # measured 1.1e-6 and 6.3e-8; element size ratio 4/3, order p + 3 = 7 at least
    assert errs[0] < 3e-6 and errs[1] < 2e-7
    assert errs[0] / errs[1] > (4 / 3) ** 7


def _far_field_wrong_sign(nodes, w, m, u, k, angles):
    gamma = np.exp(1j * np.pi / 4) / np.sqrt(8 * np.pi * k)
    xh = np.stack([np.cos(angles), np.sin(angles)], axis=1)
    return -k**2 * gamma * (np.exp(1j * k * (xh @ nodes.T)) @ (w * m * u))


def test_far_field_reciprocity_two_material():
    wl = two_material("tiny", k=5.0)
    op = Operator(wl.mesh, wl.k, wl.m, kappa=3.0)
    angs = np.array([0.0, 0.7, 2.1, 3.9, 5.5])
    B = np.stack([plane_wave(wl.mesh.nodes, wl.k, a) for a in angs], 1)
    U = np.linalg.solve(op.dense(), B)
    nodes, w = wl.mesh.nodes, wl.mesh.weights

    def table(ff):
        # T[i, a] = u_inf(xhat = angs[a] + pi; d = angs[i]); reciprocity says T = T^T
        return np.stack([ff(nodes, w, wl.m, U[:, i], wl.k, angs + np.pi) for i in range(len(angs))], 0)

    T = table(far_field)
    err = np.max(np.abs(T - T.T)) / np.max(np.abs(T))
    assert err < 2e-4                    # measured 4.4e-5 on 1,800 nodes
    Tb = table(_far_field_wrong_sign)
    assert np.max(np.abs(Tb - Tb.T)) / np.max(np.abs(Tb)) > 0.1
