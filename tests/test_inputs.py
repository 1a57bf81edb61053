"""Pins of the seeded input generators: quadrature rule and curved meshes."""
import itertools
from math import factorial

import numpy as np
import pytest

from lsinput.mesh import load_rule, disk_mesh, inclusion_disk_mesh, star_mesh, N_Q


def test_rule_exactness_degree_7():
    # 15 interior nodes for interpolation degree p = 4 with degree of exactness > p (Section 3)
    x, y, w = load_rule()
    assert x.size == 15
    for d in range(8):
        for i in range(d + 1):
            j = d - i
            exact = factorial(i) * factorial(j) / factorial(i + j + 2)
            assert abs(np.sum(w * x**i * y**j) - exact) < 2e-16
    # degree 8 is not integrated exactly (the rule's stated degree is tight)
    errs = [abs(np.sum(w * x**i * y**(8 - i)) - factorial(i) * factorial(8 - i) / factorial(10)) for i in range(9)]
    assert max(errs) > 1e-10


def test_rule_interior_positive_unisolvent():
    x, y, w = load_rule()
    assert np.all(w > 0) and abs(w.sum() - 0.5) < 1e-16
    assert min(x.min(), y.min(), (1 - x - y).min()) >= 0.039
    V = np.stack([x**a * y**(d - a) for d in range(5) for a in range(d + 1)], axis=1)
    assert np.linalg.cond(V) < 1e4


def test_rule_symmetry():
    x, y, w = load_rule()
    lam = np.stack([1 - x - y, x, y], axis=1)
    key = lambda l: tuple(np.round(np.sort(l), 14))
    base = {key(l): wi for l, wi in zip(lam, w)}
    for perm in itertools.permutations(range(3)):
        for l, wi in zip(lam[:, perm], w):
            assert abs(base[key(l)] - wi) < 1e-15


def test_disk_area_and_jacobians():
    m = disk_mesh(3)
    assert m.n_elem == 54 and m.n_nodes == 54 * N_Q
    assert abs(m.weights.sum() - np.pi) < 1e-13
    assert np.all(m.weights > 0)
    assert np.all(np.hypot(m.nodes[:, 0], m.nodes[:, 1]) < 1.0)


def test_inclusion_mesh_subdomain_areas():
    m = inclusion_disk_mesh(2, 3, 16)
    dom = m.node_domain
    assert abs(m.weights[dom == 1].sum() - np.pi * 0.09) < 1e-12
    assert abs(m.weights[dom == 0].sum() - np.pi * 0.91) < 1e-12
    inside = (m.nodes[:, 0] - 0.3) ** 2 + (m.nodes[:, 1] - 0.1) ** 2 < 0.09
    assert np.array_equal(inside, dom == 1)


def test_star_area():
    phi = 0.7
    m = star_mesh(phi, 4, 6, 60)
    th = np.linspace(0, 2 * np.pi, 400001)[:-1]
    r = 1 + 0.2 * np.cos(5 * th + phi)
    area = np.pi * np.mean(r**2)
    assert abs(m.weights.sum() - area) < 1e-8
    assert abs(m.weights[m.node_domain == 1].sum() - 0.25 * area) < 1e-8


def test_curved_edges_on_curve():
    m = inclusion_disk_mesh(2, 3, 16)
    for t in range(m.n_elem):
        for e in range(3):
            cid = m.edge_curve[t, e]
            if cid < 0:
                continue
            cx, cy, R, a, f, ph = m.curves[cid]
            for v in (m.tris[t, e], m.tris[t, (e + 1) % 3]):
                p = m.vertices[v]
                assert abs(np.hypot(p[0] - cx, p[1] - cy) - R) < 1e-15


def test_open_resonator_mesh_area_and_contrast():
    from lsinput.workloads import open_resonator
    wl = open_resonator(n_s=2, n_theta=30)
    exact = 0.5 * (1.0 - 0.8**2) * (2 * np.pi - 2 * np.pi / 9)      # truncated annulus
    assert abs(wl.mesh.weights.sum() - exact) < 1e-13
    r = np.hypot(wl.mesh.nodes[:, 0], wl.mesh.nodes[:, 1])
    th = np.arctan2(wl.mesh.nodes[:, 1], wl.mesh.nodes[:, 0])
    assert np.all((r > 0.8) & (r < 1.0) & (np.abs(th) > np.pi / 9))
    assert np.allclose(wl.m.real, np.exp(-(((r - 0.9) / 0.1201) ** 2)))
