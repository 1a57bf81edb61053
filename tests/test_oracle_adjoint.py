"""Pin of the oracle's adjoint-state gradient: central finite differences of
the same misfit (an independent route to the derivative)."""
import numpy as np

from lsinput.workloads import constant_disk
from oracle.adjoint import DenseMisfit, far_field_matrix
from oracle.operator import Operator, plane_wave


def test_adjoint_gradient_vs_central_differences():
    wl = constant_disk(k=6.0, n_rings=2)        # 360 nodes
    op = Operator(wl.mesh, wl.k, wl.m)
    V = op.naive_matrix() + op.dV.toarray()
    x, y = wl.mesh.nodes[:, 0], wl.mesh.nodes[:, 1]
    m = 1 - (1.4 + 0.2 * np.exp(-(x**2 + y**2) / 0.2)) ** 2   # smooth, non-constant contrast
    angles = 2 * np.pi * np.arange(6) / 6
    A = far_field_matrix(wl.mesh.nodes, wl.mesh.weights, wl.k, angles)
    dirs = [0.0, np.pi / 3]
    b = [plane_wave(wl.mesh.nodes, wl.k, d) for d in dirs]
    # targets from a perturbed contrast (a Gaussian blob)
    blob = 0.05 * np.exp(-((wl.mesh.nodes[:, 0] + 0.3) ** 2 + (wl.mesh.nodes[:, 1] + 0.2) ** 2) / 0.02)
    mt = 1 - (np.sqrt(1 - m) + blob) ** 2
    Lt = np.eye(m.size) + wl.k**2 * V * mt[None, :]
    t = [A @ (mt * np.linalg.solve(Lt, bb)) for bb in b]
    J = DenseMisfit(V, wl.k, b, A, t)
    g = J.gradient(m)
    rng = np.random.default_rng(7)
    idx = rng.choice(m.size, 8, replace=False)
    h = 1e-6
    for j in idx:
        e = np.zeros(m.size)
        e[j] = h
        fd = (J.value(m + e) - J.value(m - e)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-5 * np.max(np.abs(g)), (j, fd, g[j])
