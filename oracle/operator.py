"""The Nystrom operator L = I + k^2 V M (Eq. linear_system_matrix).

V = naive pair sum + VDIM correction dV (Eq. DIM_map, Eq. DIM_decomp) and
M = diag(m(y_j)).  (L u)_j = u_j + k^2 [sum_{n != j} G(y_j, y_n) w_n m_n u_n
+ sum_q dV_jq m_q u_q].  The incident field is b_j = exp(i k d . y_j)
(Eq. nystrom_linear_system, b_j = u_inc(y_j)).
"""
import numpy as np

from .bessel import hankel01
from .nystrom import naive_rows
from .vdim import correction_matrix


class Operator:
    """Plain FP64 operator on a mesh (correction assembled on demand)."""

    def __init__(self, mesh, k, m, kappa=3.0, rows_only=None):
        self.mesh, self.k, self.m, self.kappa = mesh, float(k), np.asarray(m, np.complex128), kappa
        self._dV = None
        if rows_only is None:
            self._dV = correction_matrix(mesh, k, kappa)

    @property
    def n(self):
        return self.mesh.n_nodes

    @property
    def dV(self):
        if self._dV is None:
            self._dV = correction_matrix(self.mesh, self.k, self.kappa)
        return self._dV

    def naive_matrix(self):
        """Dense naive kernel matrix K_jn = G(y_j, y_n) w_n (n != j); small meshes."""
        if getattr(self, "_K", None) is None:
            n = self.n
            nodes, w = self.mesh.nodes, self.mesh.weights
            K = np.empty((n, n), dtype=np.complex128)
            rows = np.arange(n)
            for r0 in range(0, n, 256):
                r = rows[r0:r0 + 256]
                dx = nodes[r, 0][:, None] - nodes[None, :, 0]
                dy = nodes[r, 1][:, None] - nodes[None, :, 1]
                dist = np.sqrt(dx * dx + dy * dy)
                selfm = np.zeros(dist.shape, dtype=bool)
                selfm[np.arange(r.size), r] = True
                dist[selfm] = 1.0
                h0, _ = hankel01(self.k * dist)
                g = 0.25j * h0 * w[None, :]
                g[selfm] = 0.0
                K[r0:r0 + 256] = g
            self._K = K
        return self._K

    def potential(self, f):
        """V f = naive(f) + dV f at every node."""
        if self.n <= 6000:
            return self.naive_matrix() @ f + self.dV @ f
        nodes, w = self.mesh.nodes, self.mesh.weights
        return naive_rows(nodes, w, self.k, f, np.arange(self.n)) + self.dV @ f

    def apply(self, u):
        return u + self.k**2 * self.potential(self.m * u)

    def apply_rows(self, u, rows):
        """(L u)[rows] without assembling the full correction."""
        rows = np.asarray(rows)
        f = self.m * u
        nodes, w = self.mesh.nodes, self.mesh.weights
        dVr = correction_matrix(self.mesh, self.k, self.kappa, rows=rows)
        return u[rows] + self.k**2 * (naive_rows(nodes, w, self.k, f, rows) + dVr @ f)

    def dense(self):
        """Dense L = I + k^2 (K + dV) M (small meshes only)."""
        V = self.naive_matrix() + self.dV.toarray()
        return np.eye(self.n, dtype=np.complex128) + self.k**2 * V * self.m[None, :]


def plane_wave(nodes, k, angle):
    """u_inc(y) = exp(i k d . y), d = (cos angle, sin angle)."""
    d = np.array([np.cos(angle), np.sin(angle)])
    return np.exp(1j * k * (nodes @ d))
