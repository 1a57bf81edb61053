"""Adjoint-state gradient of a far-field misfit with respect to the nodal contrast.

Misfit J(m) = 1/2 sum_d sum_a |u_inf^(d)(theta_a) - t_a^(d)|^2 over incident
directions d and receiver angles theta_a, with u^(d) = L(m)^{-1} b^(d),
L(m) = I + k^2 V diag(m) (Eq. linear_system_matrix; V does not depend on m) and
u_inf(theta_a) = sum_j A_aj m_j u_j, A_aj = -k^2 e^{i pi/4}/sqrt(8 pi k) w_j
e^{-i k xhat_a . y_j} (the far-field formula of oracle.farfield).

For real m (differentiating the real part of each nodal contrast):
    dJ/dm_j = Re sum_d u_j^(d) [ g_j^(d) - k^2 (V^T lambda^(d))_j ],
    g^(d) = A^T conj(r^(d)),  L^T lambda^(d) = m * g^(d),
which follows from dL/dm_j = k^2 V e_j e_j^T and du/dm_j = -k^2 u_j L^{-1} V e_j.
Dense matrices: small meshes only.  Pinned against central finite differences
of the same misfit (tests/test_oracle_adjoint.py).
"""
import numpy as np


def far_field_matrix(nodes, weights, k, angles):
    gamma = np.exp(1j * np.pi / 4) / np.sqrt(8 * np.pi * k)
    xh = np.stack([np.cos(angles), np.sin(angles)], axis=1)
    return -k**2 * gamma * np.exp(-1j * k * (xh @ nodes.T)) * weights[None, :]


class DenseMisfit:
    """J(m) and its adjoint gradient from the dense potential matrix V."""

    def __init__(self, V, k, b_list, A, targets):
        self.V, self.k, self.b, self.A, self.t = V, float(k), b_list, A, targets

    def L(self, m):
        return np.eye(self.V.shape[0], dtype=np.complex128) + self.k**2 * self.V * m[None, :]

    def value(self, m):
        U = np.linalg.solve(self.L(m), np.stack(self.b, axis=1))
        J = 0.0
        for c, t in enumerate(self.t):
            r = self.A @ (m * U[:, c]) - t
            J += 0.5 * np.sum(np.abs(r) ** 2)
        return J

    def gradient(self, m):
        Lm = self.L(m)
        grad = np.zeros(m.size)
        for b, t in zip(self.b, self.t):
            u = np.linalg.solve(Lm, b)
            r = self.A @ (m * u) - t
            g = self.A.T @ np.conj(r)
            lam = np.linalg.solve(Lm.T, m * g)
            grad += np.real(u * (g - self.k**2 * (self.V.T @ lam)))
        return grad
