"""Invertibility diagnostics of the preconditioner (test infrastructure; the paper's appendix
on invertibility conditions in practice).

rho(w) = <S^(C) w, w>_D / ||w||_D^2 (Eq. rho_def) with <x, y>_D = x^* D y (Eq. D_inner_product),
D the Approach II column sums (Eq. D_def), sampled over w = R_II x = T_Q^C,II T_C^Q x for
x with standard complex normal entries (Eq. rho_ranges).
"""
import numpy as np

from .precond import Preconditioner


def rho_samples(grid, nodes, k, m_grid, n_samples, seed=0):
    P = Preconditioner(grid, nodes, k, m_grid)
    rng = np.random.default_rng(seed)
    out = np.empty(n_samples, np.complex128)
    for s in range(n_samples):
        x = (rng.standard_normal(grid.n) + 1j * rng.standard_normal(grid.n)) / np.sqrt(2)
        w = P.TQC @ (P.T @ x)
        Sw = P.lu.solve(P.A @ w)
        out[s] = np.sum(P.D * np.conj(Sw) * w) / np.sum(P.D * np.abs(w) ** 2)
    return out
