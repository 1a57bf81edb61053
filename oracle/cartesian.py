"""Purely Cartesian Lippmann-Schwinger solver (test infrastructure; the paper's structured
comparison, Section 6 "Comparison with a purely Cartesian discretization").

The equation is discretised directly on the uniform grid of the box D (Eq.
LS_eq_on_cartesian_points): L^(C) = I + k^2 V^(C) M^(C), with V^(C)_il = G(z_i - z_l) h^2
for i != l and, on the diagonal, the integral of G over the disc of area h^2 (the same
reading as the preconditioner's V^(C); the Duan-Rokhlin corrected weights are not
available), M^(C) = diag(m(z_j)).  V^(C) is a two-level Toeplitz matrix, applied here by
zero-padded FFT convolution (numpy's FFT, a library primitive).  The system is solved by
GMRES left-preconditioned with the sparsifying preconditioner S^(C) = C^{-1} A
(Eq. sparsifying_min, Eq. LC_def; A and C assembled by oracle.precond, C factored by
SuperLU), or unpreconditioned.
"""
import numpy as np
import scipy.sparse.linalg as spla

from .gmres import gmres
from .precond import Preconditioner, cartesian_kernel, stencil_vectors


class CartesianLS:
    def __init__(self, grid, k, m_grid):
        self.grid, self.k = grid, float(k)
        self.m = np.asarray(m_grid, np.complex128)
        nx, ny, h = grid.nx, grid.ny, grid.h
        self.NX, self.NY = 2 * nx, 2 * ny
        da = np.arange(self.NX)
        db = np.arange(self.NY)
        da = np.where(da < nx, da, da - self.NX)             # offsets 0..nx-1, then -(nx)..-1
        db = np.where(db < ny, db, db - self.NY)
        DA, DB = np.meshgrid(da, db)
        K = cartesian_kernel(self.k, h, DA.ravel(), DB.ravel()).reshape(self.NY, self.NX)
        K[:, nx] = 0.0                                      # offset +-nx never occurs
        K[ny, :] = 0.0
        self.Khat = np.fft.fft2(K)
        # sparsifying preconditioner on the same grid and contrast (no quadrature nodes)
        P = Preconditioner.__new__(Preconditioner)
        P.grid, P.k, P.m_grid = grid, self.k, self.m
        P.v, P.sv = stencil_vectors(grid, self.k)
        P.A, P.C = P._assemble()
        self.A, self.C = P.A, P.C
        self.lu = spla.splu(self.C.tocsc())

    def potential(self, f):
        """V^(C) f by FFT convolution (f on the grid, x fastest)."""
        g = self.grid
        F = np.zeros((self.NY, self.NX), np.complex128)
        F[:g.ny, :g.nx] = f.reshape(g.ny, g.nx)
        Y = np.fft.ifft2(np.fft.fft2(F) * self.Khat)
        return Y[:g.ny, :g.nx].ravel()

    def potential_dense(self, f):
        """V^(C) f by the plain double sum (small grids only; for checking the FFT)."""
        g = self.grid
        pts = g.points()
        n = pts.shape[0]
        A_ = np.arange(g.nx)[None, :] * np.ones((g.ny, 1), int)
        B_ = np.arange(g.ny)[:, None] * np.ones((1, g.nx), int)
        a, b = A_.ravel(), B_.ravel()
        out = np.zeros(n, np.complex128)
        for i in range(n):
            out[i] = np.sum(cartesian_kernel(self.k, g.h, a[i] - a, b[i] - b) * f)
        return out

    def apply(self, u):
        return u + self.k**2 * self.potential(self.m * u)

    def S(self, x):
        return self.lu.solve(self.A @ x)

    def solve(self, b, tol=1e-8, precond=True, max_iter=600):
        """(u, residual history, iterations) of L^(C) u = b, left-preconditioned by S^(C)."""
        return gmres(self.apply, b, tol=tol, max_iter=max_iter, apply_P=self.S if precond else None)
