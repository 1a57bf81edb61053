"""Unrestarted GMRES with left preconditioning (Saad & Schultz; the paper
solves Eq. nystrom_linear_system this way, Section 6).

Reading: x0 = 0; the Arnoldi basis is built for P L with modified
Gram-Schmidt; Givens rotations keep the least-squares residual
|| P (b - L x_k) || / || P b || which is the stopping quantity (tol); max_iter
defaults to 600 (the paper's cap, Table bakeoff).
"""
import numpy as np


def gmres(apply_L, b, tol=1e-10, max_iter=600, apply_P=None):
    P = apply_P if apply_P is not None else (lambda v: v)
    r0 = P(b)
    beta = np.linalg.norm(r0)
    n = b.size
    Vb = np.zeros((max_iter + 1, n), dtype=np.complex128)
    H = np.zeros((max_iter + 1, max_iter), dtype=np.complex128)
    cs = np.zeros(max_iter, dtype=np.complex128)
    sn = np.zeros(max_iter, dtype=np.complex128)
    g = np.zeros(max_iter + 1, dtype=np.complex128)
    g[0] = beta
    hist = [1.0]
    Vb[0] = r0 / beta
    it = 0
    for j in range(max_iter):
        w = P(apply_L(Vb[j]))
        for i in range(j + 1):                     # modified Gram-Schmidt
            H[i, j] = np.vdot(Vb[i], w)
            w = w - H[i, j] * Vb[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] > 0:
            Vb[j + 1] = w / H[j + 1, j]
        for i in range(j):                         # previous rotations
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
            H[i, j] = t
        a, bb = H[j, j], H[j + 1, j]
        den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
        cs[j] = np.conj(a) / den                   # rotation [[c, s], [-conj(s), conj(c)]]
        sn[j] = np.conj(bb) / den
        H[j, j] = den
        H[j + 1, j] = 0
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        it = j + 1
        hist.append(abs(g[j + 1]) / beta)
        if hist[-1] <= tol:
            break
    y = np.linalg.solve(np.triu(H[:it, :it]), g[:it])
    x = Vb[:it].T @ y
    return x, np.array(hist), it


def ritz_values(apply_L, b, n_steps, apply_P=None):
    """Ritz values of P L: the eigenvalues of the square Hessenberg matrix of n_steps
    Arnoldi steps started from P b, with reorthogonalization (modified Gram-Schmidt, two
    passes; Section 6, Figure ritz_spectrum); fewer when the Krylov space is exhausted."""
    P = apply_P if apply_P is not None else (lambda v: v)
    r0 = P(b)
    n = b.size
    V = np.zeros((n_steps + 1, n), dtype=np.complex128)
    H = np.zeros((n_steps + 1, n_steps), dtype=np.complex128)
    V[0] = r0 / np.linalg.norm(r0)
    k = n_steps
    for j in range(n_steps):
        w = P(apply_L(V[j]))
        for _ in range(2):
            for i in range(j + 1):
                c = np.vdot(V[i], w)
                H[i, j] += c
                w = w - c * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] < 1e-14 * np.abs(H[:j + 1, j]).max():
            k = j + 1
            break
        V[j + 1] = w / H[j + 1, j]
    return np.linalg.eigvals(H[:k, :k])
