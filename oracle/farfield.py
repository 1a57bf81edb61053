"""Far-field pattern and the Mie (Fourier-Bessel) series of a constant disk.

Far field (normalisation u^s(x) ~ e^{ik|x|} / sqrt(|x|) u_inf(x/|x|), the
convention of Colton & Kress used by the energy balance Eq.
dissipativity_identity): letting |x| -> infinity in the representation formula
(Eq. representation_formula) with H0^(1)(t) ~ sqrt(2/(pi t)) e^{i(t - pi/4)} gives
u_inf(theta) = -k^2 e^{i pi/4} / sqrt(8 pi k) * sum_j w_j m_j u_j e^{-i k xhat . y_j}.

Mie series (the paper's reference solution for the constant-contrast disk,
Section 6.1): for the disk of radius R centred at the origin, interior
wavenumber k_i = k n_opt and a plane wave along angle alpha, the coefficients
(a_n, b_n) solve continuity of u and du/dr at r = R; u = sum a_n J_n(k_i r)
e^{i n (theta - alpha)} inside and u_inf = sqrt(2/(pi k)) e^{-i pi/4}
sum b_n (-i)^n e^{i n (theta - alpha)}.  Bessel functions of integer order
come from scipy.special (a library routine, independent of oracle.bessel).
"""
import numpy as np
import scipy.special as sp


def far_field(nodes, weights, m, u, k, angles):
    gamma = np.exp(1j * np.pi / 4) / np.sqrt(8 * np.pi * k)
    xh = np.stack([np.cos(angles), np.sin(angles)], axis=1)
    phase = np.exp(-1j * k * (xh @ nodes.T))
    return -k**2 * gamma * (phase @ (weights * m * u))


def mie_coefficients(k, n_opt, R=1.0, nmax=None):
    ki = k * n_opt
    if nmax is None:
        nmax = int(np.ceil(ki * R + 30))
    n = np.arange(-nmax, nmax + 1)
    Jn_i, dJn_i = sp.jv(n, ki * R), sp.jvp(n, ki * R)
    Jn, dJn = sp.jv(n, k * R), sp.jvp(n, k * R)
    Hn, dHn = sp.hankel1(n, k * R), sp.h1vp(n, k * R)
    rhs1 = (1j ** n) * Jn
    rhs2 = (1j ** n) * k * dJn
    # [[J_n(k_i R), -H_n(kR)], [k_i J_n'(k_i R), -k H_n'(kR)]] (a, b) = (rhs1, rhs2)
    det = Jn_i * (-k * dHn) - (-Hn) * (ki * dJn_i)
    a = (rhs1 * (-k * dHn) - (-Hn) * rhs2) / det
    b = (Jn_i * rhs2 - ki * dJn_i * rhs1) / det
    return n, a, b


def mie_interior(points, k, n_opt, alpha=0.0, R=1.0, nmax=None):
    n, a, _ = mie_coefficients(k, n_opt, R, nmax)
    r = np.hypot(points[:, 0], points[:, 1])
    th = np.arctan2(points[:, 1], points[:, 0]) - alpha
    return (sp.jv(n[None, :], k * n_opt * r[:, None]) * np.exp(1j * n[None, :] * th[:, None])) @ a


def mie_far_field(angles, k, n_opt, alpha=0.0, R=1.0, nmax=None):
    n, _, b = mie_coefficients(k, n_opt, R, nmax)
    amp = np.sqrt(2 / (np.pi * k)) * np.exp(-1j * np.pi / 4)
    return amp * (np.exp(1j * n[None, :] * (angles[:, None] - alpha)) @ (b * (-1j) ** n))
