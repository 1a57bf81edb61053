"""Pins of the oracle's Hankel routine: scipy (AMOS), the Wronskian, mpmath."""
import numpy as np
import pytest
import scipy.special as sp

from oracle.bessel import bessel01, hankel01


def test_hankel_vs_scipy():
    z = np.logspace(-8, 4, 20000)
    h0, h1 = hankel01(z)
    r0 = sp.hankel1(0, z)
    r1 = sp.hankel1(1, z)
    assert np.max(np.abs(h0 - r0) / np.abs(r0)) < 5e-15
    assert np.max(np.abs(h1 - r1) / np.abs(r1)) < 5e-15


def test_wronskian():
    # J1 Y0 - J0 Y1 = 2 / (pi z)  (A&S 9.1.16), across all three branches
    z = np.concatenate([np.logspace(-6, 0.6, 500), np.linspace(3.9, 4.1, 50), np.linspace(4, 25, 500),
                        np.linspace(24.9, 25.1, 50), np.logspace(1.4, 3.5, 500)])
    j0, j1, y0, y1 = bessel01(z)
    w = (j1 * y0 - j0 * y1) * np.pi * z / 2
    assert np.max(np.abs(w - 1)) < 1e-14


def test_small_argument_limit():
    z = np.array([1e-10, 1e-8])
    j0, j1, y0, y1 = bessel01(z)
    assert np.allclose(y0, (2 / np.pi) * (np.log(z / 2) + np.euler_gamma), rtol=1e-15)
    assert np.allclose(y1, -2 / (np.pi * z), rtol=1e-15)


def test_long_double_vs_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    z = np.array([1e-5, 0.3, 2.0, 3.999, 4.001, 7.3, 13.6, 24.99, 25.01, 40.0, 333.3])
    h0, h1 = hankel01(z.astype(np.longdouble))
    assert h0.dtype == np.clongdouble
    for zi, a, b in zip(z, h0, h1):
        A = mpmath.hankel1(0, mpmath.mpf(float(zi)))
        B = mpmath.hankel1(1, mpmath.mpf(float(zi)))
        ea = abs(mpmath.mpf(str(a.real)) + 1j * mpmath.mpf(str(a.imag)) - A) / abs(A)
        eb = abs(mpmath.mpf(str(b.real)) + 1j * mpmath.mpf(str(b.imag)) - B) / abs(B)
        assert float(ea) < 3e-18 and float(eb) < 3e-18, (zi, float(ea), float(eb))
