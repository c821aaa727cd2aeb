"""Mie series for a homogeneous sphere (oracle; test infrastructure only).

Used to check that DDA efficiencies of a sphere approach the exact result
as the dipole count grows.  The series follows the standard recurrences of
Bohren & Huffman (1983), ch. 4: the logarithmic derivative D_n(mx) by
downward recurrence, the Riccati-Bessel functions psi_n(x) and chi_n(x) by
upward recurrence, and

    a_n = [(D_n/m + n/x) psi_n - psi_{n-1}] / [(D_n/m + n/x) xi_n - xi_{n-1}]
    b_n = [(m D_n + n/x) psi_n - psi_{n-1}] / [(m D_n + n/x) xi_n - xi_{n-1}]
    Q_ext = (2/x^2) sum (2n+1) Re(a_n + b_n)
    Q_sca = (2/x^2) sum (2n+1) (|a_n|^2 + |b_n|^2),

with xi_n = psi_n - i chi_n and the series cut at n = x + 4 x^(1/3) + 2.
"""
from __future__ import annotations

import math

import numpy as np


def riccati_bessel(x: float, nmax: int):
    """psi_n(x) = x j_n(x) and chi_n(x) = -x y_n(x), n = 0..nmax."""
    psi = np.zeros(nmax + 1)
    chi = np.zeros(nmax + 1)
    psi_m1, psi_0 = math.cos(x), math.sin(x)
    chi_m1, chi_0 = -math.sin(x), math.cos(x)
    psi[0], chi[0] = psi_0, chi_0
    for n in range(1, nmax + 1):
        psi_n = (2 * n - 1) / x * psi_0 - psi_m1
        chi_n = (2 * n - 1) / x * chi_0 - chi_m1
        psi[n], chi[n] = psi_n, chi_n
        psi_m1, psi_0 = psi_0, psi_n
        chi_m1, chi_0 = chi_0, chi_n
    return psi, chi


def coefficients(m: complex, x: float):
    """Mie coefficients a_n, b_n for n = 1..nstop."""
    m = complex(m)
    nstop = int(x + 4.0 * x ** (1.0 / 3.0) + 2.0)
    mx = m * x
    nmx = int(max(nstop, abs(mx))) + 16
    D = np.zeros(nmx + 1, dtype=np.complex128)
    for n in range(nmx, 0, -1):
        D[n - 1] = n / mx - 1.0 / (D[n] + n / mx)
    psi, chi = riccati_bessel(x, nstop)
    xi = psi - 1j * chi
    n = np.arange(1, nstop + 1)
    Dn = D[1:nstop + 1]
    ta = Dn / m + n / x
    tb = m * Dn + n / x
    a = (ta * psi[1:] - psi[:-1]) / (ta * xi[1:] - xi[:-1])
    b = (tb * psi[1:] - psi[:-1]) / (tb * xi[1:] - xi[:-1])
    return a, b


def efficiencies(m: complex, x: float):
    """(Q_ext, Q_abs, Q_sca) of a sphere with size parameter x = k a."""
    a, b = coefficients(m, x)
    n = np.arange(1, a.size + 1)
    qext = 2.0 / x ** 2 * float(np.sum((2 * n + 1) * np.real(a + b)))
    qsca = 2.0 / x ** 2 * float(np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2)))
    return qext, qext - qsca, qsca
