"""Per-dipole permittivity gradients of C_ext and C_abs, plain dense FP64
(oracle; test infrastructure only).

A dipole's polarisability depends on its permittivity eps (= m^2) through
the prescription of Sec. 1 (CM, radiative reaction, LDR), so the diagonal
of A in Eq. 1 is A_jj = a(eps_j).  With P the solution of A P = E and a real
cross section C(P), a change d eps_j moves P by dP = -A^-1 dA P with
dA = diag(a'(eps_j) d eps_j).  Written with one adjoint vector:

  C_abs = 4 pi k sum_j w_j |P_j|^2,  w_j = -Im a(eps_j) - (2/3) k^3:
      A mu = W conj(P)   (A is complex symmetric, so conj(mu) solves A^H l = W P)
      dC = 4 pi k sum_j [ |P_j|^2 (-Im(a'_j d eps_j)) - 2 Re(mu_j . a'_j d eps_j P_j) ]
  C_ext = 4 pi k sum_j Im(E_j^* . P_j):
      A mu = conj(E)
      dC = -4 pi k sum_j Im(mu_j . a'_j d eps_j P_j)

The gradient g_j = dC/dRe(eps_j) + i dC/dIm(eps_j) follows by taking
d eps_j = 1 and d eps_j = i.  The three axes of a dipole share eps_j.
"""
from __future__ import annotations

import math

import numpy as np

from . import dda

B1, B2, B3 = dda.LDR_B1, dda.LDR_B2, dda.LDR_B3


def alpha_inverse(eps: complex, k: float, rule: str, khat=(0, 0, 1), e0=(1, 0, 0)) -> complex:
    """1/alpha as a function of eps (the prescriptions of dda.alpha_*, in eps)."""
    m = np.sqrt(complex(eps))
    if rule == "cm":
        return 1.0 / dda.alpha_cm(m)
    if rule == "cmrr":
        return 1.0 / dda.alpha_rr(m, k)
    return 1.0 / dda.alpha_ldr(m, k, khat, e0)


def alpha_inverse_derivative(eps: complex, k: float, rule: str, khat=(0, 0, 1), e0=(1, 0, 0)) -> complex:
    """d(1/alpha)/d eps in closed form.

    1/alpha_CM = (4 pi / 3)(eps + 2)/(eps - 1), whose derivative is
    -4 pi/(eps - 1)^2; the radiative-reaction term does not depend on eps;
    LDR adds (b1 + eps b2 + eps b3 S) k^2, whose derivative is (b2 + b3 S) k^2.
    """
    d = -4.0 * math.pi / (complex(eps) - 1.0) ** 2
    if rule == "ldr":
        S = float(np.sum((np.asarray(khat, dtype=float) * np.asarray(e0, dtype=complex)) ** 2).real)
        d += (B2 + B3 * S) * k * k
    return d


def _gradient(coords, ainv, dainv, k, E, which):
    n = coords.shape[0]
    A = dda.dense_matrix(coords, ainv, k)
    P = np.linalg.solve(A, E.reshape(-1)).reshape(3, n)
    if which == "abs":
        w = -np.imag(ainv.T) - (2.0 / 3.0) * k ** 3          # (3, n)
        mu = np.linalg.solve(A, (w * np.conj(P)).reshape(-1)).reshape(3, n)
        S = np.sum(mu * dainv.T * P, axis=0)                 # sum_c mu_jc a'_jc P_jc
        absP = np.abs(P) ** 2
        dx = np.sum(-absP * np.imag(dainv.T), axis=0) - 2.0 * np.real(S)
        dy = np.sum(-absP * np.real(dainv.T), axis=0) + 2.0 * np.imag(S)
    else:
        mu = np.linalg.solve(A, np.conj(E).reshape(-1)).reshape(3, n)
        S = np.sum(mu * dainv.T * P, axis=0)
        dx = -np.imag(S)
        dy = -np.real(S)
    return 4.0 * math.pi * k * (dx + 1j * dy), P


def abs_gradient_dense(coords, ainv, dainv, k, E):
    """g_j for C_abs by the dense adjoint.  ainv, dainv: (N_d, 3)."""
    return _gradient(coords, ainv, dainv, k, E, "abs")


def ext_gradient_dense(coords, ainv, dainv, k, E):
    """g_j for C_ext by the dense adjoint."""
    return _gradient(coords, ainv, dainv, k, E, "ext")


def cross_sections_for_eps(coords, eps, k, E, rule, khat=(0, 0, 1), e0=(1, 0, 0)):
    """(C_ext, C_abs) with per-dipole permittivities eps (N_d,), by dense LU."""
    ainv = np.array([[alpha_inverse(e, k, rule, khat, e0)] * 3 for e in eps])
    A = dda.dense_matrix(coords, ainv, k)
    P = np.linalg.solve(A, E.reshape(-1)).reshape(3, -1)
    return dda.c_ext(E, P, k), dda.c_abs(ainv, P, k)
