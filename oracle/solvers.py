"""Unpreconditioned Krylov solvers of OpenDDA Sec. 4, plain numpy (oracle).

Test infrastructure only.  Each follows the textbook template the paper
cites (Barrett et al. 1994 for BiCG, BiCGSTAB and QMR; Freund 1992 for the
complex-symmetric BiCG), written for complex vectors:

* Hermitian inner products x^H y where the template has x^T y for real
  data (BiCG, BiCGSTAB), bilinear products x^T y in QMR, whose Lanczos
  process runs with A and A^T.
* A^H v is applied as conj(A conj(v)) and A^T v as A v, both exact because
  the DDA matrix is complex symmetric (Sec. 3).

Starting guess x0 = 0 unless given (Sec. 6).  Stopping rule (the paper does
not define one): the recurrence residual r satisfies ||r||_2 <= tol ||b||_2;
BiCGSTAB also stops half-way when ||s||_2 <= tol ||b||_2.  Every solver
returns (x, info) with info = dict(iterations, matvecs, converged,
breakdown, rel_residual) where rel_residual is the recurrence value.
"""
from __future__ import annotations

import numpy as np


def _norm(v):
    return float(np.sqrt(np.sum(np.abs(v) ** 2)))


def _info(it, mv, conv, brk, rel):
    return dict(iterations=it, matvecs=mv, converged=conv, breakdown=brk, rel_residual=rel)


def bicg(A, b, tol=1e-8, max_iter=1000, x0=None):
    """BiCG (Fletcher 1975) with shadow residual conj(r0); two products per step."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    mv = 1 if x0 is not None else 0
    nb = _norm(b)
    rt = np.conj(r)
    p = pt = None
    rho_old = None
    rel = _norm(r) / nb
    if rel <= tol:
        return x, _info(0, mv, True, False, rel)
    for it in range(1, max_iter + 1):
        rho = np.vdot(rt, r)
        if rho == 0:
            return x, _info(it, mv, False, True, rel)
        if it == 1:
            p = r.copy()
            pt = rt.copy()
        else:
            beta = rho / rho_old
            p = r + beta * p
            pt = rt + np.conj(beta) * pt
        q = A(p)
        qt = np.conj(A(np.conj(pt)))
        mv += 2
        sigma = np.vdot(pt, q)
        if sigma == 0:
            return x, _info(it, mv, False, True, rel)
        alpha = rho / sigma
        x = x + alpha * p
        r = r - alpha * q
        rt = rt - np.conj(alpha) * qt
        rel = _norm(r) / nb
        if rel <= tol:
            return x, _info(it, mv, True, False, rel)
        rho_old = rho
    return x, _info(max_iter, mv, False, False, rel)


def bicg_sym(A, b, tol=1e-8, max_iter=1000, x0=None):
    """BiCG for complex-symmetric A (Freund 1992; COCG): one product per step.

    Algebraically identical to bicg() with shadow conj(r0) when A = A^T.
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    mv = 1 if x0 is not None else 0
    nb = _norm(b)
    p = None
    rho_old = None
    rel = _norm(r) / nb
    if rel <= tol:
        return x, _info(0, mv, True, False, rel)
    for it in range(1, max_iter + 1):
        rho = np.sum(r * r)
        if rho == 0:
            return x, _info(it, mv, False, True, rel)
        p = r.copy() if it == 1 else r + (rho / rho_old) * p
        q = A(p)
        mv += 1
        sigma = np.sum(p * q)
        if sigma == 0:
            return x, _info(it, mv, False, True, rel)
        alpha = rho / sigma
        x = x + alpha * p
        r = r - alpha * q
        rel = _norm(r) / nb
        if rel <= tol:
            return x, _info(it, mv, True, False, rel)
        rho_old = rho
    return x, _info(max_iter, mv, False, False, rel)


def bicgstab(A, b, tol=1e-8, max_iter=1000, x0=None):
    """BiCGSTAB (van der Vorst 1992) with shadow residual r0."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    mv = 1 if x0 is not None else 0
    nb = _norm(b)
    rt = r.copy()
    p = v = None
    rho_old = alpha = omega = None
    rel = _norm(r) / nb
    if rel <= tol:
        return x, _info(0, mv, True, False, rel)
    for it in range(1, max_iter + 1):
        rho = np.vdot(rt, r)
        if rho == 0:
            return x, _info(it, mv, False, True, rel)
        if it == 1:
            p = r.copy()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        v = A(p)
        mv += 1
        sigma = np.vdot(rt, v)
        if sigma == 0:
            return x, _info(it, mv, False, True, rel)
        alpha = rho / sigma
        s = r - alpha * v
        rel_s = _norm(s) / nb
        if rel_s <= tol:
            x = x + alpha * p
            return x, _info(it, mv, True, False, rel_s)
        t = A(s)
        mv += 1
        tt = np.vdot(t, t)
        if tt == 0:
            return x, _info(it, mv, False, True, rel)
        omega = np.vdot(t, s) / tt
        x = x + alpha * p + omega * s
        r = s - omega * t
        rel = _norm(r) / nb
        if rel <= tol:
            return x, _info(it, mv, True, False, rel)
        if omega == 0:
            return x, _info(it, mv, False, True, rel)
        rho_old = rho
    return x, _info(max_iter, mv, False, False, rel)


def qmr(A, b, tol=1e-8, max_iter=1000, x0=None):
    """QMR with coupled two-term recurrences, no look-ahead (Freund &
    Nachtigal 1991; template of Barrett et al. 1994 with M1 = M2 = I).

    The Lanczos pair (v, w) is biorthogonalised with the bilinear form
    w^T v; A p and A^T q are two products per step.
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    mv = 1 if x0 is not None else 0
    nb = _norm(b)
    vt = r.copy()
    rho = _norm(vt)
    wt = r.copy()
    xi = _norm(wt)
    gamma_old = 1.0
    eta = -1.0 + 0j
    theta_old = 0.0
    eps = None
    p = q = d = s = None
    rel = _norm(r) / nb
    if rel <= tol:
        return x, _info(0, mv, True, False, rel)
    for it in range(1, max_iter + 1):
        if rho == 0 or xi == 0:
            return x, _info(it, mv, False, True, rel)
        v = vt / rho
        w = wt / xi
        delta = np.sum(w * v)
        if delta == 0:
            return x, _info(it, mv, False, True, rel)
        if it == 1:
            p = v.copy()
            q = w.copy()
        else:
            p = v - (xi * delta / eps) * p
            q = w - (rho * delta / eps) * q
        pt = A(p)
        mv += 1
        eps = np.sum(q * pt)
        if eps == 0:
            return x, _info(it, mv, False, True, rel)
        beta = eps / delta
        if beta == 0:
            return x, _info(it, mv, False, True, rel)
        vt = pt - beta * v
        rho_new = _norm(vt)
        wt = A(q) - beta * w          # A^T q = A q (complex symmetric)
        mv += 1
        xi_new = _norm(wt)
        theta = rho_new / (gamma_old * abs(beta))
        gamma = 1.0 / np.sqrt(1.0 + theta * theta)
        eta = -eta * rho * gamma * gamma / (beta * gamma_old * gamma_old)
        if it == 1:
            d = eta * p
            s = eta * pt
        else:
            f = (theta_old * gamma) ** 2
            d = eta * p + f * d
            s = eta * pt + f * s
        x = x + d
        r = r - s
        rel = _norm(r) / nb
        if rel <= tol:
            return x, _info(it, mv, True, False, rel)
        rho, xi = rho_new, xi_new
        gamma_old, theta_old = gamma, theta
    return x, _info(max_iter, mv, False, False, rel)


SOLVERS = {"bicg": bicg, "bicgstab": bicgstab, "qmr": qmr, "bicg_sym": bicg_sym}
