"""Krylov solvers of OpenDDA Sec. 4, plain numpy (oracle).

Test infrastructure only.  Each follows the textbook template of the work
the paper cites for it, written for complex vectors:

* BiCG, BiCGSTAB, QMR: Barrett et al. (1994); CGS: Sonneveld (1989);
  TFQMR: Freund (1993); BiCG_sym and QMR_sym: Freund (1992), the
  complex-symmetric forms; CG: Hestenes & Stiefel (1952); RBiCGSTAB as
  BiCGSTAB(ell): Sleijpen & Fokkema (1993).
* Hermitian inner products x^H y where the real template has x^T y (BiCG,
  BiCGSTAB, CGS, TFQMR, all with the shadow vector r0 or conj(r0)),
  bilinear products x^T y where the method relies on A = A^T (BiCG_sym,
  QMR, QMR_sym, CG).
* A^H v is applied as conj(A conj(v)) and A^T v as A v, both exact because
  the DDA matrix is complex symmetric (Sec. 3).

Starting guess x0 = 0 unless given (Sec. 6).  Stopping rule (the paper does
not define one): the recurrence residual r satisfies ||r||_2 <= tol ||b||_2;
BiCGSTAB also stops half-way when ||s||_2 <= tol ||b||_2; TFQMR, which
carries no residual vector, stops when its quasi-residual bound
tau sqrt(m + 1) (an upper bound of ||r_m||_2) is <= tol ||b||_2.  Every
solver returns (x, info) with info = dict(iterations, matvecs, converged,
breakdown, rel_residual) where rel_residual is the recurrence value.

Point-Jacobi preconditioning (used by the paper's benchmark, Sec. 6):
jacobi(solver) solves the symmetrically scaled system
(S A S) y = S b, x = S y with S = diag(alpha)^(1/2) = diag(A)^(-1/2), which
keeps the matrix complex symmetric.
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


def cg(A, b, tol=1e-8, max_iter=1000, x0=None):
    """Conjugate gradients (Hestenes & Stiefel 1952) with the bilinear form
    x^T y in place of the inner product, the form that stays meaningful for
    a complex-symmetric A (van der Vorst & Melissen 1990): one product per
    step.  With that form its recurrence is the one of bicg_sym."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    mv = 1 if x0 is not None else 0
    nb = _norm(b)
    rel = _norm(r) / nb
    if rel <= tol:
        return x, _info(0, mv, True, False, rel)
    p = r.copy()
    rr = np.sum(r * r)
    for it in range(1, max_iter + 1):
        Ap = A(p)
        mv += 1
        pAp = np.sum(p * Ap)
        if pAp == 0 or rr == 0:
            return x, _info(it, mv, False, True, rel)
        a = rr / pAp
        x = x + a * p
        r = r - a * Ap
        rel = _norm(r) / nb
        if rel <= tol:
            return x, _info(it, mv, True, False, rel)
        rr_new = np.sum(r * r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, _info(max_iter, mv, False, False, rel)


def cgs(A, b, tol=1e-8, max_iter=1000, x0=None):
    """Conjugate gradients squared (Sonneveld 1989) with shadow residual r0;
    two products per step."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    mv = 1 if x0 is not None else 0
    nb = _norm(b)
    rt = r.copy()
    rel = _norm(r) / nb
    if rel <= tol:
        return x, _info(0, mv, True, False, rel)
    u = p = q = None
    rho_old = None
    for it in range(1, max_iter + 1):
        rho = np.vdot(rt, r)
        if rho == 0:
            return x, _info(it, mv, False, True, rel)
        if it == 1:
            u = r.copy()
            p = u.copy()
        else:
            beta = rho / rho_old
            u = r + beta * q
            p = u + beta * (q + beta * p)
        vh = A(p)
        mv += 1
        sigma = np.vdot(rt, vh)
        if sigma == 0:
            return x, _info(it, mv, False, True, rel)
        alpha = rho / sigma
        q = u - alpha * vh
        uh = u + q
        x = x + alpha * uh
        r = r - alpha * A(uh)
        mv += 1
        rel = _norm(r) / nb
        if rel <= tol:
            return x, _info(it, mv, True, False, rel)
        rho_old = rho
    return x, _info(max_iter, mv, False, False, rel)


def tfqmr(A, b, tol=1e-8, max_iter=1000, x0=None):
    """Transpose-free QMR (Freund 1993) with shadow vector r0.  One
    iteration is the pair of half-steps m = 2n, 2n + 1 (two products).
    Stops when the quasi-residual bound tau sqrt(m + 1) <= tol ||b||."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    mv = 1 if x0 is not None else 0
    nb = _norm(b)
    rel = _norm(r) / nb
    if rel <= tol:
        return x, _info(0, mv, True, False, rel)
    rt = r.copy()
    w = r.copy()
    u = [r.copy(), None]              # u_m for the even and the odd half-step
    Au = [A(u[0]), None]
    mv += 1
    v = Au[0].copy()
    d = np.zeros_like(b)
    tau = _norm(r)
    theta = 0.0
    eta = 0.0
    rho = np.vdot(rt, r)
    alpha = None
    for it in range(1, max_iter + 1):
        sigma = np.vdot(rt, v)
        if sigma == 0 or rho == 0:
            return x, _info(it, mv, False, True, rel)
        alpha = rho / sigma
        u[1] = u[0] - alpha * v
        Au[1] = A(u[1])
        mv += 1
        for j in (0, 1):
            m = 2 * (it - 1) + j
            w = w - alpha * Au[j]
            d = u[j] + (theta * theta * eta / alpha) * d
            theta = _norm(w) / tau
            c = 1.0 / np.sqrt(1.0 + theta * theta)
            tau = tau * theta * c
            eta = c * c * alpha
            x = x + eta * d
            rel = tau * np.sqrt(m + 1) / nb
            if rel <= tol:
                return x, _info(it, mv, True, False, rel)
        rho_new = np.vdot(rt, w)
        if rho_new == 0:
            return x, _info(it, mv, False, True, rel)
        beta = rho_new / rho
        rho = rho_new
        u[0] = w + beta * u[1]
        Au[0] = A(u[0])
        mv += 1
        v = Au[0] + beta * (Au[1] + beta * v)
    return x, _info(max_iter, mv, False, False, rel)


def qmr_sym(A, b, tol=1e-8, max_iter=1000, x0=None):
    """QMR for complex-symmetric A (Freund 1992): the QMR recurrences of
    qmr() driven by the complex-symmetric Lanczos process, whose left and
    right Lanczos vectors coincide (w_n = v_n when w_1 = v_1 and A = A^T),
    so one product per step."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    mv = 1 if x0 is not None else 0
    nb = _norm(b)
    vt = r.copy()
    rho = _norm(vt)
    gamma_old = 1.0
    eta = -1.0 + 0j
    theta_old = 0.0
    eps = None
    p = d = s = None
    rel = _norm(r) / nb
    if rel <= tol:
        return x, _info(0, mv, True, False, rel)
    for it in range(1, max_iter + 1):
        if rho == 0:
            return x, _info(it, mv, False, True, rel)
        v = vt / rho
        delta = np.sum(v * v)
        if delta == 0:
            return x, _info(it, mv, False, True, rel)
        p = v.copy() if it == 1 else v - (rho * delta / eps) * p
        pt = A(p)
        mv += 1
        eps = np.sum(p * pt)
        if eps == 0:
            return x, _info(it, mv, False, True, rel)
        beta = eps / delta
        if beta == 0:
            return x, _info(it, mv, False, True, rel)
        vt = pt - beta * v
        rho_new = _norm(vt)
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
        rho = rho_new
        gamma_old, theta_old = gamma, theta
    return x, _info(max_iter, mv, False, False, rel)


def bicgstab_l(A, b, tol=1e-8, max_iter=1000, x0=None, ell=2):
    """BiCGSTAB(ell) (Sleijpen & Fokkema 1993), the paper's restarted,
    stabilised BiCG "RBiCGSTAB" with ell = its number of starting vectors:
    each iteration ("cycle") runs ell BiCG steps that build r_j = A^j r and
    u_j = A^j u, then replaces the residual by the minimal-residual
    combination r_0 - sum_j gamma_j r_j (modified Gram-Schmidt on r_1..r_ell)
    and updates x, u alike.  Shadow vector r0, Hermitian products; 2 ell
    products per iteration.  Stopping test at the end of each cycle."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    mv = 1 if x0 is not None else 0
    nb = _norm(b)
    rel = _norm(r) / nb
    if rel <= tol:
        return x, _info(0, mv, True, False, rel)
    rt = r.copy()
    u = np.zeros_like(b)
    rho0, alpha, omega = 1.0 + 0j, 0.0 + 0j, 1.0 + 0j
    for it in range(1, max_iter + 1):
        rh = [r] + [None] * ell
        uh = [u] + [None] * ell
        rho0 = -omega * rho0
        for j in range(ell):                         # BiCG part
            rho1 = np.vdot(rt, rh[j])
            if rho0 == 0:
                return x, _info(it, mv, False, True, rel)
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                uh[i] = rh[i] - beta * uh[i]
            uh[j + 1] = A(uh[j])
            mv += 1
            gam = np.vdot(rt, uh[j + 1])
            if gam == 0:
                return x, _info(it, mv, False, True, rel)
            alpha = rho0 / gam
            for i in range(j + 1):
                rh[i] = rh[i] - alpha * uh[i + 1]
            rh[j + 1] = A(rh[j])
            mv += 1
            x = x + alpha * uh[0]
        # minimal-residual part (modified Gram-Schmidt)
        tau = np.zeros((ell + 1, ell + 1), dtype=complex)
        sigma = np.zeros(ell + 1)
        gp = np.zeros(ell + 1, dtype=complex)
        for j in range(1, ell + 1):
            for i in range(1, j):
                tau[i, j] = np.vdot(rh[i], rh[j]) / sigma[i]
                rh[j] = rh[j] - tau[i, j] * rh[i]
            sigma[j] = np.real(np.vdot(rh[j], rh[j]))
            if sigma[j] == 0:
                return x, _info(it, mv, False, True, rel)
            gp[j] = np.vdot(rh[j], rh[0]) / sigma[j]
        g = np.zeros(ell + 1, dtype=complex)
        g[ell] = gp[ell]
        omega = g[ell]
        for j in range(ell - 1, 0, -1):
            g[j] = gp[j] - sum(tau[j, i] * g[i] for i in range(j + 1, ell + 1))
        gpp = np.zeros(ell + 1, dtype=complex)
        for j in range(1, ell):
            gpp[j] = g[j + 1] + sum(tau[j, i] * g[i + 1] for i in range(j + 1, ell))
        x = x + g[1] * rh[0]
        rh[0] = rh[0] - gp[ell] * rh[ell]
        uh[0] = uh[0] - g[ell] * uh[ell]
        for j in range(1, ell):
            uh[0] = uh[0] - g[j] * uh[j]
            x = x + gpp[j] * rh[j]
            rh[0] = rh[0] - gp[j] * rh[j]
        r, u = rh[0], uh[0]
        rel = _norm(r) / nb
        if rel <= tol:
            return x, _info(it, mv, True, False, rel)
        if omega == 0:
            return x, _info(it, mv, False, True, rel)
    return x, _info(max_iter, mv, False, False, rel)


def jacobi(solver, diag):
    """Point-Jacobi (diagonal) preconditioning of `solver`, applied as the
    symmetric scaling S A S y = S b, x = S y, S = diag^(-1/2) (principal
    square root), which keeps a complex-symmetric A complex symmetric."""
    sc = 1.0 / np.sqrt(np.asarray(diag, dtype=np.complex128).reshape(-1))

    def run(A, b, tol=1e-8, max_iter=1000, x0=None):
        y0 = None if x0 is None else x0 / sc
        y, info = solver(lambda v: sc * A(sc * v), sc * b, tol=tol, max_iter=max_iter, x0=y0)
        return sc * y, info
    return run


SOLVERS = {"bicg": bicg, "bicgstab": bicgstab, "qmr": qmr, "bicg_sym": bicg_sym, "cg": cg, "cgs": cgs,
           "tfqmr": tfqmr, "qmr_sym": qmr_sym,
           "rbicgstab1": lambda *a, **k: bicgstab_l(*a, ell=1, **k),
           "rbicgstab2": lambda *a, **k: bicgstab_l(*a, ell=2, **k),
           "rbicgstab3": lambda *a, **k: bicgstab_l(*a, ell=3, **k)}
