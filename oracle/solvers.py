"""Krylov solvers of OpenDDA Sec. 4, plain numpy (oracle).

Test infrastructure only.  Each follows the textbook template of the work
the paper cites for it, written for complex vectors:

* BiCG, BiCGSTAB, QMR: Barrett et al. (1994); CGS: Sonneveld (1989);
  TFQMR: Freund (1993); BiCG_sym and QMR_sym: Freund (1992), the
  complex-symmetric forms; CG: Hestenes & Stiefel (1952); RBiCGSTAB as
  BiCGSTAB(ell): Sleijpen & Fokkema (1993).
* ML(n)BiCGSTAB (Yeung & Chan 1999): written from its definition, the
  residual at the end of each cycle (see ``mlbicgstab``), not from a
  recurrence; its n - 1 random shadow vectors come from the counter-based
  SplitMix64 generator (``splitmix64``, ``shadow_vectors``).
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


# ------------------------------------------------------------ ML(n)BiCGSTAB
_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def _mix64(z: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood 2014)."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def splitmix64(seed: int, count: int) -> list:
    """The first `count` outputs of SplitMix64 started from state `seed`:
    the state advances by the golden-ratio constant 0x9E3779B97F4A7C15 and
    each output is the mix of the new state."""
    out, st = [], seed & _M64
    for _ in range(count):
        st = (st + _GOLDEN) & _M64
        out.append(_mix64(st))
    return out


def shadow_vectors(r0: np.ndarray, nvec: int) -> np.ndarray:
    """The nvec left starting vectors of ML(n)BiCGSTAB as columns of an
    (N, nvec) array: q_1 = r0 (so that ML(1)BiCGSTAB is BiCGSTAB with the
    shadow residual r0), and for i = 1 .. nvec - 1 the vector q_(i+1) whose
    entry e (flat index into the [3][N_d] vector) is u1 + i u2, where u1 and
    u2 are the first two SplitMix64 outputs started from the state
    i * 2^40 + e, each mapped to [-1, 1) as (u >> 11) * 2^-52 - 1."""
    N = r0.size
    Q = np.zeros((N, nvec), dtype=np.complex128)
    Q[:, 0] = r0.reshape(-1)
    for i in range(1, nvec):
        for e in range(N):
            u1, u2 = splitmix64((i << 40) + e, 2)
            Q[e, i] = complex((u1 >> 11) * 2.0 ** -52 - 1.0, (u2 >> 11) * 2.0 ** -52 - 1.0)
    return Q


def _orth(v, basis):
    """v orthogonalised against the orthonormal columns in `basis` (twice)."""
    for _ in range(2):
        for q in basis:
            v = v - np.vdot(q, v) * q
    return v


def mlbicgstab(A, b, tol=1e-8, max_iter=1000, x0=None, nvec=2):
    """ML(n)BiCGSTAB (Yeung & Chan 1999), n = nvec left starting vectors
    Q = shadow_vectors(r0, n), evaluated from its definition at the end of
    every cycle (one iteration = one cycle of n + 1 products, the unit of
    the paper's Table 3):

    * phi_j, the ML(n)BiCG residual polynomial of degree j n (phi_j(0) = 1),
      is fixed by phi_j(A) r0 orthogonal to the block Krylov space
      K_j(A^H, Q) = span{(A^H)^l q_i : l < j, i <= n}: with V an orthonormal
      basis of K_(jn)(A, r0), phi_j(A) r0 = r0 - A V y where
      (W^H A V) y = W^H r0 for an orthonormal basis W of K_j(A^H, Q);
    * v_j = Omega_(j-1)(A) phi_j(A) r0, Omega_j(t) = prod_(l<=j)(1 - omega_l t);
    * omega_j minimises ||(I - omega A) v_j||: omega_j = (t^H v_j)/(t^H t),
      t = A v_j, and the cycle's residual is r_j = v_j - omega_j t;
    * x_j = x0 + S_j r0 + Omega_j(A) V y, with 1 - Omega_j(t) = t S_j(t)
      (S_j r0 = (I - omega_j A) S_(j-1) r0 + omega_j r0), so b - A x_j = r_j.

    Plain and slow (dense bases, every Omega applied factor by factor): for
    small test systems only.  Stops when ||r_j|| <= tol ||b||; matvecs
    reports the method's count j (n + 1).  info also carries `history`, the
    relative residual after each cycle."""
    x0v = np.zeros_like(b) if x0 is None else x0.copy()
    r0 = b - A(x0v) if x0 is not None else b.copy()
    nb = _norm(b)
    rel = _norm(r0) / nb
    hist = []
    if rel <= tol:
        info = _info(0, 0, True, False, rel)
        info["history"] = hist
        return x0v, info

    def AH(v):
        return np.conj(A(np.conj(v)))

    Q = shadow_vectors(r0, nvec)
    V, AV = [], []                    # orthonormal basis of K(A, r0) and A applied to it
    W, last = [], None                # orthonormal basis of K_j(A^H, Q), last block
    omegas = []
    s = np.zeros_like(r0)             # S_j r0
    x = x0v
    for j in range(1, max_iter + 1):
        # right space: K_(jn)(A, r0) by Arnoldi
        while len(V) < j * nvec:
            w = r0.copy() if not V else AV[-1].copy()
            w = _orth(w, V)
            nw = _norm(w)
            if nw == 0:
                break
            V.append(w / nw)
            AV.append(A(V[-1]))
        # left space: one more block (A^H)^(j-1) Q, orthonormalised
        block = [Q[:, i].reshape(r0.shape) for i in range(nvec)] if last is None else [AH(q) for q in last]
        last = []
        for w in block:
            w = _orth(w, W)
            nw = _norm(w)
            if nw == 0:
                continue
            W.append(w / nw)
            last.append(W[-1])
        Vm = np.stack([v.reshape(-1) for v in V], axis=1)
        AVm = np.stack([v.reshape(-1) for v in AV], axis=1)
        Wm = np.stack([v.reshape(-1) for v in W], axis=1)
        G = Wm.conj().T @ AVm
        if G.shape[0] != G.shape[1]:
            info = _info(j, j * (nvec + 1), False, True, rel)
            info["history"] = hist
            return x, info
        y = np.linalg.solve(G, Wm.conj().T @ r0.reshape(-1))
        u = r0 - (AVm @ y).reshape(r0.shape)
        v = u
        for om in omegas:
            v = v - om * A(v)
        t = A(v)
        tt = np.vdot(t, t)
        if tt == 0:
            info = _info(j, j * (nvec + 1), _norm(v) == 0, _norm(v) != 0, _norm(v) / nb)
            info["history"] = hist
            return x, info
        om = np.vdot(t, v) / tt
        omegas.append(om)
        r = v - om * t
        s = s - om * A(s) + om * r0
        z = (Vm @ y).reshape(r0.shape)
        for w_ in omegas:
            z = z - w_ * A(z)
        x = x0v + s + z
        rel = _norm(r) / nb
        hist.append(rel)
        if rel <= tol:
            info = _info(j, j * (nvec + 1), True, False, rel)
            info["history"] = hist
            return x, info
        if om == 0:
            info = _info(j, j * (nvec + 1), False, True, rel)
            info["history"] = hist
            return x, info
    info = _info(max_iter, max_iter * (nvec + 1), False, False, rel)
    info["history"] = hist
    return x, info


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
           "rbicgstab3": lambda *a, **k: bicgstab_l(*a, ell=3, **k),
           "mlbicgstab1": lambda *a, **k: mlbicgstab(*a, nvec=1, **k),
           "mlbicgstab2": lambda *a, **k: mlbicgstab(*a, nvec=2, **k),
           "mlbicgstab3": lambda *a, **k: mlbicgstab(*a, nvec=3, **k)}
