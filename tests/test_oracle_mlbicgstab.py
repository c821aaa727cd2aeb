"""Pins of the oracle's ML(n)BiCGSTAB (Yeung & Chan 1999; OpenDDA Sec. 4
and Table 3), which is written from the method's definition: the residual
at the end of each cycle of n + 1 products.  Checked against what fixes it
from outside:

* n = 1 is BiCGSTAB (van der Vorst 1992) iterate for iterate, against the
  oracle's independent BiCGSTAB (itself pinned against LU);
* every n converges to the dense LU solution;
* with as many shadow vectors as unknowns the first cycle is exact (the
  Petrov-Galerkin conditions then span the whole space);
* every cycle end equals that of an independent recurrence, the induced
  dimension reduction form of Sonneveld & van Gijzen (2008) with the same
  shadow vectors, whose residual after the first step of each cycle is, by
  the IDR theorem, the same unique vector of G_j = (I - omega_j A)(G_(j-1)
  intersected with the null space of Q^H) of that degree;
* the counter-based generator of the shadow vectors reproduces the
  published SplitMix64 outputs.
CPU only.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import dda, solvers

HERE = os.path.dirname(os.path.abspath(__file__))


def _system(nside=5, k=0.45, m=1.33 + 0.05j):
    mask = synth.sphere(nside)
    c = dda.coords_of(mask)
    ainv = np.full((c.shape[0], 3), 1.0 / dda.alpha_rr(m, k))
    A = dda.dense_matrix(c, ainv, k)
    E = dda.incident_field(c, k, [0, 0, 1], [1, 0, 0]).reshape(-1)
    return A, E


def test_splitmix64_published_outputs():
    with open(os.path.join(HERE, "golden", "splitmix64.json")) as f:
        g = json.load(f)
    assert [hex(v) for v in solvers.splitmix64(0, 3)] == [hex(int(h, 16)) for h in g["seed_0_hex"]]
    assert solvers.splitmix64(1234567, 5) == g["seed_1234567"]


def test_shadow_vectors_layout():
    r0 = np.arange(7) + 1j
    Q = solvers.shadow_vectors(r0, 3)
    assert np.array_equal(Q[:, 0], r0)
    u1, u2 = solvers.splitmix64((2 << 40) + 5, 2)
    assert Q[5, 2] == complex((u1 >> 11) * 2.0 ** -52 - 1.0, (u2 >> 11) * 2.0 ** -52 - 1.0)
    assert np.all(np.abs(Q[:, 1:].real) <= 1) and np.all(np.abs(Q[:, 1:].imag) <= 1)


def test_ml1_is_bicgstab_iterate_for_iterate():
    A, b = _system()
    op = lambda v: A @ v
    for it in (1, 2, 4, 7):
        x1, i1 = solvers.mlbicgstab(op, b, tol=0, max_iter=it, nvec=1)
        x2, i2 = solvers.bicgstab(op, b, tol=0, max_iter=it)
        assert np.abs(x1 - x2).max() <= 1e-10 * np.abs(x2).max(), it
        assert i1["matvecs"] == i2["matvecs"] == 2 * it


@pytest.mark.parametrize("nvec", [1, 2, 3])
def test_ml_converges_to_lu(nvec):
    A, b = _system()
    P = np.linalg.solve(A, b)
    x, info = solvers.mlbicgstab(lambda v: A @ v, b, tol=1e-12, max_iter=200, nvec=nvec)
    assert info["converged"]
    assert np.abs(x - P).max() <= 1e-10 * np.abs(P).max()
    assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)
    assert info["matvecs"] == info["iterations"] * (nvec + 1)


def test_full_shadow_space_is_exact_in_one_cycle():
    rng = synth.rng(3)
    n = 6
    M = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = M + M.T + 4 * np.eye(n)          # complex symmetric, well conditioned
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    x, info = solvers.mlbicgstab(lambda v: A @ v, b, tol=1e-11, max_iter=1, nvec=n)
    assert info["converged"] and info["iterations"] == 1 and info["matvecs"] == n + 1
    assert np.abs(x - np.linalg.solve(A, b)).max() <= 1e-10 * np.abs(x).max()


def _idr_cycle_ends(A, b, Q, cycles):
    """IDR(s) (Sonneveld & van Gijzen 2008, the prototype with s
    minimal-residual start-up steps) with shadow space Q (N x s); returns
    the iterate after the first step of each of `cycles` cycles."""
    N, s = Q.shape
    x = np.zeros_like(b)
    r = b.copy()
    dR = np.zeros((N, s), dtype=complex)
    dX = np.zeros((N, s), dtype=complex)
    for k in range(s):
        v = A @ r
        om = np.vdot(v, r) / np.vdot(v, v)
        dX[:, k] = om * r
        dR[:, k] = -om * v
        x = x + dX[:, k]
        r = r + dR[:, k]
    M = Q.conj().T @ dR
    f = Q.conj().T @ r
    oldest = 0
    om = None
    out = []
    for _ in range(cycles):
        for k in range(s + 1):
            c = np.linalg.solve(M, f)
            q = -dR @ c
            v = r + q
            if k == 0:
                t = A @ v
                om = np.vdot(t, v) / np.vdot(t, t)
                dR[:, oldest] = q - om * t
                dX[:, oldest] = -dX @ c + om * v
            else:
                dX[:, oldest] = -dX @ c + om * v
                dR[:, oldest] = -(A @ dX[:, oldest])
            r = r + dR[:, oldest]
            x = x + dX[:, oldest]
            dm = Q.conj().T @ dR[:, oldest]
            M[:, oldest] = dm
            f = f + dm
            oldest = (oldest + 1) % s
            if k == 0:
                out.append(x.copy())
    return out


@pytest.mark.parametrize("nvec", [2, 3])
def test_cycle_ends_match_idr_recurrence(nvec):
    A, b = _system(nside=4)
    Q = solvers.shadow_vectors(b, nvec)
    ends = _idr_cycle_ends(A, b, Q, 6)
    for j, xr in enumerate(ends, start=1):
        x, info = solvers.mlbicgstab(lambda v: A @ v, b, tol=0, max_iter=j, nvec=nvec)
        assert np.abs(x - xr).max() <= 1e-9 * np.abs(xr).max(), j
        assert info["matvecs"] == j * (nvec + 1)
