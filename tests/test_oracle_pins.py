"""Pins of the FP64 oracle against what the paper and the mathematics fix.

CPU only.  Each test names the passage, closed form or invariant it uses.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
import synth
from oracle import circulant, dda, mie, solvers


# ------------------------------------------------------------------ geometry

def _sphere_count_rule(n):
    """Count of sites with (2i+1-n)^2 + (2j+1-n)^2 + (2k+1-n)^2 <= n^2 per plane."""
    u = 2 * np.arange(n, dtype=np.int64) + 1 - n
    u2 = np.sort(u * u)
    rem = n * n - (u[:, None] ** 2 + u[None, :] ** 2)
    return int(np.searchsorted(u2, rem.reshape(-1), side="right").sum())


@pytest.mark.parametrize("n", [18, 200])
def test_sphere_counts_generator(golden, n):
    # Sec. 4 (18^3 -> 3112) and Sec. 6 / Table 4 caption (200^3 -> 4,188,896)
    m = synth.sphere(n)
    assert int(m.sum()) == golden["sphere_occupied_sites"][str(n)]
    assert dda.occupied_sites(m).size == golden["sphere_occupied_sites"][str(n)]


@pytest.mark.parametrize("n", [240, 310, 380, 480, 600])
def test_sphere_counts_rule(golden, n):
    # Table 5 system sizes; the same site-centre rule as synth.sphere
    assert _sphere_count_rule(n) == golden["sphere_occupied_sites"][str(n)]


def test_cube_count(golden):
    assert int(synth.cube(100).sum()) == golden["cube_occupied_sites"]["100"]


# --------------------------------------------------------------- bit fields

def test_occupancy_bit_positions():
    # Sec. 2 layout reading: site s -> word s // 32, bit s % 32, LSB first
    mask = np.zeros((2, 3, 7), dtype=np.uint8)       # P=2, J=3, K=7 -> 42 sites
    flat = mask.reshape(-1)
    for s in (0, 5, 31, 32, 33, 41):
        flat[s] = 1
    w = dda.pack_occupancy(mask)
    assert w.dtype == np.uint32 and w.size == 2
    assert int(w[0]) == (1 << 0) | (1 << 5) | (1 << 31)
    assert int(w[1]) == (1 << 0) | (1 << 1) | (1 << 9)
    assert np.array_equal(dda.unpack_occupancy(w, 42), flat)


def test_composition_fields(golden):
    # Sec. 2: four materials 0..3 need two bits, mask 3
    assert dda.composition_bits(4) == 2
    assert (1 << dda.composition_bits(4)) - 1 == golden["bitfield_memory"]["composition_mask_4_materials"]
    assert dda.composition_bits(1) == 1 and dda.composition_bits(2) == 1
    assert dda.composition_bits(3) == 2 and dda.composition_bits(5) == 3
    g = synth.rng(3)
    mats = g.integers(0, 5, size=(3, 4, 5, 3))
    w = dda.pack_composition(mats, 5)
    # 3-bit fields, 10 per word, field q = 3 s + axis
    assert w.size == (3 * 60 + 9) // 10
    q = 3 * 7 + 2
    assert (int(w[q // 10]) >> ((q % 10) * 3)) & 7 == mats.reshape(-1, 3)[7, 2]
    assert np.array_equal(dda.unpack_composition(w, 60, 5), mats.reshape(-1, 3))


def test_bitfield_memory_claims(golden):
    bm = golden["bitfield_memory"]
    # one occupancy bit replaces x, y, z, flag as 32-bit integers
    assert 4 * 32 // 1 == bm["occupancy_factor"]
    # three 32-bit composition integers -> three 2-bit fields
    assert (3 * 32) // (3 * dda.composition_bits(bm["n_materials"])) == bm["composition_factor_4_materials"]
    n = bm["lattice_edge"] ** 3
    ints = 7 * 4 * n / 2 ** 30
    assert round(ints, 2) == bm["integers_GB"]
    bits = dda.bitfield_bytes(n, bm["n_materials"]) / 2 ** 30
    assert bm["bitfield_GB_just_over"] < bits < 1.1 * bm["bitfield_GB_just_over"]


def test_ranks_and_coords():
    m = synth.sphere(9)
    r = dda.ranks(m)
    occ = dda.occupied_sites(m)
    assert np.array_equal(r[occ], np.arange(occ.size))
    c = dda.coords_of(m)
    P, J, K = m.shape
    assert np.array_equal((c[:, 2] * J + c[:, 1]) * K + c[:, 0], occ)


# ------------------------------------------------------- interaction tensor

def _full3(t6):
    idx = ((0, 1, 2), (1, 3, 4), (2, 4, 5))
    return np.array([[t6[idx[a][b]] for b in range(3)] for a in range(3)])


def test_static_limit_is_dipole_field():
    # k -> 0: -A r^3 = 3 r^ r^ - I, the electrostatic field of a point dipole
    r = np.array([2.0, -1.0, 3.0])
    A = _full3(dda.interaction_tensor(0.0, r))
    rh = r / np.linalg.norm(r)
    expect = -(3.0 * np.outer(rh, rh) - np.eye(3)) / np.linalg.norm(r) ** 3
    assert np.allclose(A, expect, rtol=0, atol=1e-15)


def test_far_field_is_transverse():
    # k r >> 1: -A -> k^2 e^{ikr}/r (I - r^ r^), the radiation field
    k = 3.0
    r = np.array([400.0, 300.0, 1200.0])
    rn = np.linalg.norm(r)
    A = _full3(dda.interaction_tensor(k, r))
    rh = r / rn
    expect = -k * k * np.exp(1j * k * rn) / rn * (np.eye(3) - np.outer(rh, rh))
    assert np.abs(A - expect).max() < 2e-3 * np.abs(expect).max()


def test_im_limit_at_origin():
    # Im(-A(r)) -> (2/3) k^3 I as r -> 0 (radiative reaction term)
    k = 0.7
    A = _full3(dda.interaction_tensor(k, np.array([1e-3, 2e-3, -1.5e-3])))
    assert np.allclose(-A.imag, (2.0 / 3.0) * k ** 3 * np.eye(3), atol=1e-6)


def test_table1_signs_from_parity(golden):
    # Table 1: a mirrored axis flips the sign of r_a r_b when exactly one of a, b is that axis
    t = golden["table1_mirror_signs"]
    sg = circulant.mirror_signs()
    assert np.array_equal(sg, np.array([t["x"], t["y"], t["z"]]))
    for axis in range(3):
        for m, (a, b) in enumerate(circulant.AXES):
            assert sg[axis, m] == (-1) ** ((a == axis) + (b == axis))
    # and the tensor itself obeys it
    r = np.array([2.0, 3.0, 1.0])
    t0 = dda.interaction_tensor(0.9, r)
    for axis in range(3):
        rm = r.copy()
        rm[axis] = -rm[axis]
        assert np.allclose(dda.interaction_tensor(0.9, rm), sg[axis] * t0, rtol=1e-14, atol=0)


# ----------------------------------------------------------------- matrix

def _setup(mask, k, m=1.33 + 0.01j, materials=None, refr=None):
    c = dda.coords_of(mask)
    n = c.shape[0]
    if materials is None:
        ainv = np.full((n, 3), 1.0 / dda.alpha_rr(m, k))
    else:
        tab = np.array([[dda.alpha_rr(q, k)] * 3 for q in refr])
        ainv = dda.alpha_inverse_per_dipole(tab, materials.reshape(-1, 3), n, mask)
    return c, ainv


def test_matrix_symmetric():
    # Sec. 3: A is complex symmetric
    m = synth.sphere(7)
    c, ainv = _setup(m, 0.6)
    A = dda.dense_matrix(c, ainv, 0.6)
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max()


def test_direct_equals_dense():
    m = synth.sphere(6, box=(6, 5, 7))
    c, ainv = _setup(m, 0.4)
    p = synth.complex_normal(5, (3, c.shape[0]))
    A = dda.dense_matrix(c, ainv, 0.4)
    y = dda.direct_matvec(c, ainv, 0.4, p)
    assert np.abs(A @ p.reshape(-1) - y.reshape(-1)).max() < 1e-13 * np.abs(y).max()


@pytest.mark.parametrize("shape,hollow", [((1, 1, 1), False), ((2, 3, 5), False), ((5, 4, 3), True),
                                          ((8, 8, 8), False), ((7, 3, 6), True), ((12, 5, 4), False),
                                          ((12, 24, 9), True), ((13, 12, 24), False), ((20, 7, 17), True)])
def test_fft_matvec_equals_direct_sum(shape, hollow):
    # App. A standard algorithm (circulant embedding + Eqs. 6-8) == definition
    K, J, P = shape
    g = synth.rng(K * 100 + J * 10 + P)
    mask = (g.random((P, J, K)) < (0.55 if hollow else 1.1)).astype(np.uint8)
    mask.reshape(-1)[0] = 1
    k = 0.45
    mats = np.repeat((g.random((P, J, K)) < 0.3).astype(np.uint8)[..., None], 3, axis=3)
    c, ainv = _setup(mask, k, materials=mats, refr=[1.5 + 0.01j, 1.7 + 0.1j])
    p = synth.complex_normal(7, (3, c.shape[0]))
    L = tuple(circulant.padded_length(v) for v in shape)
    col = circulant.first_column(k, K, J, P, L)
    y_fft = circulant.fft_matvec(col, mask, ainv, p)
    y_dir = dda.direct_matvec(c, ainv, k, p)
    assert np.abs(y_fft - y_dir).max() <= 1e-13 * np.abs(y_dir).max()


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 5, 2), (6, 1, 3), (9, 4, 5)])
def test_half_spectrum_and_mirror_lookup(shape):
    # Sec. 3: fused T-to-c + 1D DFTs keeping L/2+1 outputs equals the 3D DFT of
    # the circulant's first column; the signed mirror lookup recovers the rest
    K, J, P = shape
    k = 0.8
    L = tuple(circulant.padded_length(v) for v in shape)
    col = circulant.first_column(k, K, J, P, L)
    full = np.fft.fftn(col, axes=(1, 2, 3))
    half = circulant.half_spectrum(circulant.tensor_section1(k, K, J, P), L)
    H = (L[2] // 2 + 1, L[1] // 2 + 1, L[0] // 2 + 1)
    assert half.shape == (6,) + H
    scale = np.abs(full).max()
    assert np.abs(half - full[:, :H[0], :H[1], :H[2]]).max() <= 1e-13 * scale
    assert np.abs(circulant.expand_half_spectrum(half, L) - full).max() <= 1e-13 * scale


def test_padded_lengths():
    # K'' = 2K - 1 + kf: the smallest 2^a, 3 * 2^a or 5 * 2^a (a >= 3) >= 2K - 1
    ns = (1, 2, 5, 12, 13, 16, 20, 24, 48, 74, 96, 100, 128, 138, 160, 193, 256, 300, 512)
    assert [circulant.padded_length(n) for n in ns] == [2, 4, 16, 24, 32, 32, 40, 48, 96, 160, 192, 256, 256,
                                                        320, 320, 512, 512, 640, 1024]


# ---------------------------------------------------------- polarisability

def test_single_dipole_closed_form():
    # one dipole: P = alpha E; C_ext = 4 pi k Im alpha; C_sca = (8 pi/3) k^4 |alpha|^2
    k, m = 0.5, 1.7 + 0.3j
    mask = np.ones((1, 1, 1), dtype=np.uint8)
    c, ainv = _setup(mask, k, m=m)
    E = dda.incident_field(c, k, [0, 0, 1], [1, 0, 0])
    A = dda.dense_matrix(c, ainv, k)
    P = np.linalg.solve(A, E.reshape(-1)).reshape(3, 1)
    alpha = dda.alpha_rr(m, k)
    assert np.allclose(P[:, 0], alpha * np.array([1, 0, 0]))
    ce = dda.c_ext(E, P, k)
    assert abs(ce - 4 * math.pi * k * alpha.imag) < 1e-14
    cs = dda.c_sca_double_sum(c, P, k)
    assert abs(cs - 8 * math.pi / 3 * k ** 4 * abs(alpha) ** 2) < 1e-14
    # radiative reaction makes the single-dipole optical theorem exact
    assert abs(ce - dda.c_abs(ainv, P, k) - cs) < 1e-14


def test_lossless_absorbs_nothing():
    # real m: RR and LDR both give Im(1/alpha) = -(2/3) k^3, so C_abs = 0
    k = 0.4
    for alpha in (dda.alpha_rr(1.5, k), dda.alpha_ldr(1.5, k, [0, 0, 1], [1, 0, 0]),
                  dda.alpha_ldr(1.5, k, [0.6, 0, 0.8], [0.8, 0, -0.6])):
        assert abs((1.0 / alpha).imag + (2.0 / 3.0) * k ** 3) < 1e-15
    mask = synth.sphere(5)
    c, ainv = _setup(mask, k, m=1.5)
    E = dda.incident_field(c, k, [0, 0, 1], [1, 0, 0])
    P = np.linalg.solve(dda.dense_matrix(c, ainv, k), E.reshape(-1)).reshape(3, -1)
    assert abs(dda.c_abs(ainv, P, k)) < 1e-12 * dda.c_ext(E, P, k)


def test_ldr_reduces_to_cm_at_zero_k():
    for m in (1.33 + 0.01j, 2.0 + 0.5j):
        assert abs(dda.alpha_ldr(m, 0.0, [0, 0, 1], [1, 0, 0]) - dda.alpha_cm(m)) < 1e-16
        assert abs(dda.alpha_rr(m, 0.0) - dda.alpha_cm(m)) < 1e-16


def test_incident_field_phase():
    c = np.array([[0, 0, 0], [3, 1, 2]], dtype=np.int32)
    E = dda.incident_field(c, 0.5, [0, 0, 1], [0, 1, 0])
    assert np.allclose(E[:, 0], [0, 1, 0])
    assert np.allclose(E[:, 1], [0, np.exp(1j * 0.5 * 2), 0])


# ----------------------------------------------------- cross sections/solve

def _solved(mask, k, m):
    c, ainv = _setup(mask, k, m=m)
    E = dda.incident_field(c, k, [0, 0, 1], [1, 0, 0])
    A = dda.dense_matrix(c, ainv, k)
    P = np.linalg.solve(A, E.reshape(-1)).reshape(3, -1)
    return c, ainv, E, A, P


def test_optical_theorem_and_far_field():
    # C_ext = C_abs + C_sca for the exact solution; the far-field quadrature
    # does not use A at all, so it checks the double sum independently
    k = 0.5
    c, ainv, E, A, P = _solved(synth.sphere(6, box=(6, 6, 7)), k, 1.33 + 0.05j)
    ce, ca = dda.c_ext(E, P, k), dda.c_abs(ainv, P, k)
    cs = dda.c_sca_double_sum(c, P, k)
    cf = dda.c_sca_far_field(c, P, k)
    assert abs(cs - cf) < 1e-12 * cs
    assert abs(ce - ca - cs) < 1e-12 * ce


@pytest.mark.parametrize("name", ["bicg", "bicg_sym", "bicgstab", "qmr", "cg", "cgs", "tfqmr", "qmr_sym",
                                  "rbicgstab1", "rbicgstab2", "rbicgstab3"])
def test_solvers_match_lu(name):
    k = 0.45
    c, ainv, E, A, P = _solved(synth.sphere(6), k, 1.33 + 0.01j)
    x, info = solvers.SOLVERS[name](lambda v: A @ v, E.reshape(-1), tol=1e-12, max_iter=500)
    assert info["converged"]
    assert np.abs(x - P.reshape(-1)).max() <= 1e-10 * np.abs(P).max()
    # true residual within a small factor of the tolerance
    assert np.linalg.norm(E.reshape(-1) - A @ x) <= 1e-11 * np.linalg.norm(E)


def test_bicg_equals_bicg_sym_iterates():
    # shadow conj(r0) with A = A^T makes BiCG and BiCG_sym the same iteration
    k = 0.45
    c, ainv, E, A, P = _solved(synth.sphere(5), k, 1.33 + 0.01j)
    for it in (3, 7):
        x1, i1 = solvers.bicg(lambda v: A @ v, E.reshape(-1), tol=0, max_iter=it)
        x2, i2 = solvers.bicg_sym(lambda v: A @ v, E.reshape(-1), tol=0, max_iter=it)
        assert np.abs(x1 - x2).max() <= 1e-12 * np.abs(x1).max()
        assert i1["matvecs"] == 2 * i2["matvecs"]


def test_cg_and_qmr_sym_follow_their_symmetric_twins():
    # with the bilinear form, CG is BiCG_sym step for step; QMR_sym's single
    # Lanczos sequence reproduces QMR's (w_n = v_n) with half the products
    k = 0.45
    c, ainv, E, A, P = _solved(synth.sphere(5), k, 1.33 + 0.01j)
    op = lambda v: A @ v
    for it in (2, 5, 9):
        x1, i1 = solvers.bicg_sym(op, E.reshape(-1), tol=0, max_iter=it)
        x2, i2 = solvers.cg(op, E.reshape(-1), tol=0, max_iter=it)
        assert np.abs(x1 - x2).max() <= 1e-12 * np.abs(x1).max()
        assert i1["matvecs"] == i2["matvecs"] == it
        y1, j1 = solvers.qmr(op, E.reshape(-1), tol=0, max_iter=it)
        y2, j2 = solvers.qmr_sym(op, E.reshape(-1), tol=0, max_iter=it)
        assert np.abs(y1 - y2).max() <= 1e-11 * np.abs(y1).max()
        assert j1["matvecs"] == 2 * j2["matvecs"]


def test_bicgstab_l_with_one_is_bicgstab():
    # BiCGSTAB(1) is BiCGSTAB (Sleijpen & Fokkema 1993): same iterates when
    # neither stops early; BiCGSTAB(ell) for ell = 2, 3 builds the same
    # Krylov space with 2 ell products per cycle
    k = 0.45
    c, ainv, E, A, P = _solved(synth.sphere(5), k, 1.33 + 0.05j)
    b = E.reshape(-1)
    for it in (1, 3, 6):
        x1, i1 = solvers.bicgstab_l(lambda v: A @ v, b, tol=0, max_iter=it, ell=1)
        x2, i2 = solvers.bicgstab(lambda v: A @ v, b, tol=0, max_iter=it)
        assert np.abs(x1 - x2).max() <= 1e-12 * np.abs(x2).max()
        assert i1["matvecs"] == i2["matvecs"] == 2 * it
    for ell in (2, 3):
        x, info = solvers.bicgstab_l(lambda v: A @ v, b, tol=0, max_iter=2, ell=ell)
        assert info["matvecs"] == 4 * ell


def test_tfqmr_bound_covers_true_residual():
    # the quasi-residual bound tau sqrt(m+1) is an upper bound of ||r_m||,
    # so the stopping test never stops early
    k = 0.45
    c, ainv, E, A, P = _solved(synth.sphere(6), k, 1.33 + 0.05j)
    b = E.reshape(-1)
    for tol in (1e-3, 1e-6, 1e-9):
        x, info = solvers.tfqmr(lambda v: A @ v, b, tol=tol, max_iter=500)
        assert info["converged"]
        true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert true <= info["rel_residual"] * (1 + 1e-9) and true <= tol


def test_cgs_is_bicg_squared():
    # CGS's residual polynomial is the square of BiCG's: after n steps with the
    # same shadow vector, r_CGS = phi_n(A)^2 r0 where r_BiCG = phi_n(A) r0
    k = 0.45
    c, ainv, E, A, P = _solved(synth.sphere(4), k, 1.33 + 0.01j)
    b = E.reshape(-1)
    # BiCG with shadow r0 (not conj(r0)): run the recurrence by hand for phi_n
    n = 3
    r = b.copy(); rt = b.copy(); p = pt = None; rho_old = None
    alphas, betas = [], []
    for it in range(n):
        rho = np.vdot(rt, r)
        if it == 0:
            p, pt = r.copy(), rt.copy()
        else:
            beta = rho / rho_old; betas.append(beta)
            p = r + beta * p; pt = rt + np.conj(beta) * pt
        q = A @ p
        alpha = rho / np.vdot(pt, q); alphas.append(alpha)
        r = r - alpha * q
        rt = rt - np.conj(alpha) * (np.conj(A @ np.conj(pt)))
        rho_old = rho
    # phi_n(A) applied twice to r0, via the coupled recurrences phi, psi
    def apply_phi(v):
        ph, ps = v.copy(), v.copy()
        for it in range(n):
            if it > 0:
                ps = ph + betas[it - 1] * ps
            ph = ph - alphas[it] * (A @ ps)
        return ph
    target = apply_phi(apply_phi(b))
    x, info = solvers.cgs(lambda v: A @ v, b, tol=0, max_iter=n)
    assert np.abs((b - A @ x) - target).max() <= 1e-10 * np.abs(target).max()


def test_jacobi_scaling():
    # one material: diag(A) is a multiple of I, so the scaled system has the
    # same Krylov spaces and the same iterates; two materials: still the LU
    # solution
    k = 0.45
    c, ainv, E, A, P = _solved(synth.sphere(6), k, 1.33 + 0.05j)
    b = E.reshape(-1)
    op = lambda v: A @ v
    for name in ("bicgstab", "qmr_sym", "tfqmr"):
        x1, i1 = solvers.SOLVERS[name](op, b, tol=0, max_iter=6)
        x2, i2 = solvers.jacobi(solvers.SOLVERS[name], np.diag(A))(op, b, tol=0, max_iter=6)
        assert np.abs(x1 - x2).max() <= 1e-10 * np.abs(x1).max(), name
    mask = synth.sphere(6)
    mats = synth.bernoulli_materials(7, mask, 0.4)
    c2, ainv2 = _setup(mask, k, materials=mats, refr=[1.33 + 0.05j, 2.0 + 0.5j])
    A2 = dda.dense_matrix(c2, ainv2, k)
    b2 = dda.incident_field(c2, k, [0, 0, 1], [1, 0, 0]).reshape(-1)
    P2 = np.linalg.solve(A2, b2)
    for name in ("bicg_sym", "bicgstab", "qmr_sym", "tfqmr", "cgs"):
        x, info = solvers.jacobi(solvers.SOLVERS[name], np.diag(A2))(lambda v: A2 @ v, b2, tol=1e-12, max_iter=800)
        assert info["converged"], name
        assert np.abs(x - P2).max() <= 1e-9 * np.abs(P2).max(), name


def test_solver_reports_non_convergence():
    k = 0.45
    c, ainv, E, A, P = _solved(synth.sphere(6), k, 1.33 + 0.01j)
    for f in solvers.SOLVERS.values():
        x, info = f(lambda v: A @ v, E.reshape(-1), tol=1e-14, max_iter=2)
        assert not info["converged"] and info["iterations"] == 2


# ------------------------------------------------------------------- Mie

def test_riccati_bessel_against_scipy():
    # upward recurrence: exact while n <= 2x, slowly losing digits for psi
    # beyond (the series stops at n = x + 4 x^(1/3) + 2, where terms are tiny)
    x = 3.7
    psi, chi = mie.riccati_bessel(x, 12)
    n = np.arange(13)
    rel = np.abs(psi / (x * special.spherical_jn(n, x)) - 1)
    assert rel[:8].max() < 1e-13 and rel.max() < 1e-6
    assert np.allclose(chi, -x * special.spherical_yn(n, x), rtol=1e-13)


def test_mie_rayleigh_limit():
    # x -> 0: Q_abs = 4 x Im((m^2-1)/(m^2+2)), Q_sca = (8/3) x^4 |(m^2-1)/(m^2+2)|^2
    m, x = 1.5 + 0.2j, 1e-3
    qe, qa, qs = mie.efficiencies(m, x)
    f = (m * m - 1) / (m * m + 2)
    assert abs(qa / (4 * x * f.imag) - 1) < 1e-4
    assert abs(qs / (8.0 / 3.0 * x ** 4 * abs(f) ** 2) - 1) < 1e-4


def test_mie_lossless_and_extinction_paradox():
    qe, qa, qs = mie.efficiencies(1.33, 2.0)
    assert abs(qa) < 1e-12
    # extinction paradox: Q_ext -> 2 from above as x grows (edge term ~ x^(-2/3))
    q100 = mie.efficiencies(1.5 + 0.1j, 100.0)[0]
    q400 = mie.efficiencies(1.5 + 0.1j, 400.0)[0]
    assert 2.0 < q400 < q100 < 2.1


def test_mie_textbook_example():
    # Bohren & Huffman (1983), App. A sample run of their program: sphere of
    # radius 0.525 at wavelength 0.6328 (x = 5.2128), m = 1.55: Q_ext = Q_sca = 3.10543
    x = 2.0 * math.pi * 0.525 / 0.6328
    qe, qa, qs = mie.efficiencies(1.55, x)
    assert abs(qe - 3.10543) < 1e-5 and abs(qs - 3.10543) < 1e-5


def test_dda_sphere_approaches_mie():
    # convergence invariant: |Q_DDA - Q_Mie| decreases as the dipole count grows
    # (x = 2: at x = 1 the CM+RR error changes sign near D = 8, so the
    # decrease is only monotone from there on)
    m = 1.33 + 0.01j
    x = 2.0
    errs = []
    for D in (4, 8, 12):
        mask = synth.sphere(D)
        n = int(mask.sum())
        k = x / dda.a_eff(n)
        c, ainv, E, A, P = _solved(mask, k, m)
        q = dda.efficiencies([dda.c_ext(E, P, k)], n)[0]
        errs.append(abs(q / mie.efficiencies(m, x)[0] - 1))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.04


def test_oracle_build_is_idempotent():
    p1 = oracle.build()
    p2 = oracle.build()
    assert p1 == p2


# ---------------------------------------------------------------- adjoint

@pytest.mark.parametrize("rule", ["cm", "cmrr", "ldr"])
def test_alpha_inverse_derivative_against_differences(rule):
    from oracle import adjoint
    k, kh, e0 = 0.5, (0.6, 0.0, 0.8), (0.8, 0.0, -0.6)
    for eps in (1.7689 + 0.0266j, 4.0 + 2.0j):
        h = 1e-6
        fd = (adjoint.alpha_inverse(eps + h, k, rule, kh, e0) - adjoint.alpha_inverse(eps - h, k, rule, kh, e0)) / (2 * h)
        fdi = (adjoint.alpha_inverse(eps + 1j * h, k, rule, kh, e0)
               - adjoint.alpha_inverse(eps - 1j * h, k, rule, kh, e0)) / (2j * h)
        d = adjoint.alpha_inverse_derivative(eps, k, rule, kh, e0)
        assert abs(fd - d) < 1e-7 * abs(d) and abs(fdi - d) < 1e-7 * abs(d)   # holomorphic in eps


@pytest.mark.parametrize("which", ["abs", "ext"])
def test_adjoint_gradient_against_central_differences(which):
    # brute force: perturb one dipole's permittivity, re-solve densely
    from oracle import adjoint
    g = synth.rng(11)
    mask = synth.sphere(6, box=(6, 5, 6))
    c = dda.coords_of(mask)
    n = c.shape[0]
    k, rule = 0.45, "cmrr"
    eps = np.where(g.random(n) < 0.3, (2.0 + 0.5j) ** 2, (1.33 + 0.01j) ** 2)
    E = dda.incident_field(c, k, [0, 0, 1], [1, 0, 0])
    ainv = np.array([[adjoint.alpha_inverse(e, k, rule)] * 3 for e in eps])
    dainv = np.array([[adjoint.alpha_inverse_derivative(e, k, rule)] * 3 for e in eps])
    fn = adjoint.abs_gradient_dense if which == "abs" else adjoint.ext_gradient_dense
    grad, _ = fn(c, ainv, dainv, k, E)
    pick = 1 if which == "abs" else 0
    h = 1e-6
    for j in g.choice(n, size=6, replace=False):
        num = []
        for step in (h, 1j * h):
            ep, em = eps.copy(), eps.copy()
            ep[j] += step
            em[j] -= step
            cp = adjoint.cross_sections_for_eps(c, ep, k, E, rule)[pick]
            cm = adjoint.cross_sections_for_eps(c, em, k, E, rule)[pick]
            num.append((cp - cm) / (2 * h))
        fd = num[0] + 1j * num[1]
        assert abs(fd - grad[j]) <= 1e-6 * np.abs(grad).max()
