"""GPU parity of BiCG_sym, the pair-sum C_sca and the adjoint permittivity
gradients against the FP64 oracle, through the C ABI.

Gradient target (the differentiation workload): a 48^3 cube host, m = 1.33 +
0.001i, with random spherical inclusions of radius 3-6 dipoles up to 20 %
volume, m = 2.0 + 0.5i, CM + radiative reaction, |m_incl| k d = 0.5; the
oracle's dense adjoint runs on its central 12^3 crop.
"""
import math

import numpy as np
import pytest

import synth
from oracle import adjoint as oadj
from oracle import dda as odda
from oracle import solvers as osolvers

from _cases import Case, sphere16_case, random_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"
M_HOST, M_INCL = 1.33 + 0.001j, 2.0 + 0.5j
K_GRAD = 0.5 / abs(M_INCL)


@pytest.fixture(scope="module")
def dda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0908_0863_gb300 as m
    return m


@pytest.fixture(scope="module")
def crop_case():
    mask, mats = synth.cube_with_inclusions(20260004, 48)
    return Case(synth.crop_center(mask, 12), [M_HOST, M_INCL], K_GRAD, synth.crop_center(mats, 12))


def _solve_P(lat, case, method="bicgstab", precision="fp64", tol=1e-13):
    E = torch.empty((3, case.nd), dtype=torch.complex128, device=DEV)
    lat.incident_field([0, 0, 1], [1, 0, 0], E)
    P = torch.zeros_like(E)
    status, info = lat.solve(E, P, method, precision, tol=tol, max_iter=4000)
    assert status == 0, info
    return E, P


# ---------------------------------------------------------------- BiCG_sym

def test_bicg_sym_iterates_match_oracle(dda):
    case = sphere16_case()
    A = odda.dense_matrix(case.coords, case.ainv, case.k)
    E = odda.incident_field(case.coords, case.k, [0, 0, 1], [1, 0, 0])
    x, oinfo = osolvers.bicg_sym(lambda v: A @ v, E.reshape(-1), tol=1e-8, max_iter=2000)
    with case.lattice() as lat:
        Ed = torch.from_numpy(E).to(DEV)
        P = torch.zeros_like(Ed)
        status, info = lat.solve(Ed, P, "bicg_sym", "fp64", tol=1e-8, max_iter=2000)
    assert status == dda.DDA_OK
    assert abs(info["iterations"] - oinfo["iterations"]) <= 1
    assert info["matvecs"] == info["iterations"]          # one product per iteration
    assert np.abs(P.cpu().numpy().reshape(-1) - x).max() <= 1e-7 * np.abs(x).max()


def test_bicg_sym_tight_cross_sections(dda):
    case = sphere16_case()
    A = odda.dense_matrix(case.coords, case.ainv, case.k)
    E = odda.incident_field(case.coords, case.k, [0, 0, 1], [1, 0, 0])
    Pref = np.linalg.solve(A, E.reshape(-1)).reshape(3, -1)
    with case.lattice() as lat:
        Ed, P = _solve_P(lat, case, "bicg_sym", "fp64", 1e-12)
        cx = lat.cross_sections(Ed, P)
    assert abs(cx[0] / odda.c_ext(E, Pref, case.k) - 1) < 1e-10
    assert abs(cx[1] / odda.c_abs(case.ainv, Pref, case.k) - 1) < 1e-10


# -------------------------------------------------------------- C_sca sum

def test_csca_pair_sum_matches_oracle(dda):
    case = random_case((9, 7, 8), seed=21, fill=0.7)
    P = synth.complex_normal(22, (3, case.nd))
    ref = odda.c_sca_double_sum(case.coords, P, case.k)
    with case.lattice() as lat:
        got = lat.scattering_cross_section(torch.from_numpy(P).to(DEV))
        got_host = lat.scattering_cross_section(np.ascontiguousarray(P))
    assert abs(got / ref - 1) < 1e-11
    assert got == got_host


def test_optical_theorem_with_gpu_csca(dda):
    case = sphere16_case()
    with case.lattice() as lat:
        E, P = _solve_P(lat, case, "bicgstab", "fp64", 1e-13)
        cext, cabs, _ = lat.cross_sections(E, P)
        csca = lat.scattering_cross_section(P)
    assert abs((cext - cabs) / csca - 1) < 1e-10


# ---------------------------------------------------------------- adjoint

def _gpu_gradient(dda, lat, case, which, precision="fp64", tol=1e-13):
    E, P = _solve_P(lat, case, "bicgstab", precision, tol)
    dainv = dda.dda_polarizability_derivative(case.refr, case.k, "cmrr")
    g = torch.empty(case.nd, dtype=torch.complex128, device=DEV)
    status, info = lat.gradient(which, E, P, dainv, g, "bicgstab", precision, tol, 4000)
    assert status == dda.DDA_OK, info
    return g.cpu().numpy()


def _oracle_dainv(case):
    mats = case.materials.reshape(-1, 3)[odda.occupied_sites(case.mask)]
    d = np.array([oadj.alpha_inverse_derivative(m * m, case.k, "cmrr") for m in case.refr])
    return d[mats]                                             # (N_d, 3)


@pytest.mark.parametrize("which", ["abs", "ext"])
def test_gradient_matches_dense_adjoint(dda, crop_case, which):
    case = crop_case
    E = odda.incident_field(case.coords, case.k, [0, 0, 1], [1, 0, 0])
    fn = oadj.abs_gradient_dense if which == "abs" else oadj.ext_gradient_dense
    ref, _ = fn(case.coords, case.ainv, _oracle_dainv(case), case.k, E)
    with case.lattice() as lat:
        g = _gpu_gradient(dda, lat, case, which)
    assert np.abs(g - ref).max() <= 1e-9 * np.abs(ref).max()


def test_gradient_matches_central_differences(dda, crop_case):
    # 50 random dipoles: move one dipole's permittivity by +-1e-6 (real and
    # imaginary) by giving it a material of its own, re-solve, difference C_abs
    case = crop_case
    with case.lattice() as lat:
        g = _gpu_gradient(dda, lat, case, "abs")
    occ = odda.occupied_sites(case.mask)
    mats = case.materials.reshape(-1, 3)
    h = 1e-6
    pick = synth.rng(20260041).choice(case.nd, size=50, replace=False)
    for j in pick:
        s = occ[j]
        eps0 = case.refr[mats[s, 0]] ** 2
        num = []
        for step in (h, 1j * h):
            vals = []
            for sgn in (1, -1):
                m_new = np.sqrt(eps0 + sgn * step)
                mm = mats.copy()
                mm[s, :] = 2
                c2 = Case(case.mask, case.refr + [m_new], case.k, mm.reshape(case.materials.shape))
                with c2.lattice() as lat2:
                    E2, P2 = _solve_P(lat2, c2, "bicgstab", "fp64", 1e-14)
                    vals.append(lat2.cross_sections(E2, P2)[1])
            num.append((vals[0] - vals[1]) / (2 * h))
        fd = num[0] + 1j * num[1]
        assert abs(fd - g[j]) <= 1e-4 * np.abs(g).max(), (j, fd, g[j])


def test_mixed_gradient_close_to_fp64(dda):
    # the full 48^3 inclusion cube: mixed-precision forward and adjoint solves
    mask, mats = synth.cube_with_inclusions(20260004, 48)
    case = Case(mask, [M_HOST, M_INCL], K_GRAD, mats)
    with case.lattice() as lat:
        g64 = _gpu_gradient(dda, lat, case, "abs", "fp64", 1e-10)
        g32 = _gpu_gradient(dda, lat, case, "abs", "mixed", 1e-8)
    assert np.abs(g32 - g64).max() <= 1e-4 * np.abs(g64).max()


def test_autograd_function_material_gradient(dda, crop_case):
    from paper_0908_0863_gb300.autograd import CrossSection, Target
    case = crop_case
    occ = odda.occupied_sites(case.mask)
    tgt = Target(shape=case.shape, occupancy_bits=case.occ_bits, k=case.k, which="abs", rule="cmrr",
                 composition_bits=case.comp_bits, tol=1e-13)
    eps = torch.tensor([m * m for m in case.refr], dtype=torch.complex128, requires_grad=True)
    c = CrossSection.apply(eps, tgt)
    c.backward()
    ref = abs(c.item() - odda.c_abs(case.ainv, np.linalg.solve(
        odda.dense_matrix(case.coords, case.ainv, case.k),
        odda.incident_field(case.coords, case.k, [0, 0, 1], [1, 0, 0]).reshape(-1)).reshape(3, -1), case.k))
    assert ref < 1e-9 * abs(c.item())
    # finite differences on each material permittivity
    h = 1e-6
    for q in range(2):
        fd = []
        for step in (h, 1j * h):
            e_p, e_m = eps.detach().clone(), eps.detach().clone()
            e_p[q] += step
            e_m[q] -= step
            fd.append((CrossSection.apply(e_p, tgt).item() - CrossSection.apply(e_m, tgt).item()) / (2 * h))
        fdq = fd[0] + 1j * fd[1]
        assert abs(fdq - eps.grad[q].item()) <= 1e-5 * abs(eps.grad).max().item()


def test_material_sums_match_dense_adjoint(dda, crop_case):
    """dda_material_sums of the per-dipole gradient equals the oracle's
    dense-adjoint gradient summed over the dipoles of each material, and a
    permittivity passed as eps (DDA_POL_EPS) gives the polarisability and
    its derivative of the same material passed as m."""
    case = crop_case
    occ = odda.occupied_sites(case.mask)
    mats = case.materials.reshape(-1, 3)[occ, 0]
    eps = np.array([m * m for m in case.refr])
    assert np.array_equal(dda.dda_polarizability(eps, case.k, "cmrr", given="eps"),
                          dda.dda_polarizability(case.refr, case.k, "cmrr"))
    d_eps = dda.dda_polarizability_derivative(eps, case.k, "cmrr", given="eps")
    d_m = dda.dda_polarizability_derivative(case.refr, case.k, "cmrr")
    assert np.abs(d_eps - d_m).max() <= 1e-15 * np.abs(d_m).max()
    with case.lattice() as lat:
        g = _gpu_gradient(dda, lat, case, "abs", "fp64", 1e-13)
        sums = dda.dda_material_sums(lat.ctx, torch.from_numpy(g).to(DEV), case.nmat)
        sums_host = dda.dda_material_sums(lat.ctx, np.ascontiguousarray(g), case.nmat)
    assert np.array_equal(sums, sums_host)
    E = odda.incident_field(case.coords, case.k, [0, 0, 1], [1, 0, 0])
    ref, _ = oadj.abs_gradient_dense(case.coords, case.ainv, _oracle_dainv(case), case.k, E)
    want = np.array([ref[mats == q].sum() for q in range(case.nmat)])
    assert np.abs(sums - want).max() <= 1e-9 * np.abs(want).max()
