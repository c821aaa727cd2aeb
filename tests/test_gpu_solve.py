"""GPU solves and cross sections against the FP64 oracle, through the C ABI.

Config-1 target (16^3 sphere, m = 1.33 + 0.01i, |m| k d = 0.5, CM + RR,
+z incidence, x polarisation): the oracle solves the dense system by LU.
"""
import numpy as np
import pytest

import synth
from oracle import dda as odda
from oracle import solvers as osolvers

from _cases import Case, sphere16_case, random_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def dda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0908_0863_gb300 as m
    return m


@pytest.fixture(scope="module")
def sphere16():
    case = sphere16_case()
    A = odda.dense_matrix(case.coords, case.ainv, case.k)
    E = odda.incident_field(case.coords, case.k, [0, 0, 1], [1, 0, 0])
    P = np.linalg.solve(A, E.reshape(-1)).reshape(3, case.nd)
    C = (odda.c_ext(E, P, case.k), odda.c_abs(case.ainv, P, case.k))
    return case, A, E, P, C


def _solve(dda, case, method, precision, tol, max_iter=2000, khat=(0, 0, 1), e0=(1, 0, 0)):
    with case.lattice() as lat:
        E = torch.empty((3, case.nd), dtype=torch.complex128, device=DEV)
        lat.incident_field(khat, e0, E)
        P = torch.zeros_like(E)
        status, info = lat.solve(E, P, method, precision, tol=tol, max_iter=max_iter)
        cx = lat.cross_sections(E, P)
        return status, info, E.cpu().numpy(), P.cpu().numpy(), cx


def test_incident_field_matches_oracle(dda):
    case = random_case((9, 7, 5), seed=3, fill=0.6, two_materials=False)
    kh = synth.random_direction(4)[0]
    e1, _ = synth.orthogonal_polarisations(kh)
    with case.lattice() as lat:
        E = torch.empty((3, case.nd), dtype=torch.complex128, device=DEV)
        lat.incident_field(kh, e1, E)
        ref = odda.incident_field(case.coords, case.k, kh, e1)
        assert np.abs(E.cpu().numpy() - ref).max() < 1e-14


def test_cross_sections_match_oracle(dda):
    case = random_case((8, 6, 7), seed=5, fill=0.7)
    P = synth.complex_normal(6, (3, case.nd))
    E = odda.incident_field(case.coords, case.k, [0, 0, 1], [1, 0, 0])
    with case.lattice() as lat:
        cx = lat.cross_sections(torch.from_numpy(E).to(DEV), torch.from_numpy(P).to(DEV))
        cx_host = lat.cross_sections(np.ascontiguousarray(E), np.ascontiguousarray(P))
    ce, ca = odda.c_ext(E, P, case.k), odda.c_abs(case.ainv, P, case.k)
    assert abs(cx[0] - ce) <= 1e-12 * abs(ce) and abs(cx[1] - ca) <= 1e-12 * abs(ca)
    assert abs(cx[2] - (ce - ca)) <= 1e-11 * abs(ce)
    assert cx == cx_host


@pytest.mark.parametrize("method", ["bicg", "bicgstab", "qmr"])
def test_fp64_solve_sphere16_tight(dda, sphere16, method):
    # same method, x0 = 0, tol 1e-12 -> cross sections within 1e-10 of the LU solution
    case, A, E, P, C = sphere16
    status, info, Eg, Pg, cx = _solve(dda, case, method, "fp64", 1e-12)
    assert status == dda.DDA_OK, info
    assert np.abs(Eg - E).max() < 1e-14
    assert info["rel_residual_true"] < 5e-12
    assert abs(cx[0] / C[0] - 1) < 1e-10 and abs(cx[1] / C[1] - 1) < 1e-10
    assert abs(cx[2] / (C[0] - C[1]) - 1) < 1e-10
    assert np.abs(Pg - P).max() <= 1e-10 * np.abs(P).max()


@pytest.mark.parametrize("method", ["bicg", "bicgstab", "qmr"])
def test_fp64_iterates_match_oracle_solver(dda, sphere16, method):
    # the device recurrences are the oracle's: same iteration count at tol 1e-8
    case, A, E, P, C = sphere16
    status, info, Eg, Pg, cx = _solve(dda, case, method, "fp64", 1e-8)
    x, oinfo = osolvers.SOLVERS[method](lambda v: A @ v, E.reshape(-1), tol=1e-8, max_iter=2000)
    assert status == dda.DDA_OK
    assert abs(info["iterations"] - oinfo["iterations"]) <= 1
    assert np.abs(Pg.reshape(-1) - x).max() <= 1e-7 * np.abs(x).max()


@pytest.mark.parametrize("method", ["bicg", "bicgstab", "qmr"])
def test_mixed_solve_sphere16(dda, sphere16, method):
    case, A, E, P, C = sphere16
    status, info, Eg, Pg, cx = _solve(dda, case, method, "mixed", 1e-6)
    assert status == dda.DDA_OK, info
    assert info["refinements"] >= 1 and info["rel_residual_true"] <= 1e-6
    assert abs(cx[0] / C[0] - 1) < 1e-5 and abs(cx[1] / C[1] - 1) < 1e-5


def test_optical_theorem_on_gpu_solution(dda):
    # C_ext - C_abs from the GPU equals the oracle's independent C_sca
    case = random_case((7, 6, 5), seed=8, fill=0.8)
    status, info, Eg, Pg, cx = _solve(dda, case, "bicgstab", "fp64", 1e-13)
    assert status == dda.DDA_OK
    cs = odda.c_sca_double_sum(case.coords, Pg, case.k)
    assert abs(cx[2] / cs - 1) < 1e-9


def test_non_convergence_reported(dda, sphere16):
    case = sphere16[0]
    for method in ("bicg", "bicgstab", "qmr"):
        status, info, *_ = _solve(dda, case, method, "fp64", 1e-14, max_iter=3)
        assert status == dda.DDA_ERR_NOT_CONVERGED
        assert info["iterations"] == 3


def test_bad_arguments_rejected(dda):
    alpha = dda.dda_polarizability([1.5], 0.3, "cmrr")
    occ = odda.pack_occupancy(np.ones((2, 2, 2), dtype=np.uint8))
    with pytest.raises(dda.DDAError) as e:
        dda.Lattice((0, 2, 2), occ, alpha, 0.3)
    assert e.value.code == dda.DDA_ERR_ARG
    with pytest.raises(dda.DDAError):
        dda.Lattice((2, 2, 2), occ, alpha, -1.0)
    with pytest.raises(dda.DDAError):
        dda.Lattice((2, 2, 2), np.zeros(1, dtype=np.uint32), alpha, 0.3)   # nothing occupied
    with pytest.raises(dda.DDAError) as e:
        dda.Lattice((2, 2, 2), occ, np.array([[np.nan, 1, 1]], dtype=np.complex128), 0.3)
    assert e.value.code == dda.DDA_ERR_NAN
    # composition index beyond n_materials (3 and 4 materials share 2-bit fields)
    mats = np.full((2, 2, 2, 3), 3, dtype=np.uint8)
    comp = odda.pack_composition(mats, 4)
    al3 = dda.dda_polarizability([1.5, 1.7, 1.9], 0.3, "cmrr")
    with pytest.raises(dda.DDAError) as e:
        dda.Lattice((2, 2, 2), occ, al3, 0.3, comp, 3)
    assert e.value.code == dda.DDA_ERR_ARG
    # more materials than composition bits supplied
    with pytest.raises(dda.DDAError):
        dda.Lattice((2, 2, 2), occ, al3, 0.3, None, 3)


def test_polarizability_matches_oracle(dda):
    k = 0.41
    ms = [1.33 + 0.01j, 2.0 + 0.5j, 1.5]
    got = dda.dda_polarizability(ms, k, "cmrr")
    assert np.allclose(got[:, 0], [odda.alpha_rr(m, k) for m in ms], rtol=1e-15)
    kh, e = [0.6, 0.0, 0.8], [0.8, 0.0, -0.6]
    got = dda.dda_polarizability(ms, k, "ldr", kh, e)
    assert np.allclose(got[:, 1], [odda.alpha_ldr(m, k, kh, e) for m in ms], rtol=1e-15)
    got = dda.dda_polarizability(ms, k, "cm")
    assert np.allclose(got[:, 2], [odda.alpha_cm(m) for m in ms], rtol=1e-15)


def test_inner_tolerance_control_and_autotune(dda):
    """Mixed precision with a coarse inner target (rho = 1e-2) needs more FP64
    refinements and reaches the same tolerance; dda_autotune_inner picks one
    of its candidates, sets it for the tuned method only and hands it to the
    next context of the shape (a lattice shape of its own, so that no other
    test inherits the choice)."""
    m = 1.33 + 0.01j
    case = Case(synth.sphere(16, box=(16, 16, 17)), [m], 0.5 / abs(m))
    with case.lattice() as lat:
        E = torch.empty((3, case.nd), dtype=torch.complex128, device="cuda")
        lat.incident_field([0, 0, 1], [1, 0, 0], E)
        assert dda.dda_inner_tolerance(lat.ctx) == 0.0
        P = torch.zeros_like(E)
        s0, i0 = lat.solve(E, P, "bicgstab", "mixed", tol=1e-8, max_iter=2000)
        assert dda.dda_inner_tolerance(lat.ctx, 1e-2) == 1e-2
        assert dda.dda_inner_tolerance(lat.ctx, method="qmr") == 0.0
        P1 = torch.zeros_like(E)
        s1, i1 = lat.solve(E, P1, "bicgstab", "mixed", tol=1e-8, max_iter=2000)
        assert s0 == s1 == dda.DDA_OK
        assert i1["rel_residual_true"] <= 1e-8 and i1["refinements"] > i0["refinements"]
        assert float((P1 - P).norm() / P.norm()) < 1e-7
        with pytest.raises(dda.DDAError):
            dda.dda_inner_tolerance(lat.ctx, 1.5)
        with pytest.raises(dda.DDAError):
            dda.dda_inner_tolerance(lat.ctx, method=99)
        dda.dda_inner_tolerance(lat.ctx, 0.0)
        dda.dda_inner_tolerance(lat.ctx, 1e-3, method="qmr")
        rho, ms = dda.dda_autotune_inner(lat.ctx, E, "bicgstab+jacobi", 1e-8, 2000)
        assert rho in ms and ms[rho] > 0 and all(v == -1 or v > 0 for v in ms.values())
        assert dda.dda_inner_tolerance(lat.ctx) == rho
        assert dda.dda_inner_tolerance(lat.ctx, method="qmr") == 1e-3
    with case.lattice() as lat2:
        assert dda.dda_inner_tolerance(lat2.ctx) == rho
        assert dda.dda_inner_tolerance(lat2.ctx, method="qmr") == 0.0


def test_mixed_refinement_residual_products(dda):
    """The mixed refinement's true residuals from double-float products (the
    default) and from FP64 products give the same solve to 1e-10 at tol 1e-10
    (FP64 solve as the reference), both with a true residual within tol."""
    m = 1.33 + 0.01j
    case = Case(synth.sphere(18, box=(18, 17, 19)), [m], 0.5 / abs(m))
    with case.lattice() as lat:
        assert dda.dda_residual_dtype(lat.ctx) == "c128df"
        E = torch.empty((3, case.nd), dtype=torch.complex128, device="cuda")
        lat.incident_field([0.6, 0, 0.8], [0, 1, 0], E)
        Pf = torch.zeros_like(E)
        sf, _ = lat.solve(E, Pf, "bicgstab", "fp64", tol=1e-12, max_iter=4000)
        out = {}
        for rd in ("c128df", "c128"):
            assert dda.dda_residual_dtype(lat.ctx, rd) == rd
            P = torch.zeros_like(E)
            st, info = lat.solve(E, P, "bicgstab", "mixed", tol=1e-10, max_iter=4000)
            assert st == dda.DDA_OK and info["rel_residual_true"] <= 1e-10, (rd, info)
            out[rd] = (P, info)
        assert sf == dda.DDA_OK
        for rd, (P, info) in out.items():
            assert float((P - Pf).norm() / Pf.norm()) < 1e-9, rd
        with pytest.raises(dda.DDAError):
            dda.dda_residual_dtype(lat.ctx, "c64")
