"""GPU parity of CG, CGS, TFQMR, QMR_sym, BiCGSTAB(l) and ML(n)BiCGSTAB and
of point-Jacobi preconditioning against the FP64 oracle, through the C ABI.

Targets: the 16^3 sphere of the single-solve tests (one
material: Jacobi is a scalar scaling there) and a 12^3 crop of the 48^3
inclusion cube (host m = 1.33 + 0.001i, inclusions 2.0 + 0.5i), whose two
materials make diag(A) vary from site to site.
"""
import numpy as np
import pytest

import synth
from oracle import dda as odda
from oracle import solvers as osolvers

from _cases import Case, sphere16_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"
NEW = ["cg", "cgs", "tfqmr", "qmr_sym", "rbicgstab1", "rbicgstab2", "rbicgstab3", "mlbicgstab1", "mlbicgstab2",
       "mlbicgstab3"]


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
    P = np.linalg.solve(A, E.reshape(-1)).reshape(3, -1)
    return case, A, E, P


@pytest.fixture(scope="module")
def incl():
    mask, mats = synth.cube_with_inclusions(20260004, 48)
    m1, m2 = 1.33 + 0.001j, 2.0 + 0.5j
    case = Case(synth.crop_center(mask, 12), [m1, m2], 0.5 / abs(m2), synth.crop_center(mats, 12))
    A = odda.dense_matrix(case.coords, case.ainv, case.k)
    E = odda.incident_field(case.coords, case.k, [0, 0, 1], [1, 0, 0])
    P = np.linalg.solve(A, E.reshape(-1)).reshape(3, -1)
    return case, A, E, P


def _gpu_solve(case, E, method, precision, tol, max_iter=3000):
    with case.lattice() as lat:
        Ed = torch.from_numpy(np.ascontiguousarray(E)).to(DEV)
        P = torch.zeros_like(Ed)
        status, info = lat.solve(Ed, P, method, precision, tol=tol, max_iter=max_iter)
        cx = lat.cross_sections(Ed, P)
    return status, info, P.cpu().numpy(), cx


@pytest.mark.parametrize("method", NEW)
def test_new_solvers_fp64_tight(dda, sphere16, method):
    case, A, E, P = sphere16
    status, info, Pg, cx = _gpu_solve(case, E, method, "fp64", 1e-12)
    assert status == dda.DDA_OK, info
    assert info["rel_residual_true"] < 5e-12
    ce, ca = odda.c_ext(E, P, case.k), odda.c_abs(case.ainv, P, case.k)
    assert abs(cx[0] / ce - 1) < 1e-10 and abs(cx[1] / ca - 1) < 1e-10


@pytest.mark.parametrize("method", NEW)
def test_new_solvers_follow_oracle_iterates(dda, sphere16, method):
    case, A, E, P = sphere16
    x, oinfo = osolvers.SOLVERS[method](lambda v: A @ v, E.reshape(-1), tol=1e-8, max_iter=3000)
    status, info, Pg, _ = _gpu_solve(case, E, method, "fp64", 1e-8)
    assert status == dda.DDA_OK
    assert abs(info["iterations"] - oinfo["iterations"]) <= 1, (info, oinfo)
    assert abs(info["matvecs"] - oinfo["matvecs"]) <= 2, (info, oinfo)
    assert np.abs(Pg.reshape(-1) - x).max() <= 1e-6 * np.abs(x).max()


@pytest.mark.parametrize("method", ["bicgstab", "qmr_sym", "tfqmr", "rbicgstab2", "mlbicgstab2", "mlbicgstab3"])
def test_new_solvers_mixed(dda, sphere16, method):
    case, A, E, P = sphere16
    status, info, Pg, cx = _gpu_solve(case, E, method, "mixed", 1e-6)
    assert status == dda.DDA_OK, info
    assert info["rel_residual_true"] <= 1e-6
    ce, ca = odda.c_ext(E, P, case.k), odda.c_abs(case.ainv, P, case.k)
    assert abs(cx[0] / ce - 1) < 1e-5 and abs(cx[1] / ca - 1) < 1e-5


@pytest.mark.parametrize("method", ["bicg_sym", "bicgstab", "qmr_sym", "tfqmr", "cgs", "rbicgstab3", "mlbicgstab2"])
def test_jacobi_two_materials(dda, incl, method):
    case, A, E, P = incl
    status, info, Pg, cx = _gpu_solve(case, E, method + "+jacobi", "fp64", 1e-12)
    assert status == dda.DDA_OK, info
    assert info["rel_residual_true"] < 1e-10
    assert np.abs(Pg - P).max() <= 1e-9 * np.abs(P).max()
    # the same scaled iteration as the oracle's
    x, oinfo = osolvers.jacobi(osolvers.SOLVERS[method], np.diag(A))(lambda v: A @ v, E.reshape(-1), tol=1e-8,
                                                                       max_iter=3000)
    status, info, Pg, _ = _gpu_solve(case, E, method + "+jacobi", "fp64", 1e-8)
    assert status == dda.DDA_OK
    assert abs(info["iterations"] - oinfo["iterations"]) <= 1, (info, oinfo)


def test_jacobi_mixed_two_materials(dda, incl):
    case, A, E, P = incl
    status, info, Pg, cx = _gpu_solve(case, E, "bicgstab+jacobi", "mixed", 1e-6)
    assert status == dda.DDA_OK, info
    assert info["rel_residual_true"] <= 1e-6
    ce = odda.c_ext(E, P, case.k)
    assert abs(cx[0] / ce - 1) < 1e-5


def test_jacobi_single_material_is_a_scaling(dda, sphere16):
    # one material: S A S y = S b has the Krylov spaces of A x = b, so the same
    # iteration count and solution
    case, A, E, P = sphere16
    s0, i0, P0, _ = _gpu_solve(case, E, "qmr_sym", "fp64", 1e-10)
    s1, i1, P1, _ = _gpu_solve(case, E, "qmr_sym+jacobi", "fp64", 1e-10)
    assert s0 == s1 == dda.DDA_OK
    assert abs(i0["iterations"] - i1["iterations"]) <= 1
    assert np.abs(P0 - P1).max() <= 1e-9 * np.abs(P0).max()


@pytest.mark.parametrize("method", ["cg", "cgs", "tfqmr", "qmr_sym", "rbicgstab2", "mlbicgstab3"])
def test_new_solvers_batched(dda, sphere16, method):
    case, A, E, P = sphere16
    pairs = []
    for kh in synth.random_direction(20260061, 2):
        e1, e2 = synth.orthogonal_polarisations(kh)
        pairs += [(kh, e1), (kh, e2)]
    Es = np.stack([odda.incident_field(case.coords, case.k, kh, e) for kh, e in pairs])
    Ps = np.linalg.solve(A, Es.reshape(len(pairs), -1).T).T.reshape(Es.shape)
    with case.lattice() as lat:
        Ed = torch.from_numpy(Es).to(DEV)
        Pd = torch.zeros_like(Ed)
        status, stats, infos = lat.solve_batch(Ed, Pd, method, "fp64", tol=1e-11, max_iter=3000)
    assert status == dda.DDA_OK, stats
    assert np.abs(Pd.cpu().numpy() - Ps).max() <= 1e-8 * np.abs(Ps).max()


def test_ml1_is_bicgstab_on_the_gpu(dda, sphere16):
    # ML(1)BiCGSTAB computes BiCGSTAB's iterates (shadow vector r0): the same
    # iteration count and solution at a stopping tolerance the half-step test
    # of BiCGSTAB does not reach early
    case, A, E, P = sphere16
    s0, i0, P0, _ = _gpu_solve(case, E, "bicgstab", "fp64", 1e-9)
    s1, i1, P1, _ = _gpu_solve(case, E, "mlbicgstab1", "fp64", 1e-9)
    assert s0 == s1 == dda.DDA_OK
    assert abs(i0["iterations"] - i1["iterations"]) <= 1, (i0, i1)
    assert np.abs(P0 - P1).max() <= 1e-7 * np.abs(P0).max()
