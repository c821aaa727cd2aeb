"""GPU check against the paper's own validation run (Table 7).

CUBE of 100^3 dipoles (N = N_d = 10^6), normal incidence on one face, x
polarisation, lambda = 3.175 um, a_eff = 0.5 um, m = 1.63631 + 0.372i:
OpenDDA prints Q_ext = 1.265, Q_abs = 0.911, Q_sca = 0.354 (DDSCAT 1.264 /
0.911 / 0.353).  The paper does not say which polarisability it used;
lattice dispersion relations are the usual default of DDA codes; with LDR
this path reproduces all three printed values to their last digit, so the
check allows 0.0006 (half a unit of the printed digit plus margin).  10^6 dipoles are beyond the direct-sum
oracle, so this is a GPU-only check of the whole path against printed values.
"""
import math

import numpy as np
import pytest

import synth
from oracle import dda as odda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0908_0863_gb300 as m
    return m


def _cube_efficiencies(dda, rule, precision="fp64", tol=1e-10):
    t7 = {"lambda_um": 3.175, "a_eff_um": 0.5, "m": complex(1.63631, 0.372)}
    n = 100
    nd = n ** 3
    x = 2.0 * math.pi * t7["a_eff_um"] / t7["lambda_um"]
    aeff = odda.a_eff(nd)
    k = x / aeff                              # wavenumber in units of the lattice spacing
    khat, e0 = [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]
    alpha = dda.dda_polarizability([t7["m"]], k, rule, khat, e0)
    bits = odda.pack_occupancy(synth.cube(n))
    with dda.Lattice((n, n, n), bits, alpha, k) as lat:
        assert lat.n_dipoles == nd
        E = torch.empty((3, nd), dtype=torch.complex128, device="cuda")
        lat.incident_field(khat, e0, E)
        P = torch.zeros_like(E)
        status, info = lat.solve(E, P, "bicgstab", precision, tol=tol, max_iter=4000)
        assert status == dda.DDA_OK, info
        cext, cabs, csca = lat.cross_sections(E, P)
    g = math.pi * aeff ** 2
    return cext / g, cabs / g, csca / g, info


def test_table7_cube_ldr(dda, golden):
    t = golden["table7_cube_validation"]
    qe, qa, qs, info = _cube_efficiencies(dda, "ldr")
    print(f"CUBE 100^3 LDR: Q_ext {qe:.5f} Q_abs {qa:.5f} Q_sca {qs:.5f} "
          f"({info['iterations']} BiCGSTAB iterations)")
    assert abs(qe - t["Q_ext"]) <= 0.0006
    assert abs(qa - t["Q_abs"]) <= 0.0006
    assert abs(qs - t["Q_sca"]) <= 0.0006


def test_table7_cube_mixed_matches_fp64(dda):
    # the mixed-precision path reaches the same efficiencies to 1e-5
    a = _cube_efficiencies(dda, "ldr", "fp64", 1e-8)
    b = _cube_efficiencies(dda, "ldr", "mixed", 1e-8)
    for u, v in zip(a[:3], b[:3]):
        assert abs(u / v - 1) < 1e-5


def test_table3_iteration_counts(dda, golden):
    """The paper's solver benchmark (Sec. 6, Table 3): SPHERE 200^3, x =
    0.98948, m = 1.63631 + 0.372i, point-Jacobi, tol 1e-10, x0 = 0.  The
    paper does not state its stopping test; with ours (recurrence residual
    <= tol ||E||, TFQMR's quasi-residual bound, BiCGSTAB(l) at the end of a
    cycle, ML(n)BiCGSTAB at the end of a cycle of n + 1 products) every
    scheme stops within two iterations of the printed count, and BiCGSTAB,
    CGS, TFQMR, BiCGSTAB(3) and ML(n)BiCGSTAB for n = 1, 2, 3 (12, 8 and 6
    cycles) on it.  The polarisability is LDR (the reading Table 7 pins)."""
    t = golden["table3_iterations"]
    n = t["n"]
    m = complex(t["m_re"], t["m_im"])
    mask = synth.sphere(n)
    nd = int(mask.sum())
    k = t["x"] / odda.a_eff(nd)
    alpha = dda.dda_polarizability([m], k, "ldr", [0, 0, 1], [1, 0, 0])
    got = {}
    with dda.Lattice((n, n, n), odda.pack_occupancy(mask), alpha, k) as lat:
        E = torch.empty((3, nd), dtype=torch.complex128, device="cuda")
        lat.incident_field([0, 0, 1], [1, 0, 0], E)
        for method, ni in t["iterations"].items():
            P = torch.zeros_like(E)
            status, info = lat.solve(E, P, method + "+jacobi", "fp64", tol=t["tol"], max_iter=10000)
            assert status == dda.DDA_OK, (method, info)
            assert info["rel_residual_true"] <= t["tol"]
            got[method] = info["iterations"]
    print("Table 3 iterations (ours / paper):", {m: (got[m], t["iterations"][m]) for m in got})
    for method, ni in t["iterations"].items():
        assert abs(got[method] - ni) <= 2, (method, got[method], ni)
    for method in ("bicgstab", "cgs", "tfqmr", "rbicgstab3", "mlbicgstab1", "mlbicgstab2", "mlbicgstab3"):
        assert got[method] == t["iterations"][method]


def test_sphere_converges_to_mie_at_scale(dda):
    """Convergence to Mie theory at GPU scale: a sphere of fixed size
    parameter x = 3 (m = 1.33 + 0.05i) discretised with D = 16, 32, 64 and
    128 dipoles across (|m| k d from 0.5 down to 0.06, up to 1.1 M dipoles),
    solved in FP64 and compared with the oracle's Mie series.  With LDR the
    Q_abs error falls at every doubling; the Q_ext error changes sign near
    D = 32 (measured 1.8e-3, 1.2e-5, 1.5e-4, 2.9e-5), so for Q_ext the check
    is that the larger lattices stay an order of magnitude below D = 16.
    Both end below 1e-4."""
    from oracle import mie
    m = 1.33 + 0.05j
    x = 3.0
    qm = mie.efficiencies(m, x)
    err_ext, err_abs = [], []
    for D in (16, 32, 64, 128):
        mask = synth.sphere(D)
        nd = int(mask.sum())
        aeff = odda.a_eff(nd)
        k = x / aeff
        alpha = dda.dda_polarizability([m], k, "ldr", [0, 0, 1], [1, 0, 0])
        with dda.Lattice((D, D, D), odda.pack_occupancy(mask), alpha, k) as lat:
            E = torch.empty((3, nd), dtype=torch.complex128, device="cuda")
            lat.incident_field([0, 0, 1], [1, 0, 0], E)
            P = torch.zeros_like(E)
            status, info = lat.solve(E, P, "bicgstab", "fp64", tol=1e-9, max_iter=4000)
            assert status == dda.DDA_OK, info
            cext, cabs, _ = lat.cross_sections(E, P)
        g = math.pi * aeff ** 2
        err_ext.append(abs(cext / g / qm[0] - 1))
        err_abs.append(abs(cabs / g / qm[1] - 1))
    print("Q_ext / Q_abs relative errors vs Mie at D = 16, 32, 64, 128:", err_ext, err_abs)
    assert all(b < a for a, b in zip(err_abs, err_abs[1:]))
    assert max(err_ext[1:]) < err_ext[0] / 10
    assert max(err_ext + err_abs) < 5e-3
    assert err_ext[-1] < 1e-4 and err_abs[-1] < 1e-4
