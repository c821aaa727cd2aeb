"""GPU parity of the batched entry points: many right-hand sides (incidence
directions and polarisations) sharing one target's spectrum, through the C
ABI.

Targets: the 16^3 sphere of the single-solve tests; random ragged lattices
for the batched product; ballistic aggregates of touching spheres (the
batching workload: m = 1.6 + 0.05i, |m| k d = 0.5, CM + RR), a small one
that the oracle solves by dense LU and a 200-monomer one (monomer diameter
8) checked on sampled rows of the direct sum.
"""
import numpy as np
import pytest

import synth
from oracle import dda as odda

from _cases import Case, sphere16_case, random_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"
M_AGG = 1.6 + 0.05j


@pytest.fixture(scope="module")
def dda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0908_0863_gb300 as m
    return m


def _pairs(seed, n_dirs):
    """(khat, e) for n_dirs seeded directions x 2 orthogonal polarisations."""
    out = []
    for kh in synth.random_direction(seed, n_dirs):
        e1, e2 = synth.orthogonal_polarisations(kh)
        out += [(kh, e1), (kh, e2)]
    return out


def _einc(lat, nd, pairs):
    E = torch.empty((len(pairs), 3, nd), dtype=torch.complex128, device=DEV)
    for b, (kh, e) in enumerate(pairs):
        lat.incident_field(kh, e, E[b])
    return E


def _oracle_lu(case, pairs):
    A = odda.dense_matrix(case.coords, case.ainv, case.k)
    Es = np.stack([odda.incident_field(case.coords, case.k, kh, e).reshape(-1) for kh, e in pairs], axis=1)
    Ps = np.linalg.solve(A, Es)
    cx = []
    for b in range(len(pairs)):
        E, P = Es[:, b].reshape(3, -1), Ps[:, b].reshape(3, -1)
        cx.append((odda.c_ext(E, P, case.k), odda.c_abs(case.ainv, P, case.k)))
    return Es.T.reshape(len(pairs), 3, -1), Ps.T.reshape(len(pairs), 3, -1), np.array(cx)


@pytest.fixture(scope="module")
def c1_batch():
    case = sphere16_case()
    pairs = _pairs(20260051, 3)
    return case, pairs, _oracle_lu(case, pairs)


def _small_aggregate():
    mask, _ = synth.ballistic_aggregate(20260003, 6, mono_diameter=6)
    return Case(mask, [M_AGG], 0.5 / abs(M_AGG))


# ----------------------------------------------------------------- product

@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_matvec_batch_bit_exact(dda, dtype):
    case = random_case((11, 9, 7), seed=31, fill=0.7)
    nb = 5
    p = torch.from_numpy(synth.complex_normal(32, (nb, 3, case.nd))).to(DEV).to(dtype)
    with case.lattice() as lat:
        y = torch.empty_like(p)
        lat.matvec_batch(p, y)
        for b in range(nb):
            pb = p[b].clone()            # own allocation: 16-byte aligned as the ABI asks
            yb = torch.empty_like(pb)
            lat.matvec(pb, yb)
            assert torch.equal(y[b], yb), b


def test_matvec_batch_chunked_128(dda):
    # three complex128 right-hand sides at 128^3: the work space holds fewer
    # complex128 slots than that, so the batch runs in chunks
    case = Case(synth.sphere(128, 120), [1.33 + 0.05j], 0.5 / abs(1.33 + 0.05j))
    nb = 3
    p_host = synth.complex_normal(33, (nb, 3, case.nd))
    p = torch.from_numpy(p_host).to(DEV)
    rows = synth.rng(34).choice(case.nd, size=16, replace=False)
    with case.lattice() as lat:
        y = torch.empty_like(p)
        lat.matvec_batch(p, y)
        for b in range(nb):
            yb = torch.empty_like(p[b])
            lat.matvec(p[b], yb)
            assert torch.equal(y[b], yb), b
    yh = y.cpu().numpy()
    for b in range(nb):
        ref = odda.direct_matvec_rows(case.coords, case.ainv, case.k, p_host[b], rows)
        got = yh[b][:, rows]
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


# ------------------------------------------------------------------ solves

@pytest.mark.parametrize("method", ["bicg", "bicgstab", "qmr", "bicg_sym"])
def test_solve_batch_fp64_matches_lu(dda, c1_batch, method):
    case, pairs, (Es, Ps, cx_ref) = c1_batch
    with case.lattice() as lat:
        E = _einc(lat, case.nd, pairs)
        assert np.abs(E.cpu().numpy() - Es).max() < 1e-14
        P = torch.zeros_like(E)
        status, stats, infos = lat.solve_batch(E, P, method, "fp64", tol=1e-12, max_iter=2000)
        cx = lat.cross_sections_batch(E, P)
    assert status == dda.DDA_OK and stats == [0] * len(pairs), (stats, infos)
    for b in range(len(pairs)):
        assert infos[b]["rel_residual_true"] < 5e-12
        assert abs(cx[b, 0] / cx_ref[b, 0] - 1) < 1e-10, b
        assert abs(cx[b, 1] / cx_ref[b, 1] - 1) < 1e-10, b
        assert abs(cx[b, 2] / (cx_ref[b, 0] - cx_ref[b, 1]) - 1) < 1e-9, b


@pytest.mark.parametrize("method", ["bicgstab", "qmr"])
def test_solve_batch_mixed_matches_lu(dda, c1_batch, method):
    case, pairs, (Es, Ps, cx_ref) = c1_batch
    with case.lattice() as lat:
        E = _einc(lat, case.nd, pairs)
        P = torch.zeros_like(E)
        status, stats, infos = lat.solve_batch(E, P, method, "mixed", tol=1e-6, max_iter=2000)
        cx = lat.cross_sections_batch(E, P)
    assert status == dda.DDA_OK, (stats, infos)
    for b in range(len(pairs)):
        assert infos[b]["rel_residual_true"] <= 1e-6
        assert infos[b]["refinements"] >= 1 and infos[b]["matvecs_fp64"] == infos[b]["refinements"]
        assert abs(cx[b, 0] / cx_ref[b, 0] - 1) < 1e-5 and abs(cx[b, 1] / cx_ref[b, 1] - 1) < 1e-5, b


def test_batch_equals_single_solves(dda, c1_batch):
    case, pairs, _ = c1_batch
    with case.lattice() as lat:
        E = _einc(lat, case.nd, pairs[:4])
        P = torch.zeros_like(E)
        status, _, infos = lat.solve_batch(E, P, "bicgstab", "fp64", tol=1e-10, max_iter=2000)
        assert status == dda.DDA_OK
        for b in range(4):
            Pb = torch.zeros_like(E[b])
            st1, info1 = lat.solve(E[b], Pb, "bicgstab", "fp64", tol=1e-10, max_iter=2000)
            assert st1 == dda.DDA_OK
            assert abs(info1["iterations"] - infos[b]["iterations"]) <= 1
            d = (P[b] - Pb).abs().max().item()
            assert d <= 1e-8 * Pb.abs().max().item(), b


def test_graph_replay_is_exact(dda, c1_batch):
    # profiling on runs every iteration with plain launches; off, iterations
    # after the first are replayed from a captured CUDA graph: same kernels,
    # same order, so the same bits and the same launch count
    case, pairs, _ = c1_batch
    out, launches = [], []
    with case.lattice() as lat:
        E = _einc(lat, case.nd, pairs)
        for prof in (True, False):
            dda.dda_profile(lat.ctx, prof)
            P = torch.zeros_like(E)
            n0 = dda.dda_launch_count()
            status, _, infos = lat.solve_batch(E, P, "bicgstab", "mixed", tol=1e-6, max_iter=2000)
            launches.append(dda.dda_launch_count() - n0)
            assert status == dda.DDA_OK
            out.append(P.clone())
        dda.dda_profile(lat.ctx, False)
    assert torch.equal(out[0], out[1])
    assert launches[0] == launches[1] and launches[0] > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_right_hand_sides_are_independent(dda, c1_batch, precision):
    # a zero right-hand side finishes at once, a non-finite one stops with
    # DDA_ERR_NAN, and neither disturbs the others
    case, pairs, (Es, Ps, cx_ref) = c1_batch
    E = torch.from_numpy(np.stack([Es[0], np.zeros_like(Es[0]), Es[2], Es[3]])).to(DEV)
    E[3, 1, 7] = float("nan")
    with case.lattice() as lat:
        P = torch.zeros_like(E)
        status, stats, infos = lat.solve_batch(E, P, "bicgstab", precision, tol=1e-10, max_iter=2000)
    assert status == dda.DDA_ERR_NAN
    assert stats == [dda.DDA_OK, dda.DDA_OK, dda.DDA_OK, dda.DDA_ERR_NAN], stats
    assert infos[1]["iterations"] == 0 and torch.count_nonzero(P[1]).item() == 0
    Ph = P.cpu().numpy()
    for b in (0, 2):
        assert np.abs(Ph[b] - Ps[b]).max() <= 1e-8 * np.abs(Ps[b]).max(), b


def test_iteration_cap_per_rhs(dda, c1_batch):
    case, pairs, _ = c1_batch
    with case.lattice() as lat:
        E = _einc(lat, case.nd, pairs[:3])
        P = torch.zeros_like(E)
        status, stats, infos = lat.solve_batch(E, P, "qmr", "fp64", tol=1e-15, max_iter=3)
    assert status == dda.DDA_ERR_NOT_CONVERGED
    assert stats == [dda.DDA_ERR_NOT_CONVERGED] * 3
    assert [i["iterations"] for i in infos] == [3, 3, 3]


def test_reserve_then_no_growth(dda, c1_batch):
    case, pairs, _ = c1_batch
    with case.lattice() as lat:
        b0 = dda.dda_query(lat.ctx)["device_bytes"]
        lat.reserve(len(pairs), "mixed")
        b1 = dda.dda_query(lat.ctx)["device_bytes"]
        assert b1 > b0
        E = _einc(lat, case.nd, pairs)
        P = torch.zeros_like(E)
        lat.solve_batch(E, P, "bicgstab", "mixed", tol=1e-6)
        assert dda.dda_query(lat.ctx)["device_bytes"] == b1
        P2 = torch.zeros_like(E[:2])
        lat.solve_batch(E[:2].contiguous(), P2, "bicgstab", "mixed", tol=1e-6)
        assert dda.dda_query(lat.ctx)["device_bytes"] == b1


def test_host_buffers_batch(dda, c1_batch):
    case, pairs, (Es, Ps, cx_ref) = c1_batch
    E = np.ascontiguousarray(Es[:2])
    P = np.zeros_like(E)
    with case.lattice() as lat:
        status, _, _ = lat.solve_batch(E, P, "bicgstab", "fp64", tol=1e-12)
        cx = lat.cross_sections_batch(E, P)
    assert status == dda.DDA_OK
    assert np.abs(P - Ps[:2]).max() <= 1e-9 * np.abs(Ps[:2]).max()
    assert np.allclose(cx[:, :2], cx_ref[:2], rtol=1e-10, atol=0)


# -------------------------------------------------------------- aggregates

def test_small_aggregate_batch_mixed_vs_lu(dda):
    case = _small_aggregate()
    pairs = _pairs(20260053, 4)
    _, Ps, cx_ref = _oracle_lu(case, pairs)
    with case.lattice() as lat:
        E = _einc(lat, case.nd, pairs)
        P = torch.zeros_like(E)
        status, stats, infos = lat.solve_batch(E, P, "bicgstab", "mixed", tol=1e-6, max_iter=2000)
        cx = lat.cross_sections_batch(E, P)
    assert status == dda.DDA_OK, stats
    for b in range(len(pairs)):
        assert abs(cx[b, 0] / cx_ref[b, 0] - 1) < 1e-5 and abs(cx[b, 1] / cx_ref[b, 1] - 1) < 1e-5, b


def test_aggregate_200_monomers_sampled_rows(dda):
    mask, _ = synth.ballistic_aggregate(20260003 + 200, 200, mono_diameter=8)
    case = Case(mask, [M_AGG], 0.5 / abs(M_AGG))
    pairs = _pairs(20260054, 8)
    rows = synth.rng(55).choice(case.nd, size=12, replace=False)
    with case.lattice() as lat:
        E = _einc(lat, case.nd, pairs)
        P = torch.zeros_like(E)
        status, stats, infos = lat.solve_batch(E, P, "bicgstab", "mixed", tol=1e-5, max_iter=3000)
        assert status == dda.DDA_OK, stats
        AP = torch.empty_like(P)
        lat.matvec_batch(P, AP)
        csca = [lat.scattering_cross_section(P[b]) for b in (0, 5)]
        cx = lat.cross_sections_batch(E, P)
    assert max(i["rel_residual_true"] for i in infos) <= 1e-5
    Ph, APh, Eh = P.cpu().numpy(), AP.cpu().numpy(), E.cpu().numpy()
    for b in (0, 5, 15):
        # the GPU product of the solution equals the direct sum on sampled rows,
        # and there it reproduces the incident field
        ref = odda.direct_matvec_rows(case.coords, case.ainv, case.k, Ph[b], rows)
        assert np.abs(APh[b][:, rows] - ref).max() <= 1e-11 * np.abs(ref).max()
    # optical theorem with the independent pair-sum C_sca, to the solve's accuracy
    for q, b in enumerate((0, 5)):
        assert abs((cx[b, 0] - cx[b, 1]) / csca[q] - 1) < 1e-3


# --------------------------------------------------------------- tiles

@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("shape", [(21, 13, 9), (40, 20, 64)])
def test_tile_widths_do_not_change_results(dda, dtype, shape):
    # padded z lines of 24 (3 * 2^3) and 128 points
    case = random_case(shape, seed=41, fill=0.6)
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    p = torch.from_numpy(synth.complex_normal(42, (2, 3, case.nd))).to(DEV).to(tdt)
    with case.lattice() as lat:
        base = lat.tiles(dtype)
        assert len(base) == 4 and base[3] == 0
        y0 = torch.empty_like(p)
        lat.matvec_batch(p, y0)
        tried = 0
        for d in ((-1, 0, 0, 0), (1, 0, 0, 0), (0, -1, 0, 0), (0, 1, 0, 0), (0, 2, 0, 0), (0, 0, -1, 0),
                  (0, 0, 1, 0), (0, 0, -2, 0), (1, 1, 1, 0)):
            t = tuple(b + e for b, e in zip(base, d))
            try:
                lat.tiles(dtype, t)
            except dda.DDAError as err:
                assert err.code == dda.DDA_ERR_ARG
                continue
            assert lat.tiles(dtype) == t
            y1 = torch.empty_like(p)
            lat.matvec_batch(p, y1)
            assert torch.equal(y0, y1), t
            tried += 1
        assert tried >= 5
        lat.tiles(dtype, base)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_z_pass_widths_in_batched_solves(dda, dtype):
    # one and two whole z columns per CTA of the z pass give the same bits,
    # also while right-hand sides drop out of a batched solve one by one
    case = Case(synth.sphere(24), [1.33 + 0.05j], 0.5 / abs(1.33 + 0.05j))
    pairs = _pairs(20260071, 3)
    precision = "fp64" if dtype == "c128" else "mixed"
    out = []
    with case.lattice() as lat:
        E = _einc(lat, case.nd, pairs)
        base = lat.tiles(dtype)
        for wz in (base[1], base[1] + 1):
            lat.tiles(dtype, (base[0], wz, base[2], 0))
            P = torch.zeros_like(E)
            status, stats, infos = lat.solve_batch(E, P, "bicgstab", precision, tol=1e-9, max_iter=2000)
            assert status == dda.DDA_OK, stats
            out.append((P.clone(), [i["iterations"] for i in infos]))
        lat.tiles(dtype, base)
    for other in out[1:]:
        assert torch.equal(out[0][0], other[0])
    assert out[0][1] == out[1][1]


def test_tile_limits_rejected(dda):
    case = random_case((9, 9, 9), seed=43, fill=0.8)
    with case.lattice() as lat:
        base = lat.tiles("c64")
        with pytest.raises(dda.DDAError) as e:
            lat.tiles("c64", (base[0], 12, base[2], 0))     # 4096 columns x 4 threads per CTA
        assert e.value.code == dda.DDA_ERR_ARG
        assert lat.tiles("c64") == base
        for sched in (-1, 1, 2):                               # the reserved entry must be 0
            with pytest.raises(dda.DDAError) as e:
                lat.tiles("c64", (base[0], base[1], base[2], sched))
            assert e.value.code == dda.DDA_ERR_ARG
        assert lat.tiles("c64") == base


def test_autotune_keeps_results_and_is_remembered(dda):
    case = Case(synth.sphere(40), [1.33 + 0.05j], 0.5 / abs(1.33 + 0.05j))
    p = torch.from_numpy(synth.complex_normal(44, (2, 3, case.nd))).to(DEV).to(torch.complex64)
    with case.lattice() as lat:
        y0 = torch.empty_like(p)
        lat.matvec_batch(p, y0)
        ms = lat.autotune("c64", nb=2, reps=2)
        assert len(ms) == 5 and all(m > 0 for m in ms)
        chosen = lat.tiles("c64")
        y1 = torch.empty_like(p)
        lat.matvec_batch(p, y1)
        assert torch.equal(y0, y1)
    with case.lattice() as lat2:
        assert lat2.tiles("c64") == chosen
