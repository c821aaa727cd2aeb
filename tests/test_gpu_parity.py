"""GPU parity of the bit-field kernels, the tensor spectrum and the FFT
matvec against the FP64 oracle (element by element), through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import circulant
from oracle import dda as odda

from _cases import Case, sphere16_case, random_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0908_0863_gb300 as m
    return m


DEV = "cuda"


# ---------------------------------------------------------------- bit fields

@pytest.mark.parametrize("n", [1, 31, 32, 33, 1000, 4096 * 3 + 5])
def test_pack_unpack_occupancy_bit_exact(dda, n):
    g = synth.rng(n)
    mask = (g.random(n) < 0.4).astype(np.uint8)
    md = torch.from_numpy(mask).to(DEV)
    bits = torch.empty((n + 31) // 32, dtype=torch.int32, device=DEV)
    dda.dda_pack_occupancy(md, bits)
    ref = odda.pack_occupancy(mask)
    assert np.array_equal(bits.cpu().numpy().view(np.uint32), ref)
    back = torch.empty(n, dtype=torch.uint8, device=DEV)
    dda.dda_unpack_occupancy(bits, n, back)
    assert np.array_equal(back.cpu().numpy(), mask)


@pytest.mark.parametrize("nmat", [2, 3, 4, 5, 17])
def test_pack_unpack_composition_bit_exact(dda, nmat):
    n = 777
    g = synth.rng(nmat)
    mats = g.integers(0, nmat, size=(n, 3)).astype(np.uint8)
    b = odda.composition_bits(nmat)
    f = 32 // b
    bits = torch.empty((3 * n + f - 1) // f, dtype=torch.int32, device=DEV)
    dda.dda_pack_composition(torch.from_numpy(mats).to(DEV), n, nmat, bits)
    ref = odda.pack_composition(mats, nmat)
    assert np.array_equal(bits.cpu().numpy().view(np.uint32), ref)
    back = torch.empty((n, 3), dtype=torch.uint8, device=DEV)
    dda.dda_unpack_composition(bits, n, nmat, back)
    assert np.array_equal(back.cpu().numpy(), mats)


def test_pack_composition_rejects_out_of_range(dda):
    mats = torch.full((10, 3), 4, dtype=torch.uint8, device=DEV)
    bits = torch.empty(2, dtype=torch.int32, device=DEV)
    with pytest.raises(dda.DDAError) as e:
        dda.dda_pack_composition(mats, 10, 4, bits)
    assert e.value.code == dda.DDA_ERR_ARG


@pytest.mark.parametrize("n,count", [(18, 3112), (200, 4188896)])
def test_sphere_rank_count_matches_paper(dda, golden, n, count):
    # Sec. 4 (18^3) and Sec. 6 (200^3): N_d from the device popcount + scan
    mask = synth.sphere(n)
    md = torch.from_numpy(mask.reshape(-1)).to(DEV)
    bits = torch.empty((mask.size + 31) // 32, dtype=torch.int32, device=DEV)
    dda.dda_pack_occupancy(md, bits)
    alpha = dda.dda_polarizability([1.33 + 0.01j], 0.1, "cmrr")
    with dda.Lattice((n, n, n), bits, alpha, 0.1) as lat:
        assert lat.n_dipoles == count == golden["sphere_occupied_sites"][str(n)]


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 3, 2), (33, 7, 9), (16, 16, 16)])
def test_site_ranks_bit_exact(dda, shape):
    case = random_case(shape, seed=sum(shape), fill=0.6, two_materials=False)
    with case.lattice() as lat:
        r = torch.empty(case.mask.size, dtype=torch.int32, device=DEV)
        lat.site_ranks(r)
        assert np.array_equal(r.cpu().numpy().astype(np.int64), odda.ranks(case.mask))


# ------------------------------------------------------------ tensor spectrum

@pytest.mark.parametrize("shape", [(1, 1, 1), (4, 4, 4), (3, 5, 2), (9, 4, 5), (16, 8, 12), (20, 10, 40)])
def test_tensor_spectrum_matches_oracle(dda, shape):
    K, J, P = shape
    k = 0.7
    case = Case(np.ones((P, J, K), dtype=np.uint8), [1.5 + 0.1j], k)
    L = tuple(circulant.padded_length(v) for v in shape)
    half = circulant.half_spectrum(circulant.tensor_section1(k, K, J, P), L) / (L[0] * L[1] * L[2])
    half = np.ascontiguousarray(half.transpose(2, 3, 1, 0))   # stored as [Hy][Hx][Hz][6]
    with case.lattice() as lat:
        assert lat.padded == L
        out = torch.empty(half.shape, dtype=torch.complex128, device=DEV)
        lat.tensor_spectrum(out)
        got = out.cpu().numpy()
        assert np.abs(got - half).max() <= 1e-13 * np.abs(half).max()
        out32 = torch.empty(half.shape, dtype=torch.complex64, device=DEV)
        lat.tensor_spectrum(out32)
        assert np.abs(out32.cpu().numpy() - half).max() <= 1e-6 * np.abs(half).max()


# ------------------------------------------------------------------- matvec

def _matvec(dda, case, p, dtype):
    with case.lattice() as lat:
        pd = torch.from_numpy(p.astype(dtype)).to(DEV)
        yd = torch.full_like(pd, float("nan"))
        lat.matvec(pd, yd)
        torch.cuda.synchronize()
        return yd.cpu().numpy().astype(np.complex128)


SHAPES = [((1, 1, 1), 1.0), ((2, 3, 5), 1.0), ((5, 4, 3), 0.5), ((7, 3, 6), 0.55), ((12, 5, 4), 1.0),
          ((16, 16, 16), 0.7), ((24, 20, 17), 0.8), ((40, 9, 33), 0.6)]


@pytest.mark.parametrize("shape,fill", SHAPES)
def test_matvec_c128_matches_direct_sum(dda, shape, fill):
    case = random_case(shape, seed=7 * sum(shape), fill=fill)
    p = synth.complex_normal(3, (3, case.nd))
    y_ref = odda.direct_matvec(case.coords, case.ainv, case.k, p)
    y = _matvec(dda, case, p, np.complex128)
    assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()


@pytest.mark.parametrize("shape,fill", SHAPES)
def test_matvec_c64_matches_direct_sum(dda, shape, fill):
    case = random_case(shape, seed=7 * sum(shape), fill=fill)
    p = synth.complex_normal(3, (3, case.nd))
    y_ref = odda.direct_matvec(case.coords, case.ainv, case.k, p.astype(np.complex64))
    y = _matvec(dda, case, p, np.complex64)
    # complex64 FFTs of length L: error ~ eps32 * log2 L relative to the largest term
    assert np.abs(y - y_ref).max() <= 2e-6 * np.abs(y_ref).max()


def _matvec_df(dda, case, p):
    # double-float products of complex128 vectors
    with case.lattice() as lat:
        pd = torch.from_numpy(p.astype(np.complex128)).to(DEV)
        yd = torch.full_like(pd, float("nan"))
        dda.dda_matvec(lat.ctx, pd, yd, dtype="c128df")
        torch.cuda.synchronize()
        return yd.cpu().numpy()


@pytest.mark.parametrize("shape,fill", SHAPES)
def test_matvec_double_float_matches_direct_sum(dda, shape, fill):
    # about 48 significant bits per operation: a few 1e-14 after the
    # transforms, against 1e-15 for FP64 and 1e-7 for complex64
    case = random_case(shape, seed=7 * sum(shape), fill=fill)
    p = synth.complex_normal(3, (3, case.nd))
    y_ref = odda.direct_matvec(case.coords, case.ainv, case.k, p)
    y = _matvec_df(dda, case, p)
    assert np.abs(y - y_ref).max() <= 1e-11 * np.abs(y_ref).max()


@pytest.mark.parametrize("box", [(48, 40, 33), (80, 6, 5), (5, 96, 6), (6, 5, 160)])
def test_matvec_double_float_odd_lengths_and_batches(dda, box):
    # 3 * 2^a and 5 * 2^a lines on each axis (96, 80, 192, 320 points), a
    # batch of two right-hand sides equal to two single products
    case = random_case(box, seed=sum(box) + 1, fill=0.6)
    p = synth.complex_normal(4, (2, 3, case.nd))
    rows = synth.rng(5).choice(case.nd, size=min(case.nd, 48), replace=False)
    ref = odda.direct_matvec_rows(case.coords, case.ainv, case.k, p[1], rows)
    with case.lattice() as lat:
        pd = torch.from_numpy(p).to(DEV)
        yb = torch.full_like(pd, float("nan"))
        dda.dda_matvec_batch(lat.ctx, pd, yb, dtype="c128df")
        y1 = torch.full_like(pd[1], float("nan"))
        dda.dda_matvec(lat.ctx, pd[1].contiguous(), y1, dtype="c128df")
        torch.cuda.synchronize()
        yb, y1 = yb.cpu().numpy(), y1.cpu().numpy()
    assert np.array_equal(yb[1], y1)
    assert np.abs(y1[:, rows] - ref).max() <= 1e-11 * np.abs(ref).max()


def test_matvec_double_float_rejects_complex64(dda):
    case = random_case((4, 4, 4), seed=3)
    with case.lattice() as lat:
        p = torch.zeros((3, case.nd), dtype=torch.complex64, device=DEV)
        with pytest.raises(TypeError):
            dda.dda_matvec(lat.ctx, p, torch.empty_like(p), dtype="c128df")


def test_matvec_sphere16(dda):
    case = sphere16_case()
    p = synth.complex_normal(1, (3, case.nd))
    y_ref = odda.direct_matvec(case.coords, case.ainv, case.k, p)
    y = _matvec(dda, case, p, np.complex128)
    assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()


def test_matvec_ellipsoid_crop_two_materials(dda):
    # 128^3 ellipsoid (semi-axes U(0.6, 1) x 64), Bernoulli(0.3) second material,
    # LDR; the oracle runs on the central 24^3 crop
    mask, axes = synth.random_ellipsoid(20260002, 128)
    mats = synth.bernoulli_materials(20260003, mask, 0.3)
    mask_c, mats_c = synth.crop_center(mask, 24), synth.crop_center(mats, 24)
    k = 0.8 / abs(1.7 + 0.1j)
    case = Case(mask_c, [1.5 + 0.01j, 1.7 + 0.1j], k, mats_c, rule="ldr")
    p = synth.complex_normal(20260004, (3, case.nd))
    y_ref = odda.direct_matvec(case.coords, case.ainv, case.k, p)
    y = _matvec(dda, case, p, np.complex128)
    assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    y32 = _matvec(dda, case, p, np.complex64)
    assert np.abs(y32 - y_ref).max() <= 2e-6 * np.abs(y_ref).max()


@pytest.mark.parametrize("n,D", [(128, 128), (256, 250)])
def test_matvec_full_size_sampled_rows(dda, n, D):
    # full-size lattices in the benchmark's launch configuration; the oracle
    # computes 24 sampled outputs one by one (direct sums over all dipoles)
    m = 1.33 + 0.05j
    k = 0.5 / abs(m)
    mask = synth.sphere(D, box=(n, n, n))
    case = Case(mask, [m], k)
    p = synth.complex_normal(5, (3, case.nd))
    rows = synth.rng(9).choice(case.nd, size=24, replace=False)
    ref = odda.direct_matvec_rows(case.coords, case.ainv, case.k, p, rows)
    y = _matvec(dda, case, p, np.complex128)[:, rows]
    scale = np.abs(ref).max()
    assert np.abs(y - ref).max() <= 1e-11 * scale
    y32 = _matvec(dda, case, p, np.complex64)[:, rows]
    assert np.abs(y32 - ref).max() <= 5e-6 * scale


@pytest.mark.parametrize("box,D", [((96, 96, 96), 96), ((192, 160, 100), 100)])
def test_matvec_odd_radix_lengths_sampled_rows(dda, box, D):
    # lattices whose circulant lengths are 3 * 2^a or 5 * 2^a (192 = 3 * 64 on
    # all axes; 384, 320, 256): the radix-3 and radix-5 closing stages in
    # every pass and in the spectrum build, against 24 direct sums
    m = 1.33 + 0.05j
    k = 0.5 / abs(m)
    mask = synth.sphere(D, box=box)
    case = Case(mask, [m], k)
    assert case.shape == box
    p = synth.complex_normal(6, (3, case.nd))
    rows = synth.rng(10).choice(case.nd, size=24, replace=False)
    ref = odda.direct_matvec_rows(case.coords, case.ainv, case.k, p, rows)
    with case.lattice() as lat:
        assert lat.padded == tuple(circulant.padded_length(v) for v in box)
        assert any(v % 3 == 0 or v % 5 == 0 for v in lat.padded)
    y = _matvec(dda, case, p, np.complex128)[:, rows]
    scale = np.abs(ref).max()
    assert np.abs(y - ref).max() <= 1e-11 * scale
    y32 = _matvec(dda, case, p, np.complex64)[:, rows]
    assert np.abs(y32 - ref).max() <= 5e-6 * scale


ODD_LENGTHS = [24, 48, 96, 192, 384, 768, 40, 80, 160, 320, 640]


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("L", ODD_LENGTHS)
def test_matvec_every_odd_length(dda, L, axis):
    # every 3 * 2^a and 5 * 2^a circulant length on each axis (an edge of L/2
    # sites pads to L), the other two axes short and ragged: the wide thread
    # mapping of those lines in each pass, every output against the direct sum
    box = [3, 4, 5]
    box[axis] = L // 2
    case = random_case(tuple(box), seed=L + 7 * axis, fill=0.6)
    with case.lattice() as lat:
        assert lat.padded[axis] == L
    p = synth.complex_normal(L + axis, (3, case.nd))
    y_ref = odda.direct_matvec(case.coords, case.ainv, case.k, p)
    y = _matvec(dda, case, p, np.complex128)
    assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    y_ref32 = odda.direct_matvec(case.coords, case.ainv, case.k, p.astype(np.complex64))
    y32 = _matvec(dda, case, p, np.complex64)
    assert np.abs(y32 - y_ref32).max() <= 2e-6 * np.abs(y_ref32).max()


@pytest.mark.parametrize("box", [(512, 6, 5), (5, 512, 6), (6, 5, 512)])
def test_matvec_longest_lines(dda, box):
    # a 512-site edge (the largest the library takes) gives 1024-point lines:
    # along x through P2/P4, along y through P1/P5, along z through P3, with
    # the other two axes short and ragged; every output against the direct sum
    case = random_case(box, seed=sum(box), fill=0.5)
    with case.lattice() as lat:
        assert max(lat.padded) == 1024
    p = synth.complex_normal(11, (3, case.nd))
    rows = synth.rng(12).choice(case.nd, size=64, replace=False)
    ref = odda.direct_matvec_rows(case.coords, case.ainv, case.k, p, rows)
    y = _matvec(dda, case, p, np.complex128)[:, rows]
    assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max()
    y32 = _matvec(dda, case, p, np.complex64)[:, rows]
    assert np.abs(y32 - ref).max() <= 5e-6 * np.abs(ref).max()


def test_matvec_rejects_host_and_aliased(dda):
    case = random_case((4, 4, 4), seed=1, two_materials=False)
    with case.lattice() as lat:
        pd = torch.zeros((3, case.nd), dtype=torch.complex128, device=DEV)
        with pytest.raises(dda.DDAError):
            lat.matvec(pd.cpu(), pd)
        with pytest.raises(dda.DDAError):
            lat.matvec(pd, pd)
