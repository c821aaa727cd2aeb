"""GPU test of dda_occupancy_ranks_static, the rank scan that allocates no
device memory (for callers that cannot call cudaMalloc: code whose device
memory belongs to another framework's pool, or that must not allocate once
it runs).  Its output must equal the oracle's ranks (the plain prefix count
of the occupancy mask) and the ranks the regular path computes inside
dda_init_lattice and reports through dda_site_ranks, on two calls in a row
(two different targets, so the second call cannot reuse the first one's
scratch contents).  A third case has more than 1024 scan blocks, so the
block-total pass loops more than once.  Named test_zz_* so it is collected
after every other test file; it builds everything it needs, so it also runs
alone.
"""
import numpy as np
import pytest

import synth
from oracle import dda as odda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCAN_TILE_WORDS = 4096          # words per scan block
LIMIT_SITES = 4096 * SCAN_TILE_WORDS * 32


@pytest.fixture(scope="module")
def dda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0908_0863_gb300 as m
    return m


def _regular_ranks(dda, mask):
    """Per-site ranks and N_d from the existing entry points (context path)."""
    P, J, K = mask.shape
    bits = odda.pack_occupancy(mask)
    alpha = dda.dda_polarizability([1.5 + 0.1j], 0.3, "cmrr")
    with dda.Lattice((K, J, P), bits, alpha, 0.3) as lat:
        r = torch.empty(mask.size, dtype=torch.int32, device="cuda")
        lat.site_ranks(r)
        torch.cuda.synchronize()
        return r.cpu().numpy().view(np.uint32), lat.n_dipoles, bits


def _static_ranks(dda, bits, n_sites):
    dbits = torch.from_numpy(bits.view(np.int32)).cuda()
    words = torch.full(((n_sites + 31) // 32,), -1, dtype=torch.int32, device="cuda")
    total = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    dda.dda_occupancy_ranks_static(dbits, n_sites, words, total)
    torch.cuda.synchronize()
    return words.cpu().numpy().view(np.uint32), int(total.cpu().numpy().view(np.uint32)[0])


def test_static_rank_scan_matches_oracle_and_context_twice(dda):
    # two different targets in a row; padding bits set on purpose in the
    # second so the scan has to ignore them
    targets = [synth.sphere(37, box=(41, 29, 39)), (synth.rng(5).random((64, 50, 70)) < 0.37).astype(np.uint8)]
    for mask in targets:
        site_rank, nd, bits = _regular_ranks(dda, mask)
        n = mask.size
        if n % 32:
            bits = bits.copy()
            bits[-1] |= np.uint32(~((1 << (n % 32)) - 1) & 0xFFFFFFFF)
        words, total = _static_ranks(dda, bits, n)
        # against the oracle: the prefix count of the mask at each word start
        assert total == int(np.count_nonzero(mask)) == odda.occupied_sites(mask).size
        assert np.array_equal(words.astype(np.int64), odda.ranks(mask)[0::32])
        # against the regular (allocating) path
        assert total == nd
        assert np.array_equal(words, site_rank[0::32][: words.size])


def test_static_rank_scan_many_blocks(dda):
    """More than 1024 scan blocks (1100 blocks of 4096 words, 144,179,200
    sites minus a ragged tail), so the block totals are scanned in two
    rounds.  The field repeats one seeded period of 97 words; the expected
    ranks follow from the oracle's prefix count over one period:
    rank(w) = (w // 97) * (sites per period) + rank within the period."""
    period = 97
    nwords = 1100 * SCAN_TILE_WORDS
    n_sites = nwords * 32 - 13                      # ragged last word
    pmask = (synth.rng(77).random(period * 32) < 0.41).astype(np.uint8)
    pwords = odda.pack_occupancy(pmask)
    reps = -(-nwords // period)
    bits = np.tile(pwords, reps)[:nwords].copy()
    bits[-1] |= np.uint32(0xFFFFFFFF ^ ((1 << 19) - 1))   # padding bits past n_sites set
    pr = odda.ranks(pmask)[0::32]                   # rank at each word start of the period
    per = int(np.count_nonzero(pmask))
    w = np.arange(nwords, dtype=np.int64)
    expect = (w // period) * per + pr[w % period]
    last_word_mask = pmask.reshape(period, 32)[(nwords - 1) % period][:19]
    expect_total = int(expect[-1]) + int(np.count_nonzero(last_word_mask))
    assert expect_total < 2 ** 32
    words, total = _static_ranks(dda, bits, n_sites)
    assert total == expect_total
    assert np.array_equal(words.astype(np.int64), expect)


def test_static_rank_scan_rejects_oversize(dda):
    tiny = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dda.DDAError) as e:
        dda.dda_occupancy_ranks_static(tiny, LIMIT_SITES + 1, tiny, tiny)
    assert e.value.code == dda.DDA_ERR_ARG
    assert "static scratch limit" in str(e.value)


def test_static_rank_scan_rejects_host_buffers(dda):
    """Host memory passed where device memory is expected is refused on
    the host before anything is queued."""
    dev = torch.zeros(4, dtype=torch.int32, device="cuda")
    host = np.zeros(4, dtype=np.int32)
    for args in ((host, dev, dev), (dev, host, dev), (dev, dev, host)):
        with pytest.raises(dda.DDAError) as e:
            dda.dda_occupancy_ranks_static(args[0], 100, args[1], args[2])
        assert e.value.code == dda.DDA_ERR_ARG
        assert "device pointers" in str(e.value)
    torch.cuda.synchronize()
