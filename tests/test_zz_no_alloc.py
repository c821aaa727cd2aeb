"""GPU test of dda_occupancy_ranks_static, the rank scan that allocates no
device memory (for callers that cannot call cudaMalloc: code whose device
memory belongs to another framework's pool, or that must not allocate once
it runs).  Its output must equal the ranks the regular path computes inside
dda_init_lattice and reports through dda_site_ranks, on two calls in a row
(two different targets, so the second call cannot reuse the first one's
scratch contents).  Named test_zz_* so it is collected after every other
test file; it builds everything it needs, so it also runs alone.
"""
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


def test_static_rank_scan_matches_context_ranks_twice(dda):
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
        assert total == nd
        assert np.array_equal(words, site_rank[0::32][: words.size])


def test_static_rank_scan_rejects_oversize(dda):
    tiny = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dda.DDAError) as e:
        dda.dda_occupancy_ranks_static(tiny, 4096 * 4096 * 32 + 1, tiny, tiny)
    assert e.value.code == dda.DDA_ERR_ARG
    assert "static scratch limit" in str(e.value)
