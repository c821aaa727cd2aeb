"""The benchmark's same-GPU comparison arm (unpruned 3-D FFTs through
torch.fft) computes the same product y = A p as the oracle's direct sum
(Eq. 1) and as the library, so that its timing compares like with like.

The arm is measurement infrastructure, not the product path."""
import numpy as np
import pytest
import torch

import bench
import synth
from oracle import dda as odda


def _target(shape, seed):
    K, J, P = shape
    g = synth.rng(seed)
    mask = synth.ellipsoid(shape, (0.55 * K, 0.5 * J, 0.6 * P)).astype(bool)
    mask &= g.random(mask.shape) < 0.85          # hollow sites
    return mask


def test_unpruned_arm_equals_direct_sum():
    # non-cubic box, holes, RR polarisability: the arm against the oracle
    k = 0.7
    mask = _target((7, 5, 6), 11)
    nd = int(mask.sum())
    ainv = 1.0 / odda.alpha_rr(1.5 + 0.1j, k)
    p = synth.complex_normal(12, (3, nd))
    want = odda.direct_matvec(odda.coords_of(mask), np.full((nd, 3), ainv), k, p)
    arm = bench.UnprunedFFT(torch, torch.device("cpu"), mask, np.full((3, 1), ainv), k, torch.complex128)
    got = arm.matvec(torch.from_numpy(p)).numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12


@pytest.mark.gpu
def test_unpruned_arm_equals_library():
    import paper_0908_0863_gb300 as dda
    k = 0.45
    shape = (40, 36, 28)
    mask = _target(shape, 21)
    nd = int(mask.sum())
    alpha = dda.dda_polarizability([1.33 + 0.05j], k, "cmrr")
    dev = torch.device("cuda")
    ainv = torch.full((3, 1), 1.0 / complex(alpha[0, 0]), dtype=torch.complex128)
    with dda.Lattice(shape, odda.pack_occupancy(mask), alpha, k) as lat:
        for dtype, tol in ((torch.complex128, 1e-12), (torch.complex64, 2e-5)):
            arm = bench.UnprunedFFT(torch, dev, mask, ainv, k, dtype)
            p = torch.from_numpy(synth.complex_normal(22, (3, nd))).to(dtype).to(dev)
            y = torch.empty_like(p)
            lat.matvec(p, y)
            z = arm.matvec(p)
            assert float((z - y).norm() / y.norm()) < tol
