"""Shared set-up of the GPU parity tests: a target, its oracle description
and its CUDA context, built from the same seeded synthetic input."""
from __future__ import annotations

import numpy as np

import synth
from oracle import dda as odda


class Case:
    """mask (P, J, K), optional materials (P, J, K, 3), refractive indices."""

    def __init__(self, mask, refr, k, materials=None, rule="cmrr", khat=(0, 0, 1), e0=(1, 0, 0)):
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8)
        P, J, K = self.mask.shape
        self.shape = (K, J, P)
        self.refr = list(refr)
        self.nmat = len(self.refr)
        self.k = float(k)
        self.materials = materials
        self.khat, self.e0 = khat, e0
        # oracle side: polarisabilities straight from the literature formulas
        if rule == "cmrr":
            al = [odda.alpha_rr(m, k) for m in self.refr]
        elif rule == "ldr":
            al = [odda.alpha_ldr(m, k, khat, e0) for m in self.refr]
        else:
            al = [odda.alpha_cm(m) for m in self.refr]
        self.alpha = np.array([[a] * 3 for a in al], dtype=np.complex128)
        self.coords = odda.coords_of(self.mask)
        self.nd = self.coords.shape[0]
        mflat = None if materials is None else np.asarray(materials).reshape(-1, 3)
        self.ainv = odda.alpha_inverse_per_dipole(self.alpha, mflat, self.nd, self.mask)
        self.occ_bits = odda.pack_occupancy(self.mask)
        self.comp_bits = None if materials is None else odda.pack_composition(materials, self.nmat)

    def lattice(self):
        import paper_0908_0863_gb300 as dda
        return dda.Lattice(self.shape, self.occ_bits, self.alpha, self.k, self.comp_bits, self.nmat)


def random_case(shape, seed, fill=1.0, two_materials=True, k=0.45):
    K, J, P = shape
    g = synth.rng(seed)
    mask = (g.random((P, J, K)) < fill).astype(np.uint8)
    mask.reshape(-1)[0] = 1
    mats = None
    refr = [1.5 + 0.01j]
    if two_materials:
        mats = synth.bernoulli_materials(seed + 1, mask, 0.3)
        refr = [1.5 + 0.01j, 1.7 + 0.1j]
    return Case(mask, refr, k, mats)


def sphere16_case():
    """16^3 sphere of diameter 16, m = 1.33 + 0.01i, |m| k d = 0.5, CM + RR."""
    m = 1.33 + 0.01j
    return Case(synth.sphere(16), [m], 0.5 / abs(m))
