"""Seeded synthetic inputs for the DDA hot path: targets, incidences and vectors.

This module is shared by the tests, the benchmark and the oracle.  It holds no
arithmetic of the method itself (no interaction tensor, no polarisability, no
transform, no solver): only lattice geometries (boolean occupancy masks and
material indices on a K x J x P lattice), incidence directions and random
complex vectors, all drawn from numpy's PCG64 with an explicit seed.

Lattice convention (OpenDDA, Sec. 2 and App. A): site (i, j, k) with
0 <= i < K (x), 0 <= j < J (y), 0 <= k < P (z) has linear index
s = (k * J + j) * K + i, x fastest.  Masks are returned as uint8 arrays of
shape (P, J, K), so ``mask.reshape(-1)[s]`` is site s.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Target", "rng", "sphere", "cube", "ellipsoid", "random_ellipsoid",
    "bernoulli_materials", "ballistic_aggregate", "cube_with_inclusions",
    "crop_center", "complex_normal", "random_direction", "orthogonal_polarisations",
]


def rng(seed: int) -> np.random.Generator:
    """The generator every synthetic input uses: PCG64 seeded explicitly."""
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Target:
    """A target on a K x J x P lattice.

    mask:      uint8 (P, J, K); 1 = occupied site.
    materials: uint8 (P, J, K, 3) or None; material index per site and per
               axis (x, y, z) (Sec. 2: three composition flags per dipole).
               None means a single material (index 0 everywhere).
    refr:      complex refractive index of each material, index = material.
    """
    mask: np.ndarray
    refr: list = field(default_factory=list)
    materials: np.ndarray | None = None
    name: str = ""

    @property
    def shape_kjp(self):
        P, J, K = self.mask.shape
        return (K, J, P)

    @property
    def n_dipoles(self) -> int:
        return int(self.mask.sum())


def _centred_coords(K, J, P):
    """Twice the site-centre offset from the box centre along each axis.

    Site i has centre i + 1/2; the box centre is K/2, so twice the offset is
    2i + 1 - K, an exact integer (this keeps the geometry tests exact).
    """
    x = 2 * np.arange(K, dtype=np.int64) + 1 - K
    y = 2 * np.arange(J, dtype=np.int64) + 1 - J
    z = 2 * np.arange(P, dtype=np.int64) + 1 - P
    return x, y, z


def sphere(n: int, diameter: int | None = None, box: tuple | None = None) -> np.ndarray:
    """Sphere of the given diameter (in lattice spacings) centred in the box.

    A site is occupied when its centre lies inside the sphere:
    (2i+1-K)^2 + (2j+1-J)^2 + (2k+1-P)^2 <= D^2.  With D = K this reproduces
    the occupied-site counts the OpenDDA paper prints for its SPHERE targets
    (18^3 -> 3112, Sec. 4; 200^3 -> 4,188,896, Sec. 6; Table 5).
    """
    K, J, P = box if box is not None else (n, n, n)
    D = n if diameter is None else diameter
    x, y, z = _centred_coords(K, J, P)
    r2 = z[:, None, None] ** 2 + y[None, :, None] ** 2 + x[None, None, :] ** 2
    return (r2 <= D * D).astype(np.uint8)


def cube(n: int) -> np.ndarray:
    """Fully occupied n^3 box (the paper's CUBE target, Table 7)."""
    return np.ones((n, n, n), dtype=np.uint8)


def ellipsoid(box: tuple, semi_axes: tuple) -> np.ndarray:
    """Axis-aligned ellipsoid centred in the box; site centre inside.

    box = (K, J, P); semi_axes = (a, b, c) in lattice spacings along x, y, z.
    """
    K, J, P = box
    a, b, c = semi_axes
    x, y, z = _centred_coords(K, J, P)
    v = ((z[:, None, None] / (2.0 * c)) ** 2 + (y[None, :, None] / (2.0 * b)) ** 2
         + (x[None, None, :] / (2.0 * a)) ** 2)
    return (v <= 1.0).astype(np.uint8)


def random_ellipsoid(seed: int, n: int = 128, lo: float = 0.6, hi: float = 1.0):
    """Ellipsoid with semi-axes drawn uniformly in [lo, hi] * n/2, centred in n^3."""
    g = rng(seed)
    axes = tuple(float(v) for v in g.uniform(lo, hi, size=3) * (n / 2))
    return ellipsoid((n, n, n), axes), axes


def bernoulli_materials(seed: int, mask: np.ndarray, p1: float = 0.3) -> np.ndarray:
    """Per-dipole material index: 1 with probability p1, else 0 (same on all 3 axes)."""
    g = rng(seed)
    m = (g.random(mask.shape) < p1).astype(np.uint8) * mask
    return np.repeat(m[..., None], 3, axis=3)


def ballistic_aggregate(seed: int, n_monomers: int, mono_diameter: int = 8):
    """Ballistic particle-cluster aggregate of touching spheres, voxelised.

    Monomers arrive one at a time along random straight lines (direction
    uniform on the sphere, impact point uniform on a disc covering the
    cluster) and stick at first contact, so every new sphere touches one
    already placed.  The spheres are then voxelised on a lattice whose box
    is the bounding box rounded up to an even size on each axis; a site is
    occupied if its centre lies inside any sphere.  Returns (mask, centres).
    """
    g = rng(seed)
    R = mono_diameter / 2.0
    centres = [np.zeros(3)]
    while len(centres) < n_monomers:
        C = np.array(centres)
        cm = C.mean(axis=0)
        rmax = float(np.max(np.linalg.norm(C - cm, axis=1))) + 2.0 * R
        u = g.normal(size=3)
        u /= np.linalg.norm(u)
        # two unit vectors spanning the disc perpendicular to u
        a = np.cross(u, [1.0, 0.0, 0.0])
        if np.linalg.norm(a) < 1e-6:
            a = np.cross(u, [0.0, 1.0, 0.0])
        a /= np.linalg.norm(a)
        b = np.cross(u, a)
        rad = rmax * math.sqrt(g.random())
        phi = 2.0 * math.pi * g.random()
        start = cm - u * (rmax + 4.0 * R) + a * rad * math.cos(phi) + b * rad * math.sin(phi)
        # first contact along start + t u with any sphere: |start + t u - c| = 2R
        best = None
        for c in C:
            w = start - c
            bq = float(np.dot(w, u))
            cq = float(np.dot(w, w)) - (2.0 * R) ** 2
            disc = bq * bq - cq
            if disc < 0.0:
                continue
            t = -bq - math.sqrt(disc)
            if t > 0.0 and (best is None or t < best):
                best = t
        if best is None:
            continue
        centres.append(start + best * u)
    C = np.array(centres)
    lo = C.min(axis=0) - R
    hi = C.max(axis=0) + R
    dims = np.ceil(hi - lo).astype(int)
    dims = dims + (dims % 2)
    K, J, P = (int(d) for d in dims)
    shift = lo - (dims - (hi - lo)) / 2.0  # centre the aggregate in the box
    x = np.arange(K) + 0.5
    y = np.arange(J) + 0.5
    z = np.arange(P) + 0.5
    mask = np.zeros((P, J, K), dtype=bool)
    for c in C - shift:
        d2 = ((z[:, None, None] - c[2]) ** 2 + (y[None, :, None] - c[1]) ** 2
              + (x[None, None, :] - c[0]) ** 2)
        mask |= d2 <= R * R
    return mask.astype(np.uint8), C - shift


def cube_with_inclusions(seed: int, n: int = 48, rmin: float = 3.0, rmax: float = 6.0,
                         fraction: float = 0.20):
    """n^3 cube host with spherical inclusions (material 1), overlaps allowed.

    Spheres with radius uniform in [rmin, rmax] and centre uniform in the box
    are added until the fraction of sites inside any inclusion reaches
    `fraction`.  Returns (mask, materials) with materials shaped (n, n, n, 3).
    """
    g = rng(seed)
    c = np.arange(n) + 0.5
    inc = np.zeros((n, n, n), dtype=bool)
    while inc.mean() < fraction:
        r = g.uniform(rmin, rmax)
        p = g.uniform(0.0, n, size=3)
        d2 = ((c[:, None, None] - p[2]) ** 2 + (c[None, :, None] - p[1]) ** 2
              + (c[None, None, :] - p[0]) ** 2)
        inc |= d2 <= r * r
    mask = np.ones((n, n, n), dtype=np.uint8)
    mat = np.repeat(inc.astype(np.uint8)[..., None], 3, axis=3)
    return mask, mat


def crop_center(arr: np.ndarray, size: int) -> np.ndarray:
    """Central size^3 sub-box of a (P, J, K[, ...]) array."""
    P, J, K = arr.shape[:3]
    z0, y0, x0 = (P - size) // 2, (J - size) // 2, (K - size) // 2
    return np.ascontiguousarray(arr[z0:z0 + size, y0:y0 + size, x0:x0 + size])


def complex_normal(seed: int, shape, dtype=np.complex128) -> np.ndarray:
    """Circular complex normal CN(0, 1): real and imaginary parts ~ N(0, 1/2)."""
    g = rng(seed)
    v = (g.normal(size=shape) + 1j * g.normal(size=shape)) * math.sqrt(0.5)
    return v.astype(dtype)


def random_direction(seed: int, count: int = 1) -> np.ndarray:
    """`count` unit vectors uniform on the sphere, shape (count, 3)."""
    g = rng(seed)
    v = g.normal(size=(count, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def orthogonal_polarisations(khat: np.ndarray):
    """Two real unit vectors orthogonal to khat and to each other."""
    khat = np.asarray(khat, dtype=np.float64)
    ref = np.array([1.0, 0.0, 0.0]) if abs(khat[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = ref - khat * np.dot(ref, khat)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(khat, e1)
    return e1, e2
