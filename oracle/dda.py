"""Plain FP64 oracle of the DDA problem (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg use this package; the CUDA product path never imports it.

What is here, each a direct statement of the definition it follows:

* bit-fielded occupancy / composition and the compressed ordering
  (OpenDDA Sec. 2; site index s = (k J + j) K + i of App. A; zero-storage
  vectors of Sec. 4),
* polarisabilities: Clausius-Mossotti, radiative reaction (Draine 1988) and
  the lattice dispersion relation (Draine & Goodman 1993), which the paper
  cites in Sec. 1 without formulas,
* the incident plane wave at the dipoles,
* the interaction matrix of Eq. 1 (direct O(N^2) sums in ``direct.c``),
* C_ext, C_abs and two independent C_sca (exact double sum, far-field
  quadrature), following the cross-section formulas of Draine 1988 and
  Draine & Flatau 1994 (the paper prints only their values, Table 7).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _native

# ---------------------------------------------------------------- bit fields

def composition_bits(n_materials: int) -> int:
    """Bits per composition field: enough for indices 0..n_mat-1, at least 1.

    Sec. 2: four materials 0..3 need two bits (mask 3 = 0b11).
    """
    return max(1, (n_materials - 1).bit_length())


def pack_occupancy(mask: np.ndarray) -> np.ndarray:
    """Occupancy flags -> uint32 words, one bit per site (Sec. 2).

    Layout: site s sits in word s // 32 at bit s % 32 (least significant
    first), s = (k J + j) K + i.  Padding bits of the last word are zero.
    (numpy's packbits with little bit order puts site s at bit s % 8 of
    byte s // 8; four little-endian bytes make one word.)
    """
    flat = np.asarray(mask).reshape(-1).astype(bool)
    n = flat.size
    nbytes = 4 * ((n + 31) // 32)
    b = np.zeros(nbytes, dtype=np.uint8)
    packed = np.packbits(flat, bitorder="little")
    b[:packed.size] = packed
    return b.view("<u4").astype(np.uint32)


def unpack_occupancy(words: np.ndarray, n_sites: int) -> np.ndarray:
    """Inverse of pack_occupancy: bit s % 32 of word s // 32 for every site."""
    s = np.arange(n_sites, dtype=np.int64)
    w = np.asarray(words, dtype=np.uint32).astype(np.int64)
    return ((w[s >> 5] >> (s & 31)) & 1).astype(np.uint8)


def pack_composition(materials: np.ndarray, n_materials: int) -> np.ndarray:
    """Material index per site and axis -> b-bit fields in uint32 words (Sec. 2).

    materials: (P, J, K, 3) integers.  Field q = 3 s + axis holds the
    material of site s along axis (0 = x, 1 = y, 2 = z).  Each word holds
    floor(32 / b) whole fields (no field straddles two words), field q at
    word q // f, bit offset (q % f) * b.
    """
    b = composition_bits(n_materials)
    f = 32 // b
    vals = np.asarray(materials).reshape(-1).astype(np.uint64)
    if vals.size and int(vals.max()) >= n_materials:
        raise ValueError("material index out of range")
    q = np.arange(vals.size, dtype=np.int64)
    words = np.zeros((vals.size + f - 1) // f, dtype=np.uint64)
    # fields of one word occupy disjoint bits, so adding them is OR-ing them
    np.add.at(words, q // f, vals << ((q % f) * b).astype(np.uint64))
    return words.astype(np.uint32)


def unpack_composition(words: np.ndarray, n_sites: int, n_materials: int) -> np.ndarray:
    """Inverse of pack_composition -> (n_sites, 3) material indices."""
    b = composition_bits(n_materials)
    f = 32 // b
    msk = (1 << b) - 1
    q = np.arange(3 * n_sites, dtype=np.int64)
    w = np.asarray(words, dtype=np.uint32).astype(np.int64)
    return ((w[q // f] >> ((q % f) * b)) & msk).reshape(n_sites, 3)


def bitfield_bytes(n_sites: int, n_materials: int) -> int:
    """Bytes of the packed occupancy plus composition words for a lattice."""
    occ = 4 * ((n_sites + 31) // 32)
    if n_materials <= 1:
        return occ
    f = 32 // composition_bits(n_materials)
    return occ + 4 * ((3 * n_sites + f - 1) // f)


def occupied_sites(mask: np.ndarray) -> np.ndarray:
    """Linear indices s of the occupied sites in increasing order.

    This order is the compressed ordering of the solver vectors (Sec. 4):
    entry n of a compressed vector belongs to the n-th occupied site.
    """
    return np.nonzero(np.asarray(mask).reshape(-1))[0]


def ranks(mask: np.ndarray) -> np.ndarray:
    """rank[s] = number of occupied sites before s (compressed index of s)."""
    flat = np.asarray(mask).reshape(-1).astype(np.int64)
    return np.cumsum(flat) - flat


def coords_of(mask: np.ndarray) -> np.ndarray:
    """Integer (x, y, z) = (i, j, k) of the occupied sites, shape (N_d, 3) int32."""
    P, J, K = np.asarray(mask).shape
    s = occupied_sites(mask)
    i = s % K
    j = (s // K) % J
    k = s // (K * J)
    return np.stack([i, j, k], axis=1).astype(np.int32)


# ---------------------------------------------------------- polarisabilities

LDR_B1 = -1.8915316
LDR_B2 = 0.1648469
LDR_B3 = -1.7700004


def alpha_cm(m: complex) -> complex:
    """Clausius-Mossotti polarisability per unit cell volume (d = 1)."""
    eps = complex(m) ** 2
    return 3.0 / (4.0 * math.pi) * (eps - 1.0) / (eps + 2.0)


def alpha_rr(m: complex, k: float) -> complex:
    """CM with the radiative-reaction correction (Draine 1988)."""
    a = alpha_cm(m)
    return a / (1.0 - (2.0 / 3.0) * 1j * k ** 3 * a)


def alpha_ldr(m: complex, k: float, khat, e0) -> complex:
    """Lattice dispersion relation polarisability (Draine & Goodman 1993).

    alpha = alpha_CM / (1 + alpha_CM [(b1 + m^2 b2 + m^2 b3 S) k^2 - (2/3) i k^3]),
    S = sum_a (khat_a e_a)^2 for unit propagation khat and polarisation e.
    """
    a = alpha_cm(m)
    m2 = complex(m) ** 2
    e0 = np.asarray(e0, dtype=np.complex128)
    S = complex(np.sum((np.asarray(khat, dtype=np.float64) * e0) ** 2)).real
    return a / (1.0 + a * ((LDR_B1 + m2 * LDR_B2 + m2 * LDR_B3 * S) * k ** 2
                           - (2.0 / 3.0) * 1j * k ** 3))


def alpha_inverse_per_dipole(alpha_table: np.ndarray, materials_flat: np.ndarray | None,
                             n_dipoles: int, mask: np.ndarray | None = None) -> np.ndarray:
    """alpha^{-1} for each occupied dipole and axis, shape (N_d, 3) complex.

    alpha_table: (n_mat, 3) complex, polarisability of material q along axis c.
    materials_flat: (N_sites, 3) material per site and axis, or None (all 0).
    """
    alpha_table = np.asarray(alpha_table, dtype=np.complex128).reshape(-1, 3)
    if materials_flat is None:
        return np.tile(1.0 / alpha_table[0], (n_dipoles, 1))
    occ = occupied_sites(mask)
    mats = np.asarray(materials_flat).reshape(-1, 3)[occ]
    out = np.empty((n_dipoles, 3), dtype=np.complex128)
    for c in range(3):
        out[:, c] = 1.0 / alpha_table[mats[:, c], c]
    return out


# ------------------------------------------------------------ incident field

def incident_field(coords: np.ndarray, k: float, khat, e0) -> np.ndarray:
    """E_inc at each dipole: e0 exp(i k khat . r_j), r_j = (i, j, k) lattice
    coordinates (phase origin at site (0, 0, 0)).  Returns [3][N_d] complex."""
    khat = np.asarray(khat, dtype=np.float64)
    e0 = np.asarray(e0, dtype=np.complex128)
    phase = np.exp(1j * k * (coords.astype(np.float64) @ khat))
    return e0[:, None] * phase[None, :]


# ------------------------------------------------------------ matrix-vector

def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def interaction_tensor(k: float, r) -> np.ndarray:
    """The six components (xx, xy, xz, yy, yz, zz) of A_jl at displacement r != 0."""
    out = np.zeros(12)
    _native.lib().oracle_interaction_tensor(float(k), float(r[0]), float(r[1]), float(r[2]), _dp(out))
    return out[0::2] + 1j * out[1::2]


def direct_matvec(coords: np.ndarray, ainv: np.ndarray, k: float, p: np.ndarray,
                  nthreads: int = 0) -> np.ndarray:
    """y = A p by direct summation over all dipole pairs (Eq. 1).

    coords (N_d, 3) int; ainv (N_d, 3) complex; p [3][N_d] complex.
    nthreads = 0 uses the OpenMP default.
    """
    n = coords.shape[0]
    c = np.ascontiguousarray(coords, dtype=np.int32)
    a = np.ascontiguousarray(ainv, dtype=np.complex128)
    pv = np.ascontiguousarray(np.asarray(p, dtype=np.complex128).reshape(3, n))
    y = np.empty((3, n), dtype=np.complex128)
    _native.lib().oracle_direct_matvec(n, _ip(c), _dp(a), float(k), _dp(pv), _dp(y), int(nthreads))
    return y


def direct_matvec_rows(coords: np.ndarray, ainv: np.ndarray, k: float, p: np.ndarray, rows,
                       nthreads: int = 0) -> np.ndarray:
    """(A p) at the given dipoles only, each by its own direct sum; [3][len(rows)]."""
    n = coords.shape[0]
    c = np.ascontiguousarray(coords, dtype=np.int32)
    a = np.ascontiguousarray(ainv, dtype=np.complex128)
    pv = np.ascontiguousarray(np.asarray(p, dtype=np.complex128).reshape(3, n))
    rr = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.empty((3, rr.size), dtype=np.complex128)
    _native.lib().oracle_direct_matvec_rows(n, _ip(c), _dp(a), float(k), _dp(pv),
                                            rr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), rr.size,
                                            _dp(out), int(nthreads))
    return out


def dense_matrix(coords: np.ndarray, ainv: np.ndarray, k: float) -> np.ndarray:
    """Dense 3N_d x 3N_d matrix of Eq. 1, unknowns ordered [3][N_d]."""
    n = coords.shape[0]
    c = np.ascontiguousarray(coords, dtype=np.int32)
    a = np.ascontiguousarray(ainv, dtype=np.complex128)
    A = np.empty((3 * n, 3 * n), dtype=np.complex128)
    _native.lib().oracle_dense_matrix(n, _ip(c), _dp(a), float(k), _dp(A))
    return A


# ------------------------------------------------------------ cross sections

def c_ext(einc: np.ndarray, P: np.ndarray, k: float, e0_norm2: float = 1.0) -> float:
    """C_ext = (4 pi k / |E0|^2) sum_j Im(E_inc,j^* . P_j)."""
    return 4.0 * math.pi * k * float(np.sum(np.imag(np.conj(einc) * P))) / e0_norm2


def c_abs(ainv: np.ndarray, P: np.ndarray, k: float, e0_norm2: float = 1.0) -> float:
    """C_abs = (4 pi k / |E0|^2) sum_j sum_c [-Im(alpha^{-1}_jc) - (2/3) k^3] |P_jc|^2."""
    w = -np.imag(np.asarray(ainv).T) - (2.0 / 3.0) * k ** 3
    return 4.0 * math.pi * k * float(np.sum(w * np.abs(P) ** 2)) / e0_norm2


def c_sca_double_sum(coords: np.ndarray, P: np.ndarray, k: float, nthreads: int = 0) -> float:
    """C_sca from the exact pair sum of the radiated power (see direct.c)."""
    n = coords.shape[0]
    c = np.ascontiguousarray(coords, dtype=np.int32)
    pv = np.ascontiguousarray(np.asarray(P, dtype=np.complex128).reshape(3, n))
    return float(_native.lib().oracle_csca_double_sum(n, _ip(c), float(k), _dp(pv), int(nthreads)))


def c_sca_far_field(coords: np.ndarray, P: np.ndarray, k: float, n_theta: int = 48,
                    n_phi: int = 96) -> float:
    """C_sca = k^4 \\oint |sum_j (P_j - n (n . P_j)) exp(-i k n . r_j)|^2 dOmega.

    Gauss-Legendre in cos(theta) times the uniform rule in phi (exact for
    the trigonometric polynomials in phi below degree n_phi).
    """
    mu, wmu = np.polynomial.legendre.leggauss(n_theta)
    phi = 2.0 * math.pi * np.arange(n_phi) / n_phi
    wphi = 2.0 * math.pi / n_phi
    st = np.sqrt(1.0 - mu ** 2)
    nvec = np.stack([np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)),
                     np.outer(mu, np.ones(n_phi))], axis=-1).reshape(-1, 3)
    w = np.outer(wmu, np.full(n_phi, wphi)).reshape(-1)
    r = coords.astype(np.float64)
    total = 0.0
    for a in range(0, nvec.shape[0], 256):
        nv = nvec[a:a + 256]
        ph = np.exp(-1j * k * (nv @ r.T))            # (dirs, N_d)
        F = ph @ np.asarray(P).T                      # (dirs, 3): sum_j P_j e^{-ik n.r_j}
        Ft = F - nv * np.sum(nv * F, axis=1, keepdims=True)
        total += float(np.sum(w[a:a + 256] * np.sum(np.abs(Ft) ** 2, axis=1)))
    return k ** 4 * total


def a_eff(n_dipoles: int) -> float:
    """Radius of the sphere of equal volume, in lattice spacings: (3 N_d / 4 pi)^(1/3)."""
    return (3.0 * n_dipoles / (4.0 * math.pi)) ** (1.0 / 3.0)


def efficiencies(C, n_dipoles: int):
    """Q = C / (pi a_eff^2) for each cross section in C."""
    g = math.pi * a_eff(n_dipoles) ** 2
    return [c / g for c in C]
