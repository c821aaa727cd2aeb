"""Circulant-embedding form of the DDA matvec, written plainly with numpy FFTs.

Test infrastructure only.  The direct sum of ``dda.direct_matvec`` is the
definition; this module restates the two FFT formulations of the paper so
the tests can pin the readings the GPU path relies on:

* ``first_column``/``fft_matvec``: the standard algorithm (App. A, after
  Goodman et al. 1991): each of the six tensor components is embedded in a
  level-three circulant whose first column holds the Toeplitz values at all
  displacements, the vectors are zero-padded, and the product is
  iDFT(DFT(c) . DFT(x)) per Eqs. 6-8, cropped to the original octant.
* ``half_spectrum``: the paper's fused T-to-c conversion and 1D DFTs
  (Sec. 3): every line of section 1 is mirrored with the sign of Table 1,
  transformed, and only the first L/2 + 1 outputs are kept, in the order
  x, then y, then z.
* ``mirror_signs``: Table 1 of the paper.

The padded lengths L are passed in.  ``padded_length`` gives the length
the library pads each axis to: the smallest L >= 2n - 1 of the form 2^a,
3 * 2^a or 5 * 2^a (the paper's K'' = 2K - 1 + kf with kf chosen for a fast
transform, Sec. 3 and App. A).  Any L >= 2n - 1 gives the same product.
"""
from __future__ import annotations

import numpy as np

from . import dda

COMPONENTS = ("xx", "xy", "xz", "yy", "yz", "zz")
# component m -> (row axis, column axis)
AXES = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def padded_length(n: int) -> int:
    """Circulant length of an n-point Toeplitz level: the smallest L >= 2n - 1
    (and >= 2) of the form 2^a, 3 * 2^a or 5 * 2^a (a >= 3 for the last two),
    the paper's K'' = 2K - 1 + kf with kf chosen for a fast DFT (Sec. 3,
    App. A)."""
    need = max(2, 2 * n - 1)
    best = None
    for start in (2, 24, 40):
        L = start
        while L < need:
            L *= 2
        best = L if best is None else min(best, L)
    return best


def mirror_signs() -> np.ndarray:
    """Table 1: sign of the mirrored half of each component per DFT axis.

    Row = axis of the line (x, y, z), column = component (xx ... zz).
    """
    return np.array([[+1, -1, -1, +1, +1, +1],
                     [+1, -1, +1, +1, -1, +1],
                     [+1, +1, -1, +1, -1, +1]], dtype=np.int64)


def tensor_section1(k: float, K: int, J: int, P: int) -> np.ndarray:
    """t_m(i, j, k) = A_jl component m at displacement (i, j, k), 0 <= i < K etc.

    'Section 1' of the paper's Fig. 6; the displacement 0 entry is 0 (the
    diagonal is added separately, Sec. 3).  Shape (6, P, J, K).
    """
    t = np.zeros((6, P, J, K), dtype=np.complex128)
    for z in range(P):
        for y in range(J):
            for x in range(K):
                if x == 0 and y == 0 and z == 0:
                    continue
                t[:, z, y, x] = dda.interaction_tensor(k, (x, y, z))
    return t


def first_column(k: float, K: int, J: int, P: int, L: tuple) -> np.ndarray:
    """First column of the level-three circulant for each component.

    Entry (z, y, x) of an Lz x Ly x Lx grid holds A at the displacement
    (dx, dy, dz) with dx = x for x < K, dx = x - Lx for x > Lx - K, and 0 in
    between (zero padding); the same for y and z.  Built from A(r) at the
    negative displacements themselves, without the Table-1 signs.
    """
    Lx, Ly, Lz = L
    c = np.zeros((6, Lz, Ly, Lx), dtype=np.complex128)

    def disp(v, n, Ln):
        if v < n:
            return v
        if v > Ln - n:
            return v - Ln
        return None

    for z in range(Lz):
        dz = disp(z, P, Lz)
        if dz is None:
            continue
        for y in range(Ly):
            dy = disp(y, J, Ly)
            if dy is None:
                continue
            for x in range(Lx):
                dx = disp(x, K, Lx)
                if dx is None or (dx == 0 and dy == 0 and dz == 0):
                    continue
                c[:, z, y, x] = dda.interaction_tensor(k, (dx, dy, dz))
    return c


def fft_matvec(col: np.ndarray, mask: np.ndarray, ainv: np.ndarray, p: np.ndarray) -> np.ndarray:
    """y = A p through the full circulant embedding (App. A, Eqs. 6-8).

    col: first_column(...) (6, Lz, Ly, Lx); mask (P, J, K); ainv (N_d, 3);
    p [3][N_d] compressed.  Returns y [3][N_d].
    """
    _, Lz, Ly, Lx = col.shape
    P, J, K = mask.shape
    occ = dda.occupied_sites(mask)
    Y = np.fft.fftn(col, axes=(1, 2, 3))
    X = np.zeros((3, Lz, Ly, Lx), dtype=np.complex128)
    for c in range(3):
        v = np.zeros(P * J * K, dtype=np.complex128)
        v[occ] = p[c]
        X[c, :P, :J, :K] = v.reshape(P, J, K)
    X = np.fft.fftn(X, axes=(1, 2, 3))
    Q = np.empty_like(X)
    Q[0] = Y[0] * X[0] + Y[1] * X[1] + Y[2] * X[2]   # Eq. 6
    Q[1] = Y[1] * X[0] + Y[3] * X[1] + Y[4] * X[2]   # Eq. 7
    Q[2] = Y[2] * X[0] + Y[4] * X[1] + Y[5] * X[2]   # Eq. 8
    q = np.fft.ifftn(Q, axes=(1, 2, 3))
    y = np.empty((3, occ.size), dtype=np.complex128)
    for c in range(3):
        y[c] = q[c, :P, :J, :K].reshape(-1)[occ] + np.asarray(ainv)[:, c] * p[c]
    return y


def half_spectrum(t1: np.ndarray, L: tuple) -> np.ndarray:
    """The paper's fused T-to-c + DFT of the six components (Sec. 3).

    t1: section 1, (6, P, J, K).  For each axis in the order x, y, z, every
    line of n stored values is copied to a buffer of length L, its entries
    1..n-1 are mirrored to positions L-1..L-n+1 with the Table-1 sign, the
    buffer is transformed, and the first L/2 + 1 outputs are kept.
    Returns (6, Lz/2+1, Ly/2+1, Lx/2+1), unnormalised.
    """
    sg = mirror_signs()
    out = t1
    for axis, Ln in ((0, L[0]), (1, L[1]), (2, L[2])):
        arr_axis = 3 - axis          # numpy axis of x, y, z in (6, z, y, x)
        n = out.shape[arr_axis]
        H = Ln // 2 + 1
        shp = list(out.shape)
        shp[arr_axis] = Ln
        buf = np.zeros(shp, dtype=np.complex128)
        for m in range(6):
            src = np.moveaxis(out[m], arr_axis - 1, -1)
            dst = np.moveaxis(buf[m], arr_axis - 1, -1)
            dst[..., :n] = src
            if n > 1:
                dst[..., Ln - n + 1:] = sg[axis, m] * src[..., 1:][..., ::-1]
        spec = np.fft.fft(buf, axis=arr_axis)
        out = np.take(spec, np.arange(H), axis=arr_axis)
    return out


def expand_half_spectrum(half: np.ndarray, L: tuple) -> np.ndarray:
    """Full spectrum from the stored half by the mirror rule with signs.

    Index i > L/2 reads i' = L - i and multiplies component m by the Table-1
    sign of that axis; the signs of mirrored axes multiply.
    """
    Lx, Ly, Lz = L
    sg = mirror_signs()
    full = np.empty((6, Lz, Ly, Lx), dtype=np.complex128)
    ix = np.arange(Lx)
    iy = np.arange(Ly)
    iz = np.arange(Lz)
    mx = np.where(ix <= Lx // 2, ix, Lx - ix)
    my = np.where(iy <= Ly // 2, iy, Ly - iy)
    mz = np.where(iz <= Lz // 2, iz, Lz - iz)
    for m in range(6):
        sx = np.where(ix <= Lx // 2, 1, sg[0, m])
        sy = np.where(iy <= Ly // 2, 1, sg[1, m])
        sz = np.where(iz <= Lz // 2, 1, sg[2, m])
        full[m] = (half[m][np.ix_(mz, my, mx)] * sz[:, None, None] * sy[None, :, None]
                   * sx[None, None, :])
    return full
