"""GB300 (sm_103a) library for the DDA hot path of OpenDDA (arXiv:0908.0863).

The FFT-accelerated interaction-matrix product of the Discrete Dipole
Approximation, the Krylov solves built on it (BiCG, BiCGSTAB, QMR in FP64
or complex64-inside-FP64 refinement), the bit-fielded target description
and the cross sections, all as hand-written CUDA kernels behind the C ABI
of ``include/dda.h``.  This package is the thin Python binding: the names
are the C entry points; ``Lattice`` only bundles a context handle.

Importing the package loads the CUDA library and raises if it has not been
built (``__graft_entry__.build()``); there is no CPU fallback.
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    DDA_BICG, DDA_BICG_SYM, DDA_BICGSTAB, DDA_C64, DDA_C128, DDA_CG, DDA_CGS, DDA_ERR_ARG, DDA_ERR_BREAKDOWN,
    DDA_ERR_CUDA, DDA_PRECOND_JACOBI, DDA_QMR_SYM, DDA_TFQMR, method_code,
    DDA_ERR_NAN, DDA_ERR_NOT_CONVERGED, DDA_ERR_OOM, DDA_FP64, DDA_MIXED, DDA_OK, DDA_QMR, EXPORTS, DDAError,
    dda_cross_sections, dda_cross_sections_batch, dda_free, dda_gradient, dda_incident_field, dda_init_lattice,
    dda_last_error, dda_matvec_batch, dda_reserve, dda_solve_batch, dda_tiles, dda_autotune,
    dda_launch_count, dda_polarizability_derivative, dda_scattering_cross_section,
    dda_matvec, dda_occupancy_ranks_static, dda_pack_composition, dda_pack_occupancy, dda_polarizability,
    dda_profile, dda_profile_read, dda_material_sums, dda_inner_tolerance, dda_autotune_inner, dda_residual_dtype, DDA_C128DF, DDA_POL_EPS, DDA_MLBICGSTAB1, DDA_MLBICGSTAB2,
    DDA_MLBICGSTAB3,
    dda_query, dda_site_ranks, dda_solve, dda_tensor_spectrum, dda_unpack_composition, dda_unpack_occupancy,
    library_path, load,
)

load()


class Lattice:
    """A context (target + wavenumber) with the entry points as methods.

    occupancy_bits / composition_bits: packed words (numpy on the host or a
    torch tensor on the device), alpha: (n_materials, 3) complex.
    """

    def __init__(self, shape, occupancy_bits, alpha, k, composition_bits=None, n_materials=1, stream=None):
        self.shape = tuple(int(v) for v in shape)
        self.k = float(k)
        self.ctx = dda_init_lattice(self.shape, occupancy_bits, composition_bits, n_materials, alpha, k, stream)
        q = dda_query(self.ctx)
        self.n_dipoles = q["n_dipoles"]
        self.padded = q["padded"]
        self.device_bytes = q["device_bytes"]

    def close(self):
        if self.ctx:
            dda_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def matvec(self, p, y, stream=None):
        dda_matvec(self.ctx, p, y, stream)

    def matvec_batch(self, p, y, stream=None):
        dda_matvec_batch(self.ctx, p, y, stream)

    def tiles(self, dtype="c64", tiles=None):
        return dda_tiles(self.ctx, dtype, tiles)

    def autotune(self, dtype="c64", nb=1, reps=3, stream=None):
        return dda_autotune(self.ctx, dtype, nb, reps, stream)

    def reserve(self, nb, precision="mixed"):
        dda_reserve(self.ctx, nb, precision)

    def solve_batch(self, einc, p, method="bicgstab", precision="fp64", tol=1e-8, max_iter=1000, use_x0=False,
                    stream=None):
        return dda_solve_batch(self.ctx, einc, p, method, precision, tol, max_iter, use_x0, stream)

    def cross_sections_batch(self, einc, p, stream=None):
        return dda_cross_sections_batch(self.ctx, einc, p, stream)

    def incident_field(self, khat, e0, einc, stream=None):
        dda_incident_field(self.ctx, khat, e0, einc, stream)

    def solve(self, einc, p, method="bicgstab", precision="fp64", tol=1e-8, max_iter=1000, use_x0=False,
              stream=None):
        return dda_solve(self.ctx, einc, p, method, precision, tol, max_iter, use_x0, stream)

    def cross_sections(self, einc, p, stream=None):
        return dda_cross_sections(self.ctx, einc, p, stream)

    def scattering_cross_section(self, p, stream=None):
        return dda_scattering_cross_section(self.ctx, p, stream)

    def gradient(self, which, einc, p, dalpha_inv, grad, method="bicgstab", precision="fp64", tol=1e-8,
                 max_iter=1000, stream=None):
        return dda_gradient(self.ctx, which, einc, p, dalpha_inv, grad, method, precision, tol, max_iter, stream)

    def site_ranks(self, rank, stream=None):
        dda_site_ranks(self.ctx, rank, stream)

    def tensor_spectrum(self, out, stream=None):
        dda_tensor_spectrum(self.ctx, out, stream)
