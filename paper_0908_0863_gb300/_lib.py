"""ctypes binding of the C ABI in include/dda.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but convert arguments (torch tensors -> device pointers, numpy
arrays -> host pointers, streams -> cudaStream_t) and turn error codes into
exceptions.  All computation happens in the CUDA library; if that library
is missing the import of this module fails instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

DDA_OK = 0
DDA_ERR_ARG = -1
DDA_ERR_CUDA = -2
DDA_ERR_OOM = -3
DDA_ERR_NOT_CONVERGED = -4
DDA_ERR_BREAKDOWN = -5
DDA_ERR_NAN = -6
DDA_C128 = 0
DDA_C64 = 1
DDA_C128DF = 2   # complex128 vectors, double-float products
DDA_BICG, DDA_BICGSTAB, DDA_QMR, DDA_BICG_SYM = 0, 1, 2, 3
DDA_CG, DDA_CGS, DDA_TFQMR, DDA_QMR_SYM = 4, 5, 6, 7
DDA_RBICGSTAB1, DDA_RBICGSTAB2, DDA_RBICGSTAB3 = 8, 9, 10
DDA_MLBICGSTAB1, DDA_MLBICGSTAB2, DDA_MLBICGSTAB3 = 11, 12, 13
DDA_PRECOND_JACOBI = 0x100
DDA_FP64, DDA_MIXED = 0, 1
DDA_POL_CM, DDA_POL_CMRR, DDA_POL_LDR = 0, 1, 2
DDA_POL_EPS = 0x10

METHODS = {"bicg": DDA_BICG, "bicgstab": DDA_BICGSTAB, "qmr": DDA_QMR, "bicg_sym": DDA_BICG_SYM, "cg": DDA_CG,
           "cgs": DDA_CGS, "tfqmr": DDA_TFQMR, "qmr_sym": DDA_QMR_SYM, "rbicgstab1": DDA_RBICGSTAB1,
           "rbicgstab2": DDA_RBICGSTAB2, "rbicgstab3": DDA_RBICGSTAB3, "mlbicgstab1": DDA_MLBICGSTAB1,
           "mlbicgstab2": DDA_MLBICGSTAB2, "mlbicgstab3": DDA_MLBICGSTAB3}


def method_code(method) -> int:
    """A dda_method value from a name ("bicgstab", "qmr_sym+jacobi", ...) or an int."""
    if not isinstance(method, str):
        return int(method)
    base, *opts = method.split("+")
    code = METHODS[base]
    for o in opts:
        if o != "jacobi":
            raise ValueError(f"unknown solver option {o!r}")
        code |= DDA_PRECOND_JACOBI
    return code
PRECISIONS = {"fp64": DDA_FP64, "mixed": DDA_MIXED}
RULES = {"cm": DDA_POL_CM, "cmrr": DDA_POL_CMRR, "ldr": DDA_POL_LDR}

# every entry point declared in include/dda.h
EXPORTS = (
    "dda_polarizability", "dda_pack_occupancy", "dda_unpack_occupancy", "dda_pack_composition",
    "dda_unpack_composition", "dda_init_lattice", "dda_free", "dda_query", "dda_site_ranks",
    "dda_tensor_spectrum", "dda_matvec", "dda_incident_field", "dda_solve", "dda_cross_sections",
    "dda_profile", "dda_profile_read", "dda_launch_count", "dda_last_error", "dda_occupancy_ranks_static",
    "dda_material_sums", "dda_inner_tolerance", "dda_autotune_inner", "dda_residual_dtype",
    "dda_scattering_cross_section", "dda_polarizability_derivative", "dda_gradient",
    "dda_matvec_batch", "dda_reserve", "dda_solve_batch", "dda_cross_sections_batch", "dda_tiles",
    "dda_autotune",
)


class DDAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("matvecs", ctypes.c_int), ("matvecs_fp64", ctypes.c_int),
                ("refinements", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("rel_residual_true", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libdda.so (built by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"DDA CUDA library not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.dda_polarizability.argtypes = [i32, vp, d, i32, vp, vp, vp]
    L.dda_pack_occupancy.argtypes = [vp, i64, vp, vp]
    L.dda_unpack_occupancy.argtypes = [vp, i64, vp, vp]
    L.dda_pack_composition.argtypes = [vp, i64, i32, vp, vp]
    L.dda_unpack_composition.argtypes = [vp, i64, i32, vp, vp]
    L.dda_init_lattice.argtypes = [ctypes.POINTER(vp), vp, vp, vp, i32, vp, d, vp]
    L.dda_free.argtypes = [vp]
    L.dda_free.restype = None
    L.dda_query.argtypes = [vp, vp, vp, vp]
    L.dda_site_ranks.argtypes = [vp, vp, vp]
    L.dda_tensor_spectrum.argtypes = [vp, vp, i32, vp]
    L.dda_matvec.argtypes = [vp, vp, vp, i32, vp]
    L.dda_incident_field.argtypes = [vp, vp, vp, vp, vp]
    L.dda_solve.argtypes = [vp, vp, vp, i32, i32, d, i32, i32, ctypes.POINTER(SolveInfo), vp]
    L.dda_cross_sections.argtypes = [vp, vp, vp, vp, vp]
    L.dda_matvec_batch.argtypes = [vp, i32, vp, vp, i32, vp]
    L.dda_reserve.argtypes = [vp, i32, i32]
    L.dda_tiles.argtypes = [vp, i32, vp, vp]
    L.dda_autotune.argtypes = [vp, i32, i32, i32, vp, vp]
    L.dda_solve_batch.argtypes = [vp, i32, vp, vp, i32, i32, d, i32, i32, vp, vp, vp]
    L.dda_cross_sections_batch.argtypes = [vp, i32, vp, vp, vp, vp]
    L.dda_occupancy_ranks_static.argtypes = [vp, i64, vp, vp, vp]
    L.dda_material_sums.argtypes = [vp, vp, vp, vp]
    L.dda_inner_tolerance.argtypes = [vp, i32, vp, vp]
    L.dda_residual_dtype.argtypes = [vp, vp, vp]
    L.dda_autotune_inner.argtypes = [vp, vp, i32, ctypes.c_double, i32, vp, vp, vp]
    L.dda_scattering_cross_section.argtypes = [vp, vp, vp, vp]
    L.dda_polarizability_derivative.argtypes = [i32, vp, d, i32, vp, vp, vp]
    L.dda_gradient.argtypes = [vp, i32, vp, vp, vp, i32, i32, d, i32, vp, ctypes.POINTER(SolveInfo), vp]
    L.dda_profile.argtypes = [vp, i32]
    L.dda_profile_read.argtypes = [vp, vp, vp]
    L.dda_launch_count.argtypes = []
    L.dda_launch_count.restype = ctypes.c_int64
    L.dda_last_error.argtypes = []
    L.dda_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("dda_free", "dda_last_error", "dda_launch_count"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(code):
    if code != DDA_OK:
        raise DDAError(code, load().dda_last_error().decode())
    return code


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(x):
    """Device pointer of a torch tensor, or host pointer of a numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError(f"unsupported buffer type {type(x)}")


def _dtype_code(t):
    import torch
    if t.dtype == torch.complex128:
        return DDA_C128
    if t.dtype == torch.complex64:
        return DDA_C64
    raise TypeError("vectors must be complex128 or complex64")


def _c2(v, n):
    a = np.asarray(v, dtype=np.complex128).reshape(n)
    return np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1).reshape(-1))


# ------------------------------------------------------------ entry points

def dda_polarizability(m, k, rule="cmrr", khat=None, e0=None, given="m") -> np.ndarray:
    """alpha per material and axis, shape (n_materials, 3) complex128; m holds
    refractive indices (given="m") or permittivities (given="eps")."""
    m = np.atleast_1d(np.asarray(m, dtype=np.complex128))
    n = m.size
    out = np.zeros(n * 6)
    kh = None if khat is None else np.ascontiguousarray(np.asarray(khat, dtype=np.float64))
    ee = None if e0 is None else _c2(e0, 3)
    code = RULES.get(rule, rule) | (DDA_POL_EPS if given == "eps" else 0)
    _check(load().dda_polarizability(n, _ptr(_c2(m, n)), float(k), code, _ptr(kh), _ptr(ee), _ptr(out)))
    return (out[0::2] + 1j * out[1::2]).reshape(n, 3)


def dda_pack_occupancy(mask, bits, stream=None):
    _check(load().dda_pack_occupancy(_ptr(mask), mask.numel(), _ptr(bits), _stream(stream)))


def dda_unpack_occupancy(bits, n_sites, mask, stream=None):
    _check(load().dda_unpack_occupancy(_ptr(bits), int(n_sites), _ptr(mask), _stream(stream)))


def dda_pack_composition(materials, n_sites, n_materials, bits, stream=None):
    _check(load().dda_pack_composition(_ptr(materials), int(n_sites), int(n_materials), _ptr(bits),
                                       _stream(stream)))


def dda_unpack_composition(bits, n_sites, n_materials, materials, stream=None):
    _check(load().dda_unpack_composition(_ptr(bits), int(n_sites), int(n_materials), _ptr(materials),
                                         _stream(stream)))


def dda_init_lattice(shape, occupancy_bits, composition_bits, n_materials, alpha, k, stream=None):
    """Returns an opaque context handle (int).  Bit fields: numpy (host) or torch (device)."""
    ctx = ctypes.c_void_p()
    shp = np.ascontiguousarray(np.asarray(shape, dtype=np.int32).reshape(3))
    al = _c2(np.asarray(alpha, dtype=np.complex128).reshape(-1), int(n_materials) * 3)
    _check(load().dda_init_lattice(ctypes.byref(ctx), _ptr(shp), _ptr(occupancy_bits),
                                   _ptr(composition_bits), int(n_materials), _ptr(al), float(k),
                                   _stream(stream)))
    return ctx.value


def dda_free(ctx):
    load().dda_free(ctypes.c_void_p(ctx))


def dda_query(ctx):
    nd = ctypes.c_int64()
    pad = (ctypes.c_int32 * 3)()
    nb = ctypes.c_int64()
    _check(load().dda_query(ctypes.c_void_p(ctx), ctypes.byref(nd), pad, ctypes.byref(nb)))
    return {"n_dipoles": nd.value, "padded": tuple(pad), "device_bytes": nb.value}


def dda_site_ranks(ctx, rank, stream=None):
    _check(load().dda_site_ranks(ctypes.c_void_p(ctx), _ptr(rank), _stream(stream)))


def dda_tensor_spectrum(ctx, out, stream=None):
    _check(load().dda_tensor_spectrum(ctypes.c_void_p(ctx), _ptr(out), _dtype_code(out), _stream(stream)))


def _product_code(p, dtype):
    # dtype None: the tensors' precision; "c128df": double-float products of
    # complex128 tensors
    if dtype is None:
        return _dtype_code(p)
    code = _dtype_name(dtype)
    if code == DDA_C128DF and _dtype_code(p) != DDA_C128:
        raise TypeError("double-float products take complex128 vectors")
    return code


def dda_matvec(ctx, p, y, stream=None, dtype=None):
    if p.dtype != y.dtype:
        raise TypeError("p and y must have the same dtype")
    _check(load().dda_matvec(ctypes.c_void_p(ctx), _ptr(p), _ptr(y), _product_code(p, dtype), _stream(stream)))


def dda_matvec_batch(ctx, p, y, stream=None, dtype=None):
    """y[b] = A p[b] for p, y of shape (nb, 3, N_d) (device, same complex dtype)."""
    if p.dtype != y.dtype or p.shape != y.shape:
        raise TypeError("p and y must have the same dtype and shape")
    _check(load().dda_matvec_batch(ctypes.c_void_p(ctx), int(p.shape[0]), _ptr(p), _ptr(y), _product_code(p, dtype),
                                   _stream(stream)))


def _dtype_name(dtype):
    return {"c128": DDA_C128, "c64": DDA_C64, "c128df": DDA_C128DF}.get(dtype, dtype)


def dda_tiles(ctx, dtype="c64", tiles=None):
    """Current tile settings (log2 lines per CTA of P1/P5, P3 and P2/P4, and a
    reserved 0); sets them first when given (with 3 widths the fourth is 0)."""
    out = np.zeros(4, dtype=np.int32)
    tin = None
    if tiles is not None:
        tiles = list(tiles)
        if len(tiles) == 3:
            tiles.append(0)
        tin = np.ascontiguousarray(np.asarray(tiles, dtype=np.int32).reshape(4))
    _check(load().dda_tiles(ctypes.c_void_p(ctx), _dtype_name(dtype), _ptr(out), _ptr(tin)))
    return tuple(int(v) for v in out)


def dda_autotune(ctx, dtype="c64", nb=1, reps=3, stream=None):
    """Tune the tile widths; returns the per-pass milliseconds of the choice."""
    ms = np.zeros(5)
    _check(load().dda_autotune(ctypes.c_void_p(ctx), _dtype_name(dtype), int(nb), int(reps), _ptr(ms),
                               _stream(stream)))
    return [float(v) for v in ms]


def dda_reserve(ctx, nb, precision="mixed"):
    _check(load().dda_reserve(ctypes.c_void_p(ctx), int(nb), PRECISIONS.get(precision, precision)))


def dda_incident_field(ctx, khat, e0, einc, stream=None):
    kh = np.ascontiguousarray(np.asarray(khat, dtype=np.float64).reshape(3))
    _check(load().dda_incident_field(ctypes.c_void_p(ctx), _ptr(kh), _ptr(_c2(e0, 3)), _ptr(einc),
                                     _stream(stream)))


def dda_solve(ctx, einc, p, method="bicgstab", precision="fp64", tol=1e-8, max_iter=1000, use_x0=False,
              stream=None):
    """Returns (status, info dict); raises only for argument / CUDA errors."""
    info = SolveInfo()
    code = load().dda_solve(ctypes.c_void_p(ctx), _ptr(einc), _ptr(p), method_code(method),
                            PRECISIONS.get(precision, precision), float(tol), int(max_iter), int(bool(use_x0)),
                            ctypes.byref(info), _stream(stream))
    if code in (DDA_ERR_ARG, DDA_ERR_CUDA, DDA_ERR_OOM):
        _check(code)
    return code, info.as_dict()


def dda_solve_batch(ctx, einc, p, method="bicgstab", precision="fp64", tol=1e-8, max_iter=1000, use_x0=False,
                    stream=None):
    """Solves for einc, p of shape (nb, 3, N_d) complex128 (host numpy or
    device torch).  Returns (status, [per-RHS status], [per-RHS info dict]);
    raises only for argument / CUDA / allocation errors."""
    nb = int(einc.shape[0])
    infos = (SolveInfo * nb)()
    stats = np.zeros(nb, dtype=np.int32)
    code = load().dda_solve_batch(ctypes.c_void_p(ctx), nb, _ptr(einc), _ptr(p), method_code(method),
                                  PRECISIONS.get(precision, precision), float(tol), int(max_iter),
                                  int(bool(use_x0)), ctypes.cast(infos, ctypes.c_void_p), _ptr(stats),
                                  _stream(stream))
    if code in (DDA_ERR_ARG, DDA_ERR_CUDA, DDA_ERR_OOM):
        _check(code)
    return code, [int(v) for v in stats], [infos[b].as_dict() for b in range(nb)]


def dda_cross_sections_batch(ctx, einc, p, stream=None) -> np.ndarray:
    """(nb, 3) array of (C_ext, C_abs, C_sca) for einc, p of shape (nb, 3, N_d)."""
    nb = int(einc.shape[0])
    out = np.zeros(3 * nb)
    _check(load().dda_cross_sections_batch(ctypes.c_void_p(ctx), nb, _ptr(einc), _ptr(p), _ptr(out),
                                           _stream(stream)))
    return out.reshape(nb, 3)


def dda_cross_sections(ctx, einc, p, stream=None):
    out = np.zeros(3)
    _check(load().dda_cross_sections(ctypes.c_void_p(ctx), _ptr(einc), _ptr(p), _ptr(out), _stream(stream)))
    return tuple(float(v) for v in out)


def dda_scattering_cross_section(ctx, p, stream=None) -> float:
    out = np.zeros(1)
    _check(load().dda_scattering_cross_section(ctypes.c_void_p(ctx), _ptr(p), _ptr(out), _stream(stream)))
    return float(out[0])


def dda_polarizability_derivative(m, k, rule="cmrr", khat=None, e0=None, given="m") -> np.ndarray:
    """d(1/alpha)/d eps per material and axis, shape (n_materials, 3) complex128;
    m holds refractive indices (given="m") or permittivities (given="eps")."""
    m = np.atleast_1d(np.asarray(m, dtype=np.complex128))
    n = m.size
    out = np.zeros(n * 6)
    kh = None if khat is None else np.ascontiguousarray(np.asarray(khat, dtype=np.float64))
    ee = None if e0 is None else _c2(e0, 3)
    code = RULES.get(rule, rule) | (DDA_POL_EPS if given == "eps" else 0)
    _check(load().dda_polarizability_derivative(n, _ptr(_c2(m, n)), float(k), code, _ptr(kh), _ptr(ee),
                                                _ptr(out)))
    return (out[0::2] + 1j * out[1::2]).reshape(n, 3)


def dda_inner_tolerance(ctx, rho=None, method="bicgstab") -> float:
    """The mixed-precision inner reduction rho of the context for one Krylov
    method (set first when given)."""
    rin = None if rho is None else np.array([float(rho)])
    out = np.zeros(1)
    _check(load().dda_inner_tolerance(ctypes.c_void_p(ctx), method_code(method), _ptr(rin), _ptr(out)))
    return float(out[0])


def dda_residual_dtype(ctx, dtype=None) -> str:
    """Products of the mixed refinement's true residuals: "c128df" (double-float,
    the default) or "c128" (FP64); set first when given."""
    din = None if dtype is None else np.array([_dtype_name(dtype)], dtype=np.int32)
    out = np.zeros(1, dtype=np.int32)
    _check(load().dda_residual_dtype(ctypes.c_void_p(ctx), _ptr(din), _ptr(out)))
    return {DDA_C128: "c128", DDA_C128DF: "c128df"}[int(out[0])]


def dda_autotune_inner(ctx, einc, method="bicgstab", tol=1e-5, max_iter=4000, stream=None):
    """Tunes rho on einc; returns (rho, {rho candidate: solve ms or -1})."""
    rho = np.zeros(1)
    ms = np.zeros(6)
    _check(load().dda_autotune_inner(ctypes.c_void_p(ctx), _ptr(einc), method_code(method), float(tol),
                                     int(max_iter), _ptr(rho), _ptr(ms), _stream(stream)))
    return float(rho[0]), dict(zip((0.0, 1e-4, 1e-3, 1e-2, 3e-2, 1e-1), (float(v) for v in ms)))


def dda_material_sums(ctx, v, n_materials, stream=None) -> np.ndarray:
    """Per-material sums of a per-dipole complex128 field v ([N_d], host or
    device), shape (n_materials,) complex128."""
    out = np.zeros(2 * int(n_materials))
    _check(load().dda_material_sums(ctypes.c_void_p(ctx), _ptr(v), _ptr(out), _stream(stream)))
    return out[0::2] + 1j * out[1::2]


def dda_gradient(ctx, which, einc, p, dalpha_inv, grad, method="bicgstab", precision="fp64", tol=1e-8,
                 max_iter=1000, stream=None):
    """Per-dipole d C / d eps (which: 'ext' or 'abs'); returns (status, info)."""
    w = {"ext": 0, "abs": 1}.get(which, which)
    da = _c2(np.asarray(dalpha_inv, dtype=np.complex128).reshape(-1), np.asarray(dalpha_inv).size)
    info = SolveInfo()
    code = load().dda_gradient(ctypes.c_void_p(ctx), int(w), _ptr(einc), _ptr(p), _ptr(da),
                               method_code(method), PRECISIONS.get(precision, precision), float(tol),
                               int(max_iter), _ptr(grad), ctypes.byref(info), _stream(stream))
    if code in (DDA_ERR_ARG, DDA_ERR_CUDA, DDA_ERR_OOM, DDA_ERR_NAN):
        _check(code)
    return code, info.as_dict()


def dda_occupancy_ranks_static(bits, n_sites, word_rank, n_occupied, stream=None):
    """Rank scan of an occupancy bit field that allocates no device memory
    (device tensors in, device tensors out; see include/dda.h)."""
    _check(load().dda_occupancy_ranks_static(_ptr(bits), int(n_sites), _ptr(word_rank), _ptr(n_occupied),
                                             _stream(stream)))


def dda_profile(ctx, enable=True):
    _check(load().dda_profile(ctypes.c_void_p(ctx), int(bool(enable))))


def dda_profile_read(ctx):
    """{'c128'|'c64': [(launches, ms) for P1..P5]} of the recorded passes."""
    counts = np.zeros(10, dtype=np.int64)
    ms = np.zeros(10)
    _check(load().dda_profile_read(ctypes.c_void_p(ctx), _ptr(counts), _ptr(ms)))
    return {name: [(int(counts[d * 5 + q]), float(ms[d * 5 + q])) for q in range(5)]
            for d, name in ((0, "c128"), (1, "c64"))}


def dda_launch_count() -> int:
    return int(load().dda_launch_count())


def dda_last_error() -> str:
    return load().dda_last_error().decode()
