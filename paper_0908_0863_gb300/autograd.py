"""torch.autograd view of the DDA cross sections (argument marshalling only).

``CrossSection.apply(eps, target)`` returns C_ext or C_abs of a target whose
materials have the complex permittivities ``eps`` (one per material, a
complex128 tensor).  The forward pass builds a context, solves A P = E_inc
and sums the cross section; the backward pass runs the adjoint entry point
``dda_gradient`` (one extra solve with the same matrix, A^T = A) and
``dda_material_sums``, which adds the per-dipole gradients of each material
(the material of a dipole is its composition field, axis x).  The gradient
follows PyTorch's convention for real outputs of complex inputs:
dC/dRe(eps) + i dC/dIm(eps).  The permittivities go to the library as they
are (DDA_POL_EPS); all arithmetic runs in the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import _lib


@dataclass
class Target:
    shape: tuple                      # (K, J, P)
    occupancy_bits: np.ndarray        # uint32 words (host)
    k: float
    which: str = "abs"                # "abs" or "ext"
    rule: str = "cmrr"
    khat: tuple = (0.0, 0.0, 1.0)
    e0: tuple = (1.0, 0.0, 0.0)
    composition_bits: np.ndarray | None = None
    method: str = "bicgstab"
    precision: str = "fp64"
    tol: float = 1e-10
    max_iter: int = 4000
    extras: dict = field(default_factory=dict)


def _solve(eps, tgt: Target):
    import torch
    m = np.ascontiguousarray(eps.detach().cpu().numpy().astype(np.complex128))   # permittivities
    alpha = _lib.dda_polarizability(m, tgt.k, tgt.rule, tgt.khat, tgt.e0, given="eps")
    ctx = _lib.dda_init_lattice(tgt.shape, tgt.occupancy_bits, tgt.composition_bits, m.size, alpha, tgt.k)
    nd = _lib.dda_query(ctx)["n_dipoles"]
    E = torch.empty((3, nd), dtype=torch.complex128, device="cuda")
    _lib.dda_incident_field(ctx, tgt.khat, tgt.e0, E)
    P = torch.zeros_like(E)
    status, info = _lib.dda_solve(ctx, E, P, tgt.method, tgt.precision, tgt.tol, tgt.max_iter)
    if status != _lib.DDA_OK:
        _lib.dda_free(ctx)
        raise _lib.DDAError(status, f"forward solve failed: {info}")
    return ctx, m, E, P, nd


class CrossSection:
    """Namespace of the torch.autograd.Function (created lazily so that
    importing this module does not need torch)."""

    _fn = None

    @classmethod
    def apply(cls, eps, tgt: Target):
        if cls._fn is None:
            cls._fn = _make_function()
        return cls._fn.apply(eps, tgt)


def _make_function():
    import torch

    class _CrossSection(torch.autograd.Function):
        @staticmethod
        def forward(fctx, eps, tgt):
            ctx, m, E, P, nd = _solve(eps, tgt)
            try:
                cx = _lib.dda_cross_sections(ctx, E, P)
            finally:
                _lib.dda_free(ctx)
            fctx.tgt = tgt
            fctx.state = (E, P, m)
            fctx.eps_device = eps.device
            return torch.tensor(cx[0] if tgt.which == "ext" else cx[1], dtype=torch.float64, device=eps.device)

        @staticmethod
        def backward(fctx, grad_out):
            tgt = fctx.tgt
            E, P, m = fctx.state
            alpha = _lib.dda_polarizability(m, tgt.k, tgt.rule, tgt.khat, tgt.e0, given="eps")
            dainv = _lib.dda_polarizability_derivative(m, tgt.k, tgt.rule, tgt.khat, tgt.e0, given="eps")
            ctx = _lib.dda_init_lattice(tgt.shape, tgt.occupancy_bits, tgt.composition_bits, m.size, alpha, tgt.k)
            try:
                g = torch.empty(P.shape[1], dtype=torch.complex128, device="cuda")
                status, info = _lib.dda_gradient(ctx, tgt.which, E, P, dainv, g, tgt.method, tgt.precision,
                                                 tgt.tol, tgt.max_iter)
                if status != _lib.DDA_OK:
                    raise _lib.DDAError(status, f"adjoint solve failed: {info}")
                per_mat = torch.from_numpy(_lib.dda_material_sums(ctx, g, m.size))
            finally:
                _lib.dda_free(ctx)
            return (grad_out.cpu() * per_mat).to(fctx.eps_device), None

    return _CrossSection
