"""Plain, slow, FP64 CPU oracle of the DDA interaction-matrix product and solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import, call, link or execute
anything in this package.  The product (``paper_0908_0863_gb300``) never
imports it, shares no code with it, and fails loudly when its CUDA library
is missing instead of falling back to anything here.

Modules (each function cites the passage of the OpenDDA paper it follows):

* ``dda``       bit fields, polarisabilities, incident field, direct-sum
                matvec (C, ``direct.c``), dense matrix, cross sections.
* ``circulant`` the circulant-embedding FFT form (App. A) and the paper's
                half-spectrum tensor transforms with the Table-1 signs.
* ``solvers``   BiCG, BiCG_sym, BiCGSTAB, QMR (Sec. 4).
* ``mie``       Mie series for the sphere-convergence check.

Parity pins: every function is checked in ``tests/test_oracle_*.py``
against values the paper prints, closed forms, invariants or brute force.
"""
from . import circulant, dda, mie, solvers  # noqa: F401
from ._native import build  # noqa: F401
