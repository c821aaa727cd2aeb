"""CPU checks of the C ABI: the library builds, loads and exports every
entry point include/dda.h declares (no GPU call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "dda.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(dda_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from conftest import build_library
    return ctypes.CDLL(build_library())


def test_every_declared_entry_point_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_0908_0863_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()


def test_polarizability_host_only(lib):
    # dda_polarizability runs on the host: callable without a GPU
    import numpy as np
    from paper_0908_0863_gb300 import _lib
    out = _lib.dda_polarizability([1.5 + 0.1j], 0.3, "cmrr")
    from oracle import dda as odda
    assert abs(out[0, 0] - odda.alpha_rr(1.5 + 0.1j, 0.3)) < 1e-15
    with pytest.raises(_lib.DDAError):
        _lib.dda_polarizability([1.5], 0.3, 7)
    assert np.isfinite(out).all()


def test_last_error_after_failure(lib):
    from paper_0908_0863_gb300 import _lib
    with pytest.raises(_lib.DDAError) as e:
        _lib.dda_polarizability([], 0.3, "cm")
    assert "dda_polarizability" in str(e.value)
    assert "dda_polarizability" in _lib.dda_last_error()
