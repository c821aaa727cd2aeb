"""The quick-start block of README.md runs as written: a 64^3 sphere solved
with mixed-precision BiCGSTAB to 1e-5, with physically consistent cross
sections (lossy material: C_abs > 0, C_sca > 0; C_sca = C_ext - C_abs)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _quick_start():
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert blocks, "README.md has no python block"
    return blocks[0]


def test_readme_has_quick_start():
    code = _quick_start()
    compile(code, "README.md", "exec")
    assert "lat.solve(" in code and "lat.cross_sections(" in code


@pytest.mark.gpu
def test_readme_quick_start_runs():
    import paper_0908_0863_gb300 as dda
    scope = {}
    exec(compile(_quick_start(), "README.md", "exec"), scope)
    assert scope["status"] == dda.DDA_OK, scope["info"]
    assert scope["info"]["rel_residual_true"] <= 1e-5
    c_ext, c_abs, c_sca = scope["c_ext"], scope["c_abs"], scope["c_sca"]
    assert c_abs > 0 and c_sca > 0
    assert abs(c_ext - c_abs - c_sca) <= 1e-12 * abs(c_ext)
