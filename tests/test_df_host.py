"""Double-float arithmetic of the mixed refinement's residual products
(csrc/df.cuh), compiled for the host and checked against exact rational
arithmetic: the two-sum is error-free, the conversion from a double keeps
about 48 bits, and the sum, difference, product and multiply-add stay within
their error bounds, also under cancellation.  The same header is what the
device passes instantiate; its error-free transforms round every operation
on its own on both sides."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0908_0863_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.fixture(scope="module")
def df_host(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs a host C++ compiler and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("df") / "df_host")
    subprocess.run([cxx, "-O2", "-std=c++17", "-w", "-ffp-contract=off", f"-I{CSRC}", f"-I{CUDA_INC}",
                    os.path.join(ROOT, "tests", "df_host.cpp"), "-o", exe], check=True)

    def run(cases):
        text = "".join(f"{op} {float(a).hex()} {float(b).hex()}\n" for op, a, b in cases)
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
        rows = [[Fraction(float.fromhex(w)) for w in line.split()] for line in out if line]
        assert len(rows) == len(cases)
        return rows
    return run


def _operands(seed, n, cancel=False):
    """Seeded doubles of random sign with magnitudes 2^-30..2^30; with
    cancel, b = -a (1 + 2^-k u) for k in 20..50 (partial cancellation down
    to about 2^-50 of |a|)."""
    rng = np.random.default_rng(seed)
    a = rng.choice([-1.0, 1.0], n) * np.exp2(rng.uniform(-30, 30, n))
    if cancel:
        b = -a * (1.0 + np.exp2(-rng.integers(20, 51, n).astype(float)) * rng.uniform(-1, 1, n))
    else:
        b = rng.choice([-1.0, 1.0], n) * np.exp2(rng.uniform(-30, 30, n))
    return a, b


def _df(hi, lo):
    return hi + lo


def _normalised(hi, lo):
    """|lo| at most half an ulp of hi: hi is the float nearest hi + lo."""
    return float(np.float32(float(hi + lo))) == float(hi)


def test_two_sum_is_error_free(df_host):
    a, b = _operands(1, 400)
    a32, b32 = a.astype(np.float32).astype(float), b.astype(np.float32).astype(float)
    rows = df_host([("two_sum", x, y) for x, y in zip(a32, b32)])
    for x, y, r in zip(a32, b32, rows):
        assert r[4] + r[5] == Fraction(x) + Fraction(y)
        assert r[4] == Fraction(float(np.float32(x) + np.float32(y)))


def test_conversion_keeps_48_bits(df_host):
    a, b = _operands(2, 300)
    rows = df_host([("add", x, y) for x, y in zip(a, b)])
    for x, r in zip(a, rows):
        assert abs(_df(r[0], r[1]) - Fraction(x)) <= Fraction(2) ** -48 * abs(Fraction(x))
        assert _normalised(r[0], r[1])


@pytest.mark.parametrize("cancel", [False, True])
def test_sum_and_difference_bounds(df_host, cancel):
    a, b = _operands(3 + cancel, 400, cancel)
    for op, sign in (("add", 1), ("sub", -1)):
        if cancel and op == "sub":
            b = -b    # a - (-b') cancels in the same way
        rows = df_host([(op, x, y) for x, y in zip(a, b)])
        for r in rows:
            x, y = _df(r[0], r[1]), _df(r[2], r[3])
            exact = x + sign * y
            err = abs(_df(r[4], r[5]) - exact)
            assert err <= Fraction(2) ** -45 * (abs(x) + abs(y)), (op, float(err / (abs(x) + abs(y))))
            assert _normalised(r[4], r[5])


def test_exact_cancellation_and_zero(df_host):
    rows = df_host([("add", 1.0 + 2.0 ** -30, -1.0), ("sub", 3.0, 3.0), ("add", 0.0, 0.0),
                    ("mul", 0.0, 5.0), ("add", 1.0 + 2.0 ** -40, -(1.0 + 2.0 ** -41))])
    assert _df(rows[0][4], rows[0][5]) == Fraction(2) ** -30
    assert rows[1][4] == 0 and rows[1][5] == 0
    assert rows[2][4] == 0 and rows[2][5] == 0
    assert rows[3][4] == 0 and rows[3][5] == 0
    # both operands carry their low parts: the difference 2^-41 is exact
    assert _df(rows[4][4], rows[4][5]) == Fraction(2) ** -41


def test_product_and_multiply_add_bounds(df_host):
    a, b = _operands(5, 400)
    rows = df_host([("mul", x, y) for x, y in zip(a, b)])
    for r in rows:
        x, y = _df(r[0], r[1]), _df(r[2], r[3])
        err = abs(_df(r[4], r[5]) - x * y)
        assert err <= Fraction(2) ** -45 * abs(x * y), float(err / abs(x * y))
        assert _normalised(r[4], r[5])
    # x * y + x with y near -1: the sum cancels
    a, b = _operands(6, 300, cancel=True)
    rows = df_host([("fma", x, y / x) for x, y in zip(a, b)])
    for r in rows:
        x, y = _df(r[0], r[1]), _df(r[2], r[3])
        err = abs(_df(r[4], r[5]) - (x * y + x))
        assert err <= Fraction(2) ** -44 * (abs(x * y) + abs(x))
