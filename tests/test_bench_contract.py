"""bench.py keeps its one-line JSON contract: the reference arm (the FP64
oracle on the host cores) on CPU, and our arm on a small sphere on the GPU.
The keys and their types are checked, not the numbers."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout):
    env = dict(os.environ, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=timeout, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def _common(d):
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"):
        assert key in d, key
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["data"] == "synthetic" and "workload" in d["config"]
    assert d["warmup"] >= 3 and d["value"] > 0
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in d["e2e"], key
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in d["cpu_baseline"], key
    assert d["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_contract():
    d = _run(["--impl", "reference", "--edge", "16", "--diameter", "16", "--steps", "1", "--warmup", "3",
              "--cpu-rows", "20"], timeout=600)
    _common(d)
    assert d["impl"] == "reference" and d["dtype"] == "f64"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["value"] == d["value"]


def test_warmup_below_three_is_refused():
    env = dict(os.environ, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--warmup", "2"],
                       capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert r.returncode != 0 and "warmup" in r.stderr


@pytest.mark.gpu
def test_our_arm_contract():
    d = _run(["--edge", "32", "--diameter", "30", "--steps", "3", "--warmup", "3", "--batch", "2",
              "--cpu-rows", "20", "--ellipsoid-matvecs", "20", "--agg-count", "1", "--agg-directions", "2"],
             timeout=900)
    _common(d)
    assert "impl" not in d and d["n_gpus"] == 1
    assert d["gpu_launches"] > 0
    for key in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert key in d["clocks"], key
    rl = d["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in rl, key
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s" and abs(rl["frac"] - rl["achieved"] / rl["peak"]) < 1e-9
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    f64 = d["fp64_roofline"]
    assert f64["bound"] == "alu" and 0 < f64["frac"]
    assert d["unpruned_cufft"]["c128"]["rel_diff_vs_library"] < 1e-12
    assert d["unpruned_cufft"]["c64"]["rel_diff_vs_library"] < 2e-5
    assert d["job"]["status"] == [0]
    # the extras of the default line: mixed against FP64 on the same right-hand
    # side (BiCGSTAB and QMR), the set-up time, the two-material ellipsoid,
    # the x passes on rows of 3 * 2^a and 5 * 2^a points and the aggregate
    # workload
    mv = d["mixed_vs_fp64"]
    for method in ("bicgstab", "qmr"):
        r = mv[method]
        assert r["mixed"]["status"] == 0 and r["fp64"]["status"] == 0
        assert r["mixed"]["rel_residual_true"] <= 1e-5 and r["fp64"]["rel_residual_true"] <= 1e-5
        assert max(r["rel_diff_cext_cabs_csca"]) < 1e-4
    assert d["context_setup"]["ms"] > 0
    for name in ("c64", "c128"):
        assert d["ellipsoid_128"][name]["matvecs_per_s"] > 0
    agg = d["aggregates"]
    assert agg["solves"] == 4 and agg["value"] > 0 and agg["aggregates"][0]["status"] == [0]
    rows = d["x_rows"]["rows"]
    assert sorted(rows, key=int) == ["160", "192", "320", "384"]
    for r in rows.values():
        assert r["P2_ms"] > 0 and r["P4_ms"] > 0 and r["P2_GBps"] > 0
    assert d["e2e"]["steps"] >= 1
    df = d["fft_matvecs"]["c128df"]
    assert df["ms"] > 0 and df["rel_diff_vs_c128"] < 1e-12
    # Table 4's workload: SPHERE 200^3, FP64 solves with point-Jacobi to 1e-10
    t4 = d["table4_sphere200"]
    assert t4["n_dipoles"] == 4188896 and t4["setup_ms"] > 0 and t4["product_ms_c128"] > 0
    for method, ni in (("bicgstab", 12), ("bicg_sym", 21), ("qmr_sym", 21)):
        r = t4[method]
        assert r["status"] == 0 and r["rel_residual_true"] <= 1e-10 and abs(r["iterations"] - ni) <= 2
        assert r["iteration_ms"] > 0 and r["device_gb"] > 0
