#!/usr/bin/env python
"""Benchmark of the DDA hot path on GB300 (one JSON line on stdout).

Workload: the large single target of the benchmark plan -- a sphere of
diameter 250 dipoles in a 256^3 lattice (N_d = 8,181,840; padded DFT grid
512^3), m = 1.33 + 0.05i, |m| k d = 0.5, Clausius-Mossotti polarisability
with radiative reaction, incidence along a seeded random direction with two
orthogonal polarisations.

One step = one whole job on that target through the C ABI:
  pack the occupancy bit field from the device mask (Sec. 2),
  build the context (ranks, alpha^-1, Green's-tensor spectrum, Sec. 3),
  for each of the two polarisations: incident field, mixed-precision
  BiCGSTAB solve to 1e-5 (complex64 FFT products inside FP64 refinement,
  Sec. 4), cross sections; then free the context.
value = products with A (FFT matvecs, any precision) per second over the
whole job, max over ranks; solves/s and the per-precision matvec rates are
reported beside it.  e2e repeats the job through the public API with host
buffers: the occupancy bits, each incident field E and each solution P
cross the host boundary inside dda_init_lattice, dda_solve and
dda_cross_sections.

Extras of the default line (rank 0, after the timed region): the roofline
of the dominant pass; complex64 and complex128 product rates; mixed against
FP64 solves of the same right-hand side with BiCGSTAB and QMR to 1e-5
(seconds, products, true residuals, the relative differences of the cross
sections); the two-material LDR ellipsoid in 128^3 with 1,000 timed products
in each precision; the context set-up (spectrum build) time; the batch of 16
directions sharing the spectrum; the x passes on rows of 160, 192, 320 and
384 points; the ballistic-aggregate batching workload; the unpruned cuFFT
comparison.

--impl reference times the oracle (plain FP64 direct sum, O(N_d^2)) on the
host cores on a bounded sample of the same product: a few hundred rows of
A p, scaled to whole products per second.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FFT-matvecs/s and solves/s at 256³ lattice, HBM GB/s vs roofline, mixed vs FP64"
UNIT = "FFT-matvecs/s"
N_EDGE, DIAM = 256, 250
M_REFR = 1.33 + 0.05j
K_WAVE = 0.5 / abs(M_REFR)
SEED = 20260005
TOL = 1e-5


def workload_name(n, d):
    return f"sphere D={d} in {n}^3 lattice, m=1.33+0.05i, |m|kd=0.5, CM+RR, 2 polarisations, mixed BiCGSTAB 1e-5"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ replicas
def replica_incidence(rank):
    """Replicas (weak scaling): rank r solves its own seeded incidence
    direction with its two orthogonal polarisations; no data is exchanged."""
    import synth
    khat = synth.random_direction(SEED + rank)[0]
    return khat, synth.orthogonal_polarisations(khat)


def reduce_over_ranks(dist, ms, totals, device):
    """Whole-job figures: the slowest rank's time and the sum of the work."""
    if dist is None:
        return ms, [float(v) for v in totals]
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tt = torch.tensor([float(v) for v in totals], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(t.item()), [float(v) for v in tt.tolist()]


# --------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    import paper_0908_0863_gb300 as dda

    n, D = args.edge, args.diameter
    mask = synth.sphere(D, box=(n, n, n))
    shape = (n, n, n)
    nsites = mask.size
    mask_dev = torch.from_numpy(mask.reshape(-1)).to(dev)
    bits = torch.empty((nsites + 31) // 32, dtype=torch.int32, device=dev)
    alpha = dda.dda_polarizability([M_REFR], K_WAVE, "cmrr")
    khat, pols = replica_incidence(rank)
    stream = torch.cuda.current_stream(dev)

    dda.dda_pack_occupancy(mask_dev, bits)
    probe = dda.Lattice(shape, bits, alpha, K_WAVE)
    nd = probe.n_dipoles
    # tile widths tuned once per process (untimed); every later context of
    # this shape starts with them
    tuned = {dt: {"pass_ms": probe.autotune(dt, nb=1, reps=3), "tiles": probe.tiles(dt)}
             for dt in ("c64", "c128")} if args.autotune else None
    if args.autotune:
        # the mixed-precision inner target, tuned on the first right-hand side
        E0 = torch.empty((3, probe.n_dipoles), dtype=torch.complex128, device=dev)
        dda.dda_incident_field(probe.ctx, khat, pols[0], E0)
        rho, rho_ms = dda.dda_autotune_inner(probe.ctx, E0, args.method, args.tol, args.max_iter)
        tuned["inner"] = {"rho": rho, "solve_ms": {str(k): v for k, v in rho_ms.items()}}
        del E0
    probe.close()
    E = torch.empty((3, nd), dtype=torch.complex128, device=dev)
    P = torch.empty_like(E)
    stats = {"matvecs": 0, "matvecs_fp64": 0, "iters": 0, "solves": 0, "refinements": 0, "worst_true": 0.0,
             "status": [], "cx": None}
    pass_ms = {"c128": [[0, 0.0] for _ in range(5)], "c64": [[0, 0.0] for _ in range(5)]}

    def job(record, host=None):
        if host is None:
            dda.dda_pack_occupancy(mask_dev, bits)
            src = bits
        else:
            src = host["bits"]
        ctx = dda.dda_init_lattice(shape, src, None, 1, alpha, K_WAVE)
        try:
            if record:
                dda.dda_profile(ctx, True)
            for q, e in enumerate(pols):
                if host is None:
                    dda.dda_incident_field(ctx, khat, e, E)
                    status, info = dda.dda_solve(ctx, E, P, args.method, "mixed", args.tol, args.max_iter)
                    cx = dda.dda_cross_sections(ctx, E, P)
                else:
                    # the caller's host arrays, as a user of the library passes them
                    Eh, Ph = host["E"][q], host["P"][q]
                    status, info = dda.dda_solve(ctx, Eh, Ph, args.method, "mixed", args.tol, args.max_iter)
                    cx = dda.dda_cross_sections(ctx, Eh, Ph)
                if record:
                    stats["matvecs"] += info["matvecs"] + info["matvecs_fp64"]
                    stats["matvecs_fp64"] += info["matvecs_fp64"]
                    stats["iters"] += info["iterations"]
                    stats["refinements"] += info["refinements"]
                    stats["solves"] += 1
                    stats["status"].append(status)
                    stats["worst_true"] = max(stats["worst_true"], info["rel_residual_true"])
                    stats["cx"] = cx
            if record:
                prof = dda.dda_profile_read(ctx)
                for dt in prof:
                    for q, (c, ms) in enumerate(prof[dt]):
                        pass_ms[dt][q][0] += c
                        pass_ms[dt][q][1] += ms
        finally:
            dda.dda_free(ctx)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        job(False)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = dda.dda_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.profiler.start()   # profiler range = the timed steps (no-op without a profiler)
    ev0.record(stream)
    for _ in range(args.steps):
        job(True)
    ev1.record(stream)
    barrier()
    torch.cuda.profiler.stop()
    clocks = sampler.stop()
    launches = dda.dda_launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    ms_max, totals = reduce_over_ranks(dist, ms, [stats["matvecs"], stats["solves"]], dev)
    value = totals[0] / (ms_max / 1e3)
    solves_per_s = totals[1] / (ms_max / 1e3)

    # ---- end to end through the public API with host buffers (pinned): the
    # occupancy bits and both incident fields go in, both solutions come
    # out, every step, inside the library calls
    host = {"bits": torch.empty(bits.numel(), dtype=torch.int32).pin_memory(),
            "E": [torch.empty(E.shape, dtype=E.dtype).pin_memory() for _ in pols],
            "P": [torch.empty(P.shape, dtype=P.dtype).pin_memory() for _ in pols]}
    host["bits"].copy_(bits.cpu())
    ctx0 = dda.dda_init_lattice(shape, bits, None, 1, alpha, K_WAVE)
    for q, e in enumerate(pols):
        dda.dda_incident_field(ctx0, khat, e, E)
        host["E"][q].copy_(E.cpu())
    dda.dda_free(ctx0)
    hostnp = {"bits": host["bits"].numpy(), "E": [t.numpy() for t in host["E"]], "P": [t.numpy() for t in host["P"]]}
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        job(False, host=hostnp)
    barrier()
    e2e_s = time.perf_counter() - t0
    # a job makes the same products as in the timed loop; ranks run replicas
    per_job_mv = stats["matvecs"] / max(1, args.steps)
    e2e_value = per_job_mv * e2e_steps / e2e_s * world
    # per step: bits, then per polarisation E into dda_solve and E, P into
    # dda_cross_sections; P out of dda_solve and the three cross sections
    h2d = host["bits"].numel() * 4 + len(pols) * (2 * E.numel() * 16 + P.numel() * 16)
    d2h = len(pols) * (P.numel() * 16 + 3 * 8)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64 (complex64 FFT products, FP64 refinement)",
        "data": "synthetic",
        "config": {"workload": workload_name(n, D), "lattice": [n, n, n], "padded": [2 * n] * 3, "n_dipoles": nd,
                   "method": args.method, "precision": "mixed", "tol": args.tol, "polarisations": 2,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2 (working set ~15 GB per job)"},
        "solves_per_s": solves_per_s,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps, "how": "the same job through dda_init_lattice, dda_solve and "
                                          "dda_cross_sections with pinned host buffers (bits, E in, P out)"},
        "job": {"matvecs_per_solve": stats["matvecs"] / max(1, stats["solves"]),
                "fp64_matvecs_per_solve": stats["matvecs_fp64"] / max(1, stats["solves"]),
                "iterations_per_solve": stats["iters"] / max(1, stats["solves"]),
                "refinements_per_solve": stats["refinements"] / max(1, stats["solves"]),
                "worst_true_rel_residual": stats["worst_true"], "status": sorted(set(stats["status"])),
                "cross_sections_last": stats["cx"]},
    }
    result["passes"] = {dt: [{"launches": c, "ms_avg": (t / c if c else None)} for c, t in pass_ms[dt]]
                        for dt in pass_ms}
    if tuned:
        result["autotune"] = tuned
    if rank == 0 and not args.no_extras:
        result.update(extras(args, dda, torch, dev, shape, bits, alpha, nd, pass_ms, khat, pols, mask))
    if rank == 0 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(args, nd, mask)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def algorithmic_bytes(n, nd, esize):
    """Bytes each matvec pass must move at least (complex element size esize)."""
    K = J = P = n
    Lx = Ly = Lz = 2 * n
    Hx = Hy = Hz = n + 1
    V = 3 * nd * esize                      # compressed vector
    A = 3 * K * Ly * P * esize              # y-transformed volume
    B = 3 * Lx * Ly * P * esize             # xy-transformed volume
    T = 6 * Hx * Hy * Hz * esize            # half spectrum
    return {"P1": V + A, "P2": A + B, "P3": 2 * B + T, "P4": B + A, "P5": A + 2 * V,
            "matvec_min": 3 * V + 4 * A + T}


def matvec_flops(n):
    """Algorithmic flops of one product at lattice edge n (padded L = 2n per
    axis): 5 L log2 L per transformed line over the pruned line counts of the
    five passes, plus 84 per point of the padded grid for the spectrum
    product (Eqs. 6-8)."""
    K = J = P = n
    L = 2 * n
    lines = 3 * K * P + 3 * L * P + 2 * 3 * L * L + 3 * L * P + 3 * K * P
    return lines * 5 * L * math.log2(L) + 84 * L ** 3


def fp64_peak_tflops(torch, dev, size=8192, reps=3):
    """Dense FP64 rate of this GPU: cuBLAS DGEMM (torch.matmul, float64)."""
    a = torch.randn((size, size), dtype=torch.float64, device=dev)
    b = torch.randn_like(a)
    torch.matmul(a, b)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        torch.matmul(a, b)
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    del a, b
    return 2.0 * size ** 3 / (ms / 1e3) / 1e12


# what the P3 traffic figure depends on: the P3 section of the kernel header
# (from its P3 banner to the P5 banner) and the headers it includes
KERNEL_SOURCES = ("fft_reg.cuh", "fft.cuh", "matvec.cuh", "common.cuh")
P3_SECTION = ("// ---------------------------------------------------------------- P3",
              "// ---------------------------------------------------------------- P5")


def kernel_sources_hash():
    """First 16 hex digits of the SHA-256 of the z-pass kernel source: the P3
    section of csrc/matvec_kernels.cuh followed by KERNEL_SOURCES."""
    import hashlib
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_0908_0863_gb300/csrc/matvec_kernels.cuh")) as f:
        text = f.read()
    a, b = text.index(P3_SECTION[0]), text.index(P3_SECTION[1])
    h.update(text[a:b].encode())
    for rel in (f"paper_0908_0863_gb300/csrc/{f}" for f in KERNEL_SOURCES):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` at the bench size, from the ncu
    summaries under profiles/ ("traffic-bench:" lines), or None when no
    summary covers it or the kernel sources changed since the capture."""
    pdir = os.path.join(ROOT, "profiles")
    try:
        names = sorted(os.listdir(pdir))
    except OSError:
        return None
    want = kernel_sources_hash()
    pat = re.compile(r"traffic-bench: kernel=(.+?) bytes=(\d+) sources=([0-9a-f]+)")
    for name in names:
        if not name.endswith(".md"):
            continue
        with open(os.path.join(pdir, name)) as f:
            for m in pat.finditer(f.read()):
                if m.group(1) == kernel and m.group(3) == want:
                    return {"bytes": int(m.group(2)), "source": f"profiles/{name}"}
    return None


def extras(args, dda, torch, dev, shape, bits, alpha, nd, pass_ms, khat, pols, mask):
    """Roofline of the dominant kernel, per-precision matvec rates, FP64 solve."""
    out = {}
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    peak_note = "of measured" if "hbm_gbs" in peaks else "of fallback"
    # dominant pass by summed device time inside the timed steps
    best = None
    for dt, arr in pass_ms.items():
        for q, (c, t) in enumerate(arr):
            if c and (best is None or t > best[3]):
                best = (dt, q, c, t)
    if best:
        dt, q, c, t = best
        esize = 16 if dt == "c128" else 8
        ab = algorithmic_bytes(args.edge, nd, esize)[f"P{q + 1}"]
        avg = t / c
        achieved = ab / (avg / 1e3) / 1e9
        kernel = f"P{q + 1} ({dt})"
        traffic = measured_traffic(kernel) if args.edge == N_EDGE else None
        out["roofline"] = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": hbm,
                           "unit": "GB/s", "frac": achieved / hbm,
                           "traffic": traffic["bytes"] if traffic else None,
                           "traffic_source": traffic["source"] if traffic else None,
                           "algorithmic_bytes": ab, "avg_ms": avg, "launches": c, "peak_source": peak_note}
    # separate device-timed matvec loops (outside the timed region)
    ctx = dda.dda_init_lattice(shape, bits, None, 1, alpha, K_WAVE)
    try:
        rates = {}
        for name, dtype, reps in (("c64", torch.complex64, 20), ("c128", torch.complex128, 3)):
            p = torch.randn((3, nd), dtype=dtype, device=dev)
            y = torch.empty_like(p)
            dda.dda_matvec(ctx, p, y)
            torch.cuda.synchronize(dev)
            dda.dda_profile(ctx, True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                dda.dda_matvec(ctx, p, y)
            e1.record()
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            prof = dda.dda_profile_read(ctx)[name]
            dda.dda_profile(ctx, False)
            ab = algorithmic_bytes(args.edge, nd, 16 if name == "c128" else 8)
            rates[name] = {"matvecs_per_s": 1e3 / ms, "ms": ms,
                           "algorithmic_GBps": ab["matvec_min"] / (ms / 1e3) / 1e9,
                           "five_pass_GBps": sum(ab[f"P{i}"] for i in range(1, 6)) / (ms / 1e3) / 1e9,
                           "pass_ms": [t / c if c else None for c, t in prof]}
            del p, y
        # the double-float product of the mixed refinement's residuals
        # (complex128 in and out), against the FP64 product of the same vector
        p = torch.randn((3, nd), dtype=torch.complex128, device=dev)
        y, y64 = torch.empty_like(p), torch.empty_like(p)
        dda.dda_matvec(ctx, p, y64)
        dda.dda_matvec(ctx, p, y, dtype="c128df")
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            dda.dda_matvec(ctx, p, y, dtype="c128df")
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / 3
        rates["c128df"] = {"matvecs_per_s": 1e3 / ms, "ms": ms,
                           "rel_diff_vs_c128": float((y - y64).norm() / y64.norm()),
                           "what": "double-float product (float pairs), complex128 in and out"}
        del p, y, y64
        out["fft_matvecs"] = rates
        # the complex128 product is FP64-ALU-bound: its algorithmic flops
        # against the DGEMM rate measured here
        peak64 = fp64_peak_tflops(torch, dev)
        fl = matvec_flops(args.edge)
        ach = fl / (rates["c128"]["ms"] / 1e3) / 1e12
        out["fp64_roofline"] = {"bound": "alu", "kernel": "c128 matvec (P1-P5)", "achieved": ach, "peak": peak64,
                                "unit": "TFLOP/s", "frac": ach / peak64, "flops_per_matvec": fl,
                                "peak_source": "cuBLAS DGEMM 8192^3 (torch.matmul, float64) measured in this run"}
        if args.fp64_solve:
            out["mixed_vs_fp64"] = mixed_vs_fp64(dda, torch, dev, ctx, nd, khat, pols[0], args)
        for meth in [m for m in args.also_methods.split(",") if m]:
            out.setdefault("other_methods", {})[meth] = timed_single_solve(dda, torch, dev, ctx, nd, khat, pols[0],
                                                                           meth, args)
        if args.batch > 0:
            out["batch"] = timed_batch(dda, torch, dev, ctx, nd, args)
        if args.unpruned:
            out["unpruned_cufft"] = timed_unpruned(dda, torch, dev, ctx, mask, alpha, nd)
    finally:
        dda.dda_free(ctx)
    out["context_setup"] = timed_setup(dda, torch, dev, shape, bits, alpha)
    if args.ellipsoid_matvecs > 0:
        out["ellipsoid_128"] = ellipsoid_matvecs(dda, torch, dev, args.ellipsoid_matvecs, hbm)
    if args.row_sweep:
        out["x_rows"] = x_pass_rows(dda, torch, dev, hbm)
    if args.aggregates:
        out["aggregates"] = aggregates_workload(dda, torch, dev, args, extra=True)
    if args.table4:
        out["table4_sphere200"] = table4_sphere200(dda, torch, dev, args)
    return out


def timed_solve(dda, torch, dev, ctx, E, method, precision, args):
    """One solve of A P = E (device) from zero; seconds by host wall clock
    around the synchronising call."""
    P = torch.empty_like(E)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    status, info = dda.dda_solve(ctx, E, P, method, precision, args.tol, args.max_iter)
    dt = time.perf_counter() - t0
    cx = dda.dda_cross_sections(ctx, E, P)
    rec = {"method": method, "precision": precision, "seconds": dt, "solves_per_s": 1.0 / dt, "status": status,
           "iterations": info["iterations"], "matvecs": info["matvecs"], "matvecs_fp64": info["matvecs_fp64"],
           "refinements": info["refinements"], "rel_residual_true": info["rel_residual_true"],
           "cross_sections": cx}
    return rec, P


def mixed_vs_fp64(dda, torch, dev, ctx, nd, khat, e0, args):
    """The bench target's first right-hand side solved to the bench tolerance
    with BiCGSTAB and QMR, each in mixed precision (complex64 products in
    FP64 refinement, the method's own tuned inner target) and in FP64: time,
    products, true residual (one FP64 product), and the mixed result's
    relative difference from the FP64 one in C_ext, C_abs, C_sca and in P."""
    E = torch.empty((3, nd), dtype=torch.complex128, device=dev)
    dda.dda_incident_field(ctx, khat, e0, E)
    res = {"tol": args.tol, "what": "same right-hand side, BiCGSTAB and QMR, mixed and FP64"}
    for method in ("bicgstab", "qmr"):
        if args.autotune and method != args.method:
            # each method's own inner target (untimed), as the job's method has
            dda.dda_autotune_inner(ctx, E, method, args.tol, args.max_iter)
        mixed, Pm = timed_solve(dda, torch, dev, ctx, E, method, "mixed", args)
        mixed["inner_rho"] = dda.dda_inner_tolerance(ctx, method=method)
        fp64, Pf = timed_solve(dda, torch, dev, ctx, E, method, "fp64", args)
        diff = [abs(a / b - 1.0) for a, b in zip(mixed["cross_sections"], fp64["cross_sections"])]
        pdiff = float((Pm - Pf).norm() / Pf.norm())
        res[method] = {"mixed": mixed, "fp64": fp64, "speedup_mixed_over_fp64": fp64["seconds"] / mixed["seconds"],
                       "rel_diff_cext_cabs_csca": diff, "rel_diff_P": pdiff}
        del Pm, Pf
    del E
    return res


def timed_setup(dda, torch, dev, shape, bits, alpha, reps=3):
    """Context set-up of the bench target (ranks, alpha^-1 table, the FP64
    Green's-tensor spectrum build with its complex64 copy, workspace), the
    step the paper times as tensor creation + DFT (Table 4)."""
    ms = []
    for r in range(reps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx = dda.dda_init_lattice(shape, bits, None, 1, alpha, K_WAVE)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        dda.dda_free(ctx)
        if r:
            ms.append(dt * 1e3)
    return {"ms": statistics.median(ms), "samples_ms": ms,
            "what": "dda_init_lattice at 256^3 (padded 512^3): device allocations, ranks, alpha^-1, spectrum "
                    "(section 1 + x/y/z line DFTs in FP64, complex64 copy)"}


# The paper's solver benchmark target (Sec. 6, Tables 3 and 4): SPHERE 200^3
# (N_d = 4,188,896), size parameter x = 0.98948, m = 1.63631 + 0.372i,
# point-Jacobi, tol 1e-10, x0 = 0; Table 4 prints, per scheme, the serial
# (one NEMO core) and 4-thread times per iteration and per product, the
# tensor set-up (creation + DFT) and the memory, all in FP64.
T4_N = 200
T4_X = 0.98948
T4_M = 1.63631 + 0.372j
T4_TOL = 1e-10
T4_PAPER = {"bicgstab": {"iteration_s": 68.3, "product_s": 32.7, "memory_gb": 3.1},
            "bicg_sym": {"iteration_s": 33.9, "product_s": 32.4, "memory_gb": 2.6},
            "qmr_sym": {"iteration_s": 35.1, "product_s": 33.1, "memory_gb": 3.1},
            "tensor_setup_s": 13.4, "omp4_tensor_setup_s": 3.8}


def table4_sphere200(dda, torch, dev, args):
    """Table 4's workload on the GPU: context set-up (the tensor creation +
    DFT step), FP64 and complex64 products, and FP64 solves with point-Jacobi
    to 1e-10 by BiCGSTAB, BiCG_sym and QMR_sym (time per iteration = solve
    time / iterations; products per iteration from the solver's count), with
    the device memory of the context, beside the paper's serial figures."""
    import synth
    mask = synth.sphere(T4_N)
    nd = int(mask.sum())
    a_eff = (3.0 * nd / (4.0 * math.pi)) ** (1.0 / 3.0)     # effective radius, lattice spacing 1
    k = T4_X / a_eff
    alpha = dda.dda_polarizability([T4_M], k, "ldr", [0, 0, 1], [1, 0, 0])
    shape = (T4_N,) * 3
    mask_dev = torch.from_numpy(mask.reshape(-1)).to(dev)
    bits = torch.empty((mask.size + 31) // 32, dtype=torch.int32, device=dev)
    dda.dda_pack_occupancy(mask_dev, bits)
    del mask_dev
    setup = []
    for r in range(3):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx = dda.dda_init_lattice(shape, bits, None, 1, alpha, k)
        torch.cuda.synchronize(dev)
        if r:
            setup.append((time.perf_counter() - t0) * 1e3)
        if r < 2:
            dda.dda_free(ctx)
    out = {"what": "SPHERE 200^3, x = 0.98948, m = 1.63631+0.372i, LDR, point-Jacobi, FP64 solves to 1e-10 from "
                   "x0 = 0 (Sec. 6, Tables 3 and 4); paper: one NEMO core, FP64",
           "n_dipoles": nd, "setup_ms": statistics.median(setup), "paper": T4_PAPER}
    try:
        E = torch.empty((3, nd), dtype=torch.complex128, device=dev)
        dda.dda_incident_field(ctx, [0, 0, 1], [1, 0, 0], E)
        for name, dtype, reps in (("c128", torch.complex128, 5), ("c64", torch.complex64, 20)):
            p = E.to(dtype)
            y = torch.empty_like(p)
            dda.dda_matvec(ctx, p, y)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                dda.dda_matvec(ctx, p, y)
            e1.record()
            torch.cuda.synchronize(dev)
            out[f"product_ms_{name}"] = e0.elapsed_time(e1) / reps
            del p, y
        P = torch.empty_like(E)
        for method in ("bicgstab", "bicg_sym", "qmr_sym"):
            P.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            status, info = dda.dda_solve(ctx, E, P, method + "+jacobi", "fp64", T4_TOL, 10000)
            dt = time.perf_counter() - t0
            q = dda.dda_query(ctx)
            out[method] = {"status": status, "seconds": dt, "iterations": info["iterations"],
                           "matvecs": info["matvecs"], "iteration_ms": dt * 1e3 / max(1, info["iterations"]),
                           "rel_residual_true": info["rel_residual_true"],
                           "device_gb": q["device_bytes"] / 1e9,
                           "speedup_per_iteration_vs_paper_serial":
                               T4_PAPER[method]["iteration_s"] * 1e3 / (dt * 1e3 / max(1, info["iterations"]))}
        out["speedup_product_vs_paper_serial"] = T4_PAPER["bicgstab"]["product_s"] * 1e3 / out["product_ms_c128"]
        del E, P
    finally:
        dda.dda_free(ctx)
    return out


ELL_SEED = 20260002
ELL_M = (1.5 + 0.01j, 1.7 + 0.1j)


def ellipsoid_matvecs(dda, torch, dev, reps, hbm):
    """The matvec-throughput workload: a seeded random ellipsoid (semi-axes
    uniform in 0.6-1.0 x 64) in a 128^3 lattice, two materials (m1 = 1.5 +
    0.01i, m2 = 1.7 + 0.1i by a Bernoulli(0.3) draw, one composition bit),
    LDR with |m2| k d = 0.8, p complex normal; `reps` timed products in
    complex64 and in complex128 after 10 untimed ones (CUDA events)."""
    import numpy as np

    import synth
    mask, axes = synth.random_ellipsoid(ELL_SEED, 128)
    mats = synth.bernoulli_materials(ELL_SEED + 1, mask, 0.3)
    k = 0.8 / abs(ELL_M[1])
    alpha = dda.dda_polarizability(list(ELL_M), k, "ldr", [0, 0, 1], [1, 0, 0])
    n = mask.size
    md = torch.from_numpy(mask.reshape(-1)).to(dev)
    bits = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    dda.dda_pack_occupancy(md, bits)
    matd = torch.from_numpy(np.ascontiguousarray(mats.reshape(-1))).to(dev)
    cbits = torch.empty((3 * n + 31) // 32, dtype=torch.int32, device=dev)
    dda.dda_pack_composition(matd, n, 2, cbits)
    ctx = dda.dda_init_lattice((128, 128, 128), bits, cbits, 2, alpha, k)
    out = {"what": f"ellipsoid semi-axes {tuple(round(a, 2) for a in axes)} in 128^3, two materials "
                   "(Bernoulli 0.3), LDR, |m2|kd = 0.8", "reps": reps}
    try:
        nd = dda.dda_query(ctx)["n_dipoles"]
        out["n_dipoles"] = nd
        g = torch.Generator(device="cpu").manual_seed(ELL_SEED)
        for name, dtype in (("c64", torch.complex64), ("c128", torch.complex128)):
            p = torch.randn((3, nd), dtype=dtype, generator=g).to(dev)
            y = torch.empty_like(p)
            for _ in range(10):
                dda.dda_matvec(ctx, p, y)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                dda.dda_matvec(ctx, p, y)
            e1.record()
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            es = 16 if name == "c128" else 8
            ab = algorithmic_bytes(128, nd, es)
            out[name] = {"matvecs_per_s": 1e3 / ms, "ms": ms,
                         "algorithmic_GBps": ab["matvec_min"] / (ms / 1e3) / 1e9,
                         "five_pass_GBps": sum(ab[f"P{i}"] for i in range(1, 6)) / (ms / 1e3) / 1e9,
                         "five_pass_frac_of_hbm": sum(ab[f"P{i}"] for i in range(1, 6)) / (ms / 1e3) / 1e9 / hbm}
            del p, y
    finally:
        dda.dda_free(ctx)
    return out


# x edges whose rows pad to 3 * 2^a and 5 * 2^a points (160, 192, 320, 384)
ROW_EDGES = (80, 96, 160, 192)


def x_pass_rows(dda, torch, dev, hbm, reps=20):
    """The x passes (P2 forward, P4 inverse) on rows of 3 * 2^a and 5 * 2^a
    points: full K x 128 x 128 boxes, K in ROW_EDGES, complex64, default
    tiles, `reps` products after 3 untimed ones; device time per pass from
    the library's CUDA events, GB/s of the algorithmic bytes A + B."""
    import numpy as np
    out = {"what": "P2/P4 on K x 128 x 128 full boxes (rows of 160, 192, 320, 384 points), complex64, "
                   "algorithmic bytes A + B per pass", "rows": {}}
    m = 1.33 + 0.05j
    k = 0.5 / abs(m)
    alpha = dda.dda_polarizability([m], k, "cmrr")
    for K in ROW_EDGES:
        J = P = 128
        mask = np.ones((P, J, K), dtype=np.uint8)
        md = torch.from_numpy(mask.reshape(-1)).to(dev)
        bits = torch.empty((mask.size + 31) // 32, dtype=torch.int32, device=dev)
        dda.dda_pack_occupancy(md, bits)
        ctx = dda.dda_init_lattice((K, J, P), bits, None, 1, alpha, k)
        try:
            q = dda.dda_query(ctx)
            nd = q["n_dipoles"]
            Lx, Ly, _ = q["padded"]
            g = torch.Generator(device="cpu").manual_seed(SEED + K)
            p = torch.randn((3, nd), dtype=torch.complex64, generator=g).to(dev)
            y = torch.empty_like(p)
            for _ in range(3):
                dda.dda_matvec(ctx, p, y)
            torch.cuda.synchronize(dev)
            dda.dda_profile(ctx, True)
            for _ in range(reps):
                dda.dda_matvec(ctx, p, y)
            torch.cuda.synchronize(dev)
            prof = dda.dda_profile_read(ctx)["c64"]
            dda.dda_profile(ctx, False)
            ms = [t / c for c, t in prof]
            b = 3 * Ly * P * (K + Lx) * 8
            out["rows"][str(Lx)] = {"lattice": [K, J, P], "P2_ms": ms[1], "P4_ms": ms[3],
                                    "P2_GBps": b / (ms[1] / 1e3) / 1e9, "P4_GBps": b / (ms[3] / 1e3) / 1e9,
                                    "P2_frac_of_hbm": b / (ms[1] / 1e3) / 1e9 / hbm,
                                    "tiles": list(dda.dda_tiles(ctx, "c64"))}
            del p, y
        finally:
            dda.dda_free(ctx)
    return out


def timed_single_solve(dda, torch, dev, ctx, nd, khat, e0, method, args):
    """One mixed-precision solve of the bench target with another method."""
    E = torch.empty((3, nd), dtype=torch.complex128, device=dev)
    P = torch.empty_like(E)
    dda.dda_incident_field(ctx, khat, e0, E)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    status, info = dda.dda_solve(ctx, E, P, method, "mixed", args.tol, args.max_iter)
    dt = time.perf_counter() - t0
    return {"method": method, "seconds": dt, "solves_per_s": 1.0 / dt, "status": status,
            "iterations": info["iterations"], "matvecs": info["matvecs"], "matvecs_fp64": info["matvecs_fp64"],
            "rel_residual_true": info["rel_residual_true"]}


def timed_batch(dda, torch, dev, ctx, nd, args):
    """args.batch incidence directions (first polarisation of each) solved
    together in one batched mixed-precision solve sharing the spectrum."""
    import synth
    nbt = args.batch
    dirs = synth.random_direction(SEED + 1000, nbt)
    E = torch.empty((nbt, 3, nd), dtype=torch.complex128, device=dev)
    for b, kh in enumerate(dirs):
        dda.dda_incident_field(ctx, kh, synth.orthogonal_polarisations(kh)[0], E[b])
    P = torch.zeros_like(E)
    dda.dda_reserve(ctx, nbt, "mixed")
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    l0 = dda.dda_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    status, stats, infos = dda.dda_solve_batch(ctx, E, P, args.method, "mixed", args.tol, args.max_iter)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    launches = dda.dda_launch_count() - l0
    cx = dda.dda_cross_sections_batch(ctx, E, P)
    mv = sum(i["matvecs"] + i["matvecs_fp64"] for i in infos)
    return {"rhs": nbt, "what": f"{nbt} seeded incidence directions, first polarisation each, "
                                "one dda_solve_batch call (mixed, shared spectrum)",
            "seconds": ms / 1e3, "solves_per_s": nbt / (ms / 1e3), "matvecs_per_s": mv / (ms / 1e3),
            "iterations": [i["iterations"] for i in infos], "refinements": [i["refinements"] for i in infos],
            "worst_true_rel_residual": max(i["rel_residual_true"] for i in infos),
            "status": sorted(set(stats)), "gpu_launches": int(launches),
            "device_bytes": dda.dda_query(ctx)["device_bytes"],
            "c_ext_range": [float(cx[:, 0].min()), float(cx[:, 0].max())]}


# --------------------------------------------- unpruned cuFFT comparison
class UnprunedFFT:
    """Same-GPU comparison arm: the product y = A p done with unpruned 3-D
    FFTs (cuFFT, through torch.fft) on the whole zero-padded grid
    2K x 2J x 2P -- three forward transforms of the padded components, the
    6-component spectrum product of Eqs. 6-8 at every frequency, three
    inverse transforms, then the diagonal alpha^-1 p (Sec. 3).  Nothing is
    pruned: every transform runs over all lines of all three axes.  It builds
    its own spectrum from the interaction tensor, so it also checks the
    library's product independently.  Timed beside the library's path, never
    used by it.

    mask: bool [P][J][K] occupancy (x fastest); ainv: complex alpha^-1 per
    occupied site and axis, shape [3][N_d] or broadcastable to it."""

    def __init__(self, torch, dev, mask, ainv, k, cdtype):
        import numpy as np
        self.torch = torch
        P, J, K = mask.shape
        self.L = (2 * P, 2 * J, 2 * K)
        self.cdtype = cdtype
        z, y, x = np.nonzero(mask)     # C order = x-fastest site order
        L0, L1, L2 = self.L
        self.idx = torch.from_numpy((z * L1 + y) * L2 + x).to(dev)
        self.ainv = torch.as_tensor(ainv, dtype=cdtype, device=dev)
        self.Y = self._spectrum(torch, dev, (P, J, K), k)
        self.X = torch.zeros((3,) + self.L, dtype=cdtype, device=dev)
        self.Q = torch.empty_like(self.X)

    def _spectrum(self, torch, dev, n, k):
        """DFT of t = -G on the padded grid: displacement i for i < n,
        i - 2n for i > n, zero at i = n (the extension element) and at r = 0."""
        f64 = torch.float64
        axes = []
        for na, La in zip(n, self.L):
            i = torch.arange(La, dtype=f64, device=dev)
            d = torch.where(i < na, i, i - La)
            axes.append((d, i == na))
        (z, zn), (y, yn), (x, xn) = axes
        z, y, x = z.view(-1, 1, 1), y.view(1, -1, 1), x.view(1, 1, -1)
        r2 = z * z + y * y + x * x
        dead = (r2 == 0) | zn.view(-1, 1, 1) | yn.view(1, -1, 1) | xn.view(1, 1, -1)
        r2 = torch.where(dead, torch.ones_like(r2), r2)
        r = torch.sqrt(r2)
        ikr = torch.complex(torch.zeros_like(r), k * r)
        e = torch.exp(ikr) / (r2 * r)
        # G_ab = a delta_ab + b x_a x_b, t = -G
        a = -(e * (k * k * r2 - 1.0 + ikr))
        b = -(e * ((3.0 - 3.0 * ikr) / r2 - k * k))
        a = torch.where(dead, torch.zeros_like(a), a)
        b = torch.where(dead, torch.zeros_like(b), b)
        del r, ikr, e
        comp = {"x": x, "y": y, "z": z}
        Y = []
        for m in ("xx", "xy", "xz", "yy", "yz", "zz"):
            t = b * (comp[m[0]] * comp[m[1]])
            if m[0] == m[1]:
                t = t + a
            Y.append(torch.fft.fftn(t.to(self.cdtype), dim=(0, 1, 2)))
            del t
        return Y

    def matvec(self, p):
        torch = self.torch
        X, Q, Y = self.X, self.Q, self.Y
        X.zero_()
        X.view(3, -1)[:, self.idx] = p
        F = torch.fft.fftn(X, dim=(1, 2, 3))
        for a, row in enumerate(((0, 1, 2), (1, 3, 4), (2, 4, 5))):
            torch.mul(Y[row[0]], F[0], out=Q[a])
            Q[a].addcmul_(Y[row[1]], F[1])
            Q[a].addcmul_(Y[row[2]], F[2])
        del F
        q = torch.fft.ifftn(Q, dim=(1, 2, 3))
        return self.ainv * p + q.view(3, -1)[:, self.idx]


def timed_unpruned(dda, torch, dev, ctx, mask, alpha, nd):
    """ms per product of the unpruned cuFFT arm against the library's
    product on the same random p, with their relative difference."""
    out = {}
    ainv = torch.full((3, 1), 1.0 / complex(alpha[0, 0]), dtype=torch.complex128)
    for name, dtype, reps in (("c64", torch.complex64, 5), ("c128", torch.complex128, 2)):
        arm = UnprunedFFT(torch, dev, mask, ainv, K_WAVE, dtype)
        p = torch.randn((3, nd), dtype=dtype, device=dev)
        y = torch.empty_like(p)
        dda.dda_matvec(ctx, p, y)
        z = arm.matvec(p)
        torch.cuda.synchronize(dev)
        diff = float((z - y).norm() / y.norm())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            arm.matvec(p)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": ms, "matvecs_per_s": 1e3 / ms, "rel_diff_vs_library": diff}
        del arm, p, y, z
        torch.cuda.empty_cache()
    out["what"] = ("unpruned 3-D cuFFT (torch.fft) on the whole padded grid: 3 forward + 6-component "
                   "spectrum product + 3 inverse, scatter/gather and diagonal included; not the product path")
    return out


# ------------------------------------------------------------ aggregates
AGG_MONOMERS = (20, 45, 70, 95, 120, 145, 170, 200)
AGG_REFR = 1.6 + 0.05j
AGG_SEED = 20260003


def aggregates_workload(dda, torch, dev, args, extra=False):
    """Batching workload: 8 seeded ballistic aggregates of touching spheres
    (monomer diameter 8, 20-200 monomers, uneven lattices), each solved for
    64 seeded incidence directions x 2 polarisations in one batched
    mixed-precision call sharing that aggregate's spectrum; per-orientation
    C_ext and C_abs.  Returns the timed figures (CUDA events around the
    solves of all aggregates, context set-up included); extra=True (inside
    the default bench line) times one pass after one warm-up and skips the
    single-call comparison."""
    import numpy as np

    import synth

    k = 0.5 / abs(AGG_REFR)
    alpha = dda.dda_polarizability([AGG_REFR], k, "cmrr")
    ndir = args.agg_directions
    targets = []
    for i, nm in enumerate(AGG_MONOMERS[:args.agg_count]):
        mask, _ = synth.ballistic_aggregate(AGG_SEED + nm, nm, mono_diameter=8)
        dirs = synth.random_direction(AGG_SEED + 1000 + i, ndir)
        pairs = []
        for kh in dirs:
            e1, e2 = synth.orthogonal_polarisations(kh)
            pairs += [(kh, e1), (kh, e2)]
        targets.append((nm, mask, pairs))

    def solve_target(nm, mask, pairs, detail):
        P_, J_, K_ = mask.shape
        m_dev = torch.from_numpy(np.ascontiguousarray(mask).reshape(-1)).to(dev)
        bits = torch.empty((mask.size + 31) // 32, dtype=torch.int32, device=dev)
        dda.dda_pack_occupancy(m_dev, bits)
        ctx = dda.dda_init_lattice((K_, J_, P_), bits, None, 1, alpha, k)
        try:
            nd = dda.dda_query(ctx)["n_dipoles"]
            nb = len(pairs)
            E = torch.empty((nb, 3, nd), dtype=torch.complex128, device=dev)
            for b, (kh, e) in enumerate(pairs):
                dda.dda_incident_field(ctx, kh, e, E[b])
            P = torch.zeros_like(E)
            status, stats, infos = dda.dda_solve_batch(ctx, E, P, args.agg_method, "mixed", args.tol, args.max_iter)
            cx = dda.dda_cross_sections_batch(ctx, E, P)
            if detail is not None:
                q = dda.dda_query(ctx)
                detail.append({"monomers": nm, "lattice": [K_, J_, P_], "padded": list(q["padded"]),
                               "n_dipoles": nd, "rhs": nb, "status": sorted(set(stats)),
                               "iterations_mean": float(np.mean([i["iterations"] for i in infos])),
                               "matvecs": int(sum(i["matvecs"] + i["matvecs_fp64"] for i in infos)),
                               "worst_true_rel_residual": max(i["rel_residual_true"] for i in infos),
                               "q_ext_mean": float(np.mean(cx[:, 0])) / (np.pi * (3 * nd / (4 * np.pi)) ** (2 / 3)),
                               "tiles_c64": list(dda.dda_tiles(ctx, "c64")),
                               "device_bytes": q["device_bytes"]})
            return sum(i["matvecs"] + i["matvecs_fp64"] for i in infos), len(pairs)
        finally:
            dda.dda_free(ctx)

    if args.autotune:
        # tile widths per aggregate shape, tuned once before the timed region
        for nm, mask, _ in targets:
            P_, J_, K_ = mask.shape
            m_dev = torch.from_numpy(np.ascontiguousarray(mask).reshape(-1)).to(dev)
            bits = torch.empty((mask.size + 31) // 32, dtype=torch.int32, device=dev)
            dda.dda_pack_occupancy(m_dev, bits)
            ctx = dda.dda_init_lattice((K_, J_, P_), bits, None, 1, alpha, k)
            try:
                dda.dda_autotune(ctx, "c64", nb=8, reps=2)
            finally:
                dda.dda_free(ctx)
    warm = 1 if extra else args.warmup
    steps = 1 if extra else args.steps
    for _ in range(warm):
        solve_target(targets[0][0], targets[0][1], targets[0][2][:4], None)
    torch.cuda.synchronize(dev)
    sampler = None
    if not extra:
        sampler = ClockSampler(0)
        sampler.start()
    l0 = dda.dda_launch_count()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    detail = []
    mv = solves = 0
    if not extra:
        torch.cuda.profiler.start()   # profiler range = the timed steps (no-op without a profiler)
    e0.record(stream)
    for _ in range(steps):
        for nm, mask, pairs in targets:
            a, b = solve_target(nm, mask, pairs, detail if len(detail) < len(targets) else None)
            mv += a
            solves += b
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if not extra:
        torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1)
    out = {"value": solves / (ms / 1e3), "unit": "solves/s", "ms_per_step": ms / steps, "steps": steps,
           "solves": solves, "matvecs_per_s": mv / (ms / 1e3), "gpu_launches": int(dda.dda_launch_count() - l0),
           "method": args.agg_method, "precision": "mixed", "tol": args.tol,
           "workload": f"{len(targets)} ballistic aggregates ({', '.join(str(t[0]) for t in targets)} monomers of "
                       f"diameter 8), m=1.6+0.05i, |m|kd=0.5, CM+RR, {ndir} directions x 2 polarisations each, "
                       f"one dda_solve_batch per aggregate",
           "aggregates": detail}
    if sampler is not None:
        out["clocks"] = sampler.stop()
    if not extra:
        # the same solves one right-hand side per call, on a sample of 8
        nm, mask, pairs = targets[-1]
        t0 = time.perf_counter()
        solve_target(nm, mask, pairs[:8], None)
        t_batched8 = time.perf_counter() - t0
        t0 = time.perf_counter()
        for pr in pairs[:8]:
            solve_target(nm, mask, [pr], None)
        t_single8 = time.perf_counter() - t0
        out["batched_vs_single_8rhs_largest"] = {"batched_s": t_batched8, "single_calls_s": t_single8,
                                                 "speedup": t_single8 / t_batched8}
    return out


def run_aggregates(args):
    """--workload aggregates: the batching workload as its own JSON line."""
    import torch

    import paper_0908_0863_gb300 as dda

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    r = aggregates_workload(dda, torch, dev, args, extra=False)
    print(json.dumps({
        "metric": "batched mixed-precision solves/s: 8 ballistic aggregates x 64 orientations x 2 polarisations",
        "value": r["value"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64+f64 (complex64 FFT products, FP64 refinement)", "data": "synthetic",
        "config": {"workload": r["workload"], "parallelism": "single",
                   "batch": "one dda_solve_batch per aggregate (all its orientations)"},
        "matvecs_per_s": r["matvecs_per_s"], "clocks": r.get("clocks"), "gpu_launches": r["gpu_launches"],
        "aggregates": r["aggregates"], "batched_vs_single_8rhs_largest": r["batched_vs_single_8rhs_largest"],
    }), flush=True)


# ---------------------------------------------------------- oracle timing
def oracle_rows_sample(nd, mask, rows_count, threads):
    """Time the oracle's direct sum on rows_count rows of A p; returns
    (products per second extrapolated to whole products, seconds, rows)."""
    import numpy as np

    import synth
    from oracle import dda as odda
    coords = odda.coords_of(mask)
    ainv = np.full((nd, 3), 1.0 / odda.alpha_rr(M_REFR, K_WAVE))
    p = synth.complex_normal(SEED, (3, nd))
    rows = synth.rng(SEED + 1).choice(nd, size=rows_count, replace=False)
    odda.direct_matvec_rows(coords, ainv, K_WAVE, p, rows[:1], nthreads=threads)  # warm
    t0 = time.perf_counter()
    odda.direct_matvec_rows(coords, ainv, K_WAVE, p, rows, nthreads=threads)
    dt = time.perf_counter() - t0
    return rows_count / nd / dt, dt


def cpu_baseline(args, nd, mask):
    threads = os.cpu_count() or 1
    rate, dt = oracle_rows_sample(nd, mask, args.cpu_rows, threads)
    rows1 = max(1, args.cpu_rows // 10)
    rate1, dt1 = oracle_rows_sample(nd, mask, rows1, 1)
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{args.cpu_rows} rows of A p by direct FP64 summation over all {nd} dipoles "
                      f"({dt:.1f} s), scaled to whole products",
            "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                              "sample": f"{rows1} rows on one thread ({dt1:.1f} s), scaled to whole products"}}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    n, D = args.edge, args.diameter
    mask = synth.sphere(D, box=(n, n, n))
    nd = int(mask.sum())
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_rows_sample(nd, mask, max(1, args.cpu_rows // 10), threads)
    t0 = time.perf_counter()
    rows_done = 0
    for _ in range(args.steps):
        oracle_rows_sample(nd, mask, args.cpu_rows, threads)
        rows_done += args.cpu_rows
    dt = time.perf_counter() - t0
    value = rows_done / nd / dt
    sample = f"{args.cpu_rows} rows of A p per step by direct FP64 summation over all {nd} dipoles, scaled to whole products"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(n, D), "lattice": [n, n, n], "n_dipoles": nd},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--edge", type=int, default=N_EDGE)
    ap.add_argument("--diameter", type=int, default=DIAM)
    ap.add_argument("--method", default="bicgstab")
    ap.add_argument("--tol", type=float, default=TOL)
    ap.add_argument("--max-iter", type=int, default=4000)
    ap.add_argument("--cpu-rows", type=int, default=200)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64-solve", dest="fp64_solve", action="store_false",
                    help="skip the mixed-vs-FP64 BiCGSTAB and QMR solves of the extras")
    ap.add_argument("--ellipsoid-matvecs", type=int, default=1000,
                    help="timed products per precision on the 128^3 two-material ellipsoid (0: skip)")
    ap.add_argument("--no-row-sweep", dest="row_sweep", action="store_false",
                    help="skip the x-pass sweep over rows of 160, 192, 320 and 384 points")
    ap.add_argument("--no-aggregates", dest="aggregates", action="store_false",
                    help="skip the ballistic-aggregate batching workload of the extras")
    ap.add_argument("--no-table4", dest="table4", action="store_false",
                    help="skip the SPHERE 200^3 solver-benchmark timings (Table 4's workload) of the extras")
    ap.add_argument("--agg-method", default="bicgstab")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="jobs timed end to end through host buffers (at most --steps)")
    ap.add_argument("--also-methods", default="", help="comma-separated methods to time one mixed solve each")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default tile widths instead of tuning them before the warm-up")
    ap.add_argument("--no-unpruned", dest="unpruned", action="store_false",
                    help="skip the unpruned cuFFT comparison extra")
    ap.add_argument("--batch", type=int, default=16, help="right-hand sides of the batched-solve extra (0: skip)")
    ap.add_argument("--workload", default="sphere256", choices=["sphere256", "aggregates"],
                    help="sphere256: the headline metric; aggregates: the batched orientation-averaging workload")
    ap.add_argument("--agg-count", type=int, default=len(AGG_MONOMERS))
    ap.add_argument("--agg-directions", type=int, default=64)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "aggregates":
        run_aggregates(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
