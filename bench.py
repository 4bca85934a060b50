#!/usr/bin/env python3
"""Benchmark of the temporally blocked stencil sweep (GCell-updates/s).

One step = one call of the library's run entry point advancing the workload
grid T time steps (all passes of the N.5D-blocked sweep plus the halo copy),
on seeded synthetic inputs of the paper's benchmark shapes (Section 5.1:
16384^2 2D grids, 512^3 3D grids, 1000 iterations).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...    # the CPU oracle, timed on host cores

Prints one JSON line (rank 0).  For N > 1 (torchrun) every rank runs an
independent replica of the workload on its own GPU: the sweep has no
exchange step on one grid, so the job scales weakly with no collective on
the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2001_01473_gb300 import inputs  # noqa: E402

STAR, BOX = inputs.STAR, inputs.BOX

# name -> (ndim, shape, radius, dtype, interior dims, T)
WORKLOADS = {
    "star2d1r-f32": (2, STAR, 1, "f32", (16384, 16384), 1000),
    "star2d2r-f32": (2, STAR, 2, "f32", (16384, 16384), 1000),
    "star2d3r-f32": (2, STAR, 3, "f32", (16384, 16384), 1000),
    "star2d4r-f32": (2, STAR, 4, "f32", (16384, 16384), 1000),
    "box2d1r-f32": (2, BOX, 1, "f32", (16384, 16384), 1000),
    "box2d2r-f32": (2, BOX, 2, "f32", (16384, 16384), 1000),
    "star2d1r-f64": (2, STAR, 1, "f64", (16384, 16384), 1000),
    "star2d2r-f64": (2, STAR, 2, "f64", (16384, 16384), 1000),
    "box2d1r-f64": (2, BOX, 1, "f64", (16384, 16384), 1000),
    "star2d3r-f64": (2, STAR, 3, "f64", (16384, 16384), 1000),
    "star2d4r-f64": (2, STAR, 4, "f64", (16384, 16384), 1000),
    "box2d2r-f64": (2, BOX, 2, "f64", (16384, 16384), 1000),
    "box2d1r-f16": (2, BOX, 1, "f16", (16384, 16384), 1000),
    "box2d1r-f32c": (2, BOX, 1, "f32c", (16384, 16384), 1000),
    "star3d1r-f32": (3, STAR, 1, "f32", (512, 512, 512), 200),
    "star3d2r-f32": (3, STAR, 2, "f32", (512, 512, 512), 200),
    "star3d3r-f32": (3, STAR, 3, "f32", (512, 512, 512), 200),
    "star3d4r-f32": (3, STAR, 4, "f32", (512, 512, 512), 200),
    "box3d1r-f32": (3, BOX, 1, "f32", (512, 512, 512), 200),
    "box2d3r-f32": (2, BOX, 3, "f32", (16384, 16384), 1000),
    "box2d4r-f32": (2, BOX, 4, "f32", (16384, 16384), 1000),
    "box3d2r-f32": (3, BOX, 2, "f32", (512, 512, 512), 200),
    "box3d3r-f32": (3, BOX, 3, "f32", (512, 512, 512), 200),
    "box3d4r-f32": (3, BOX, 4, "f32", (512, 512, 512), 200),
    "star3d1r-f64": (3, STAR, 1, "f64", (512, 512, 512), 200),
    "box3d1r-f64": (3, BOX, 1, "f64", (512, 512, 512), 200),
    "star3d2r-f64": (3, STAR, 2, "f64", (512, 512, 512), 200),
    "star3d3r-f64": (3, STAR, 3, "f64", (512, 512, 512), 200),
    "star3d4r-f64": (3, STAR, 4, "f64", (512, 512, 512), 200),
    # the small bit-exact case: 512^2 FP32, T = 64 (1 MB grid, inside L2: the
    # timed steps flush L2 in between, and the oracle leg checks every cell)
    "star2d1r-f32-512": (2, STAR, 1, "f32", (512, 512), 64),
    # smaller grids for profiler captures (still larger than the 129 MB L2)
    "star2d1r-f32-8k": (2, STAR, 1, "f32", (8192, 8192), 100),
    "box2d2r-f32-8k": (2, BOX, 2, "f32", (8192, 8192), 100),
    "star3d1r-f32-320": (3, STAR, 1, "f32", (320, 320, 320), 30),
}
# Division-type stencils (Table 4's j* rows): the same chain divided every step
# by DIVISOR, exactly ("div") or through the rounded reciprocal ("rcp"); the
# coefficients are the normalised ones scaled by DIVISOR.
DIVISOR = 7.0
DIV_WORKLOADS = {
    "j2d5pt-f32": (2, STAR, 1, "f32", (16384, 16384), 1000, "div"),
    "j2d5pt-rcp-f32": (2, STAR, 1, "f32", (16384, 16384), 1000, "rcp"),
    "j2d9pt-f32": (2, STAR, 2, "f32", (16384, 16384), 1000, "div"),
    "j2d9pt-gol-f32": (2, BOX, 1, "f32", (16384, 16384), 1000, "div"),
    "j3d27pt-f32": (3, BOX, 1, "f32", (512, 512, 512), 200, "div"),
    "j2d5pt-f64": (2, STAR, 1, "f64", (16384, 16384), 1000, "div"),
}
DEFAULT_WORKLOAD = "star2d1r-f32"


def workload(name):
    """(ndim, shape, R, dtype, dims, T, post); post is None for the plain method."""
    if name in DIV_WORKLOADS:
        return DIV_WORKLOADS[name]
    return WORKLOADS[name] + (None,)


def workload_coeffs(ndim, shape, R, post):
    c = inputs.normalised_coeffs(inputs.coeff_count(ndim, shape, R), 0)
    return c * DIVISOR if post else c

# The paper's V100 SXM2 "Tuned" figures (Table 5) for the same stencil,
# precision, grid and iteration count, in GCell/s (GFLOP/s / FLOP per cell).
PAPER_V100_GCELLS = {
    "star2d1r-f32": 5631 / 9, "star2d2r-f32": 6319 / 17, "star2d3r-f32": 7132 / 25,
    "star2d4r-f32": 7244 / 33, "box2d1r-f32": 6693 / 17, "box2d2r-f32": 9163 / 49,
    "star2d1r-f64": 3306 / 9, "star2d2r-f64": 3071 / 17, "box2d1r-f64": 2984 / 17,
    "box2d3r-f32": 10227 / 97, "box2d4r-f32": 10772 / 161,
    "j2d5pt-f32": 6160 / 10, "j2d9pt-f32": 6398 / 18, "j2d9pt-gol-f32": 6865 / 18,
}
# Table 5's 3D rows are for 512^3 with 1000 iterations; this benchmark runs
# the 512^3 grids for T = 200, so they are context, not the same workload.
PAPER_V100_3D_CONTEXT = {
    "star3d1r-f32": 2887 / 13, "star3d2r-f32": 2910 / 25, "star3d3r-f32": 3118 / 37,
    "star3d4r-f32": 2808 / 49, "box3d1r-f32": 6284 / 53, "box3d2r-f32": 8666 / 249,
    "box3d3r-f32": 9351 / 685, "box3d4r-f32": 9707 / 1457, "j3d27pt-f32": 6251 / 54,
}

# GB300 unit counts and clock used for the ALU peak: 152 SMs x 128 FP32 lanes
# x 2 flops x 2070 MHz.  FP64 from the FP32:FP64 ratio the device reports.
NOMINAL_SMS = 152
NOMINAL_FP32_LANES = 128
NOMINAL_MAX_MHZ = 2070.0
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20   # written between timed steps of grids that fit in L2 (129 MB)


def bytes_per_cell(dtype: str) -> int:
    return {"f32": 4, "f64": 8, "f16": 2, "f32c": 4}[dtype]


def flops_per_cell(ndim: int, shape: int, R: int, dtype: str, post=None) -> int:
    """Algorithmic flops of one cell-update: one multiply + (n-1) fma = 2n-1
    (Table 4), plus one for a division-type stencil's division.  The
    compensated form counts Dot2's 10 flops per term."""
    n = inputs.coeff_count(ndim, shape, R)
    if dtype == "f32c":
        # first term: product + its error by fma (2); each later term: TwoProduct
        # (2), TwoSum (6), error accumulation (2); the final sum p + s (1)
        return 10 * n - 7
    return 2 * n - 1 + (1 if post else 0)


def built_degrees(ndim, shape, R, dtype, post=None):
    """Degrees bT compiled for a stencil (any tile variant), from kernels.py."""
    from paper_2001_01473_gb300 import kernels as K
    dt = {"f32": "DT_F32", "f64": "DT_F64", "f16": "DT_F16S", "f32c": "DT_F32C"}[dtype]
    sh = K.STAR if shape == STAR else K.BOX
    out = set()
    if post:
        tabs = [(t[0], t[1], t[2], t[4]) for t in (K.KERNELS_DIV_2D if ndim == 2 else K.KERNELS_DIV_3D)]
        tabs += [(t[0], t[1], t[2], t[4]) for t in K.KERNELS_DIV_2D_WIDE] if ndim == 2 else []
    elif ndim == 2:
        tabs = [(t[0], t[1], t[2], t[5]) for t in K.KERNELS_2D + K.KERNELS_2D_WIDE]
    else:
        tabs = [(t[0], t[1], t[2], t[5]) for t in K.KERNELS_3D]
        tabs += [(K.STAR, t[0], t[1], "DT_F32") for t in K.KERNELS_3D_STAR]
        tabs += [(K.BOX, t[0], range(1, 2), t[2]) for t in K.KERNELS_3D_BOX1]
    for s2, r2, bts, d2 in tabs:
        if s2 == sh and r2 == R and d2 == dt:
            out.update(bts)
    return sorted(out)


def smem_bytes_per_cell(ndim, shape, R, dtype, bt):
    """Shared-memory bytes the kernel moves per cell-update, counted from its
    design (the B_smem of the roofline's shared-memory term):
      2D sweep: the staged input row, written by TMA and read once per pass:
        2w / bT;
      3D sweep: that, plus per level the y exchange: each cell stored once
        and 2R rows of neighbours read per RW rows a warp owns:
        wc (1 + 2R / RW), wc the compute word;
      3D one-level high-order box: the staged plane written once and read
        over (RW + 2R) rows x (V + 2R) cells per RW x V cells of a thread."""
    from paper_2001_01473_gb300 import kernels as K
    w = bytes_per_cell(dtype)
    wc = 8 if dtype == "f64" else 4
    if ndim == 2:
        return 2.0 * w / bt
    if shape == BOX and R >= 2:
        rw = {(r, s): rw for r, s, _d, _nw, rw in K.KERNELS_3D_BOX1}[(R, "double" if dtype == "f64" else "float")]
        v = 4
        return w * (1.0 + (rw + 2 * R) * (v + 2 * R) / (rw * v))
    st = {"f64": "double", "f16": "__half"}.get(dtype, "float")
    _v, rw = K.geom3d(K.STAR if shape == STAR else K.BOX, R, st)
    return 2.0 * w / bt + wc * (1.0 + 2.0 * R / rw)


def roof_terms(ndim, shape, R, dtype, bt, post, hbm_gbs, smem_gbs, alu_tflops):
    """The three roof terms in cell-updates/s: HBM bytes per bT steps at the
    copy bandwidth, shared-memory bytes at the shared-memory bandwidth, flops at
    the FMA peak; the roof is their minimum."""
    w = bytes_per_cell(dtype)
    terms = {"hbm": hbm_gbs * 1e9 * bt / (2.0 * w),
             "smem": smem_gbs * 1e9 / smem_bytes_per_cell(ndim, shape, R, dtype, bt),
             "alu": alu_tflops * 1e12 / flops_per_cell(ndim, shape, R, dtype, post)}
    return terms


def load_measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            with open(p) as f:
                d = json.load(f)
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


# ---------------------------------------------------------------------------
# Distributed plumbing (replicas; no collective on the data path).

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend=backend)
    return dist


def reduce_max(x: float, dist, device=None) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist, device=None):
    if dist is None:
        return
    import torch
    if device is not None and str(device).startswith("cuda"):
        dist.barrier(device_ids=[torch.cuda.current_device()])
    else:
        dist.barrier()


# ---------------------------------------------------------------------------
# Clock sampling during the timed region.

def summarize_clocks(rows) -> dict:
    """Summary of nvidia-smi samples taken during the timed region (rows of the
    ClockSampler fields as strings): median and maximum SM clock, the largest
    power draw, and every throttle reason seen active in any sample."""
    def num(s):
        try:
            return float(s)
        except ValueError:
            return float("nan")
    sm = [num(r[1]) for r in rows]
    mx = [num(r[2]) for r in rows]
    pw = [num(r[3]) for r in rows]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4)
                      if r[5 + i].lower() in ("active", "1", "yes")})
    loaded = [s for s, p in zip(sm, pw) if p == p] or sm
    return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx),
            "power_w_max": max(p for p in pw if p == p) if any(p == p for p in pw) else None,
            "samples": len(rows), "reasons": reasons}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return summarize_clocks(rows)


# ---------------------------------------------------------------------------
# Traffic from the committed ncu summary (valid only for the kernel source it
# was taken on).

def kernel_source_digest() -> str:
    h = hashlib.sha1()
    for f in ("sweep2d.cuh", "device_common.cuh"):
        with open(os.path.join(ROOT, "paper_2001_01473_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def committed_traffic(workload: str, bt: int, tile: int):
    """dram bytes per launch of the sweep kernel recorded under profiles/ for
    this workload, degree and tile width, if taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "sweep2d_traffic.md")
    if not os.path.exists(p):
        return None
    digest = kernel_source_digest()
    pat = re.compile(r"^\|\s*%s\s*\|\s*%d\s*\|\s*%d\s*\|\s*([0-9.eE+]+)\s*\|\s*([0-9.eE+]+)\s*\|"
                     r"\s*([0-9a-f]+)\s*\|" % (re.escape(workload), bt, tile))
    with open(p) as f:
        for line in f:
            m = pat.match(line.strip())
            if m and m.group(3) == digest:
                # recorded on a smaller grid: scale by the cells of a full launch
                return float(m.group(1)) * float(m.group(2))
    return None


# ---------------------------------------------------------------------------
# The paper's analytic model (Section 4) next to the measurement.

PAPER_FP64_NOMINAL_GFLOPS = 1250.0   # GB300's nominal FP64 rate (the model takes theoretical compute)


def paper_model_report(an5d, ndim, shape, R, dtype, dims, post, bt, hsn, tile, value, inrun):
    """The paper's model on this GPU's peaks (compute: nominal FMA rate from the
    unit counts; global and shared memory: the in-run micro-benchmarks), for
    (a) this run's configuration read as the paper's design (one thread per
    cell of the tile) and (b) the model's own best configuration over the
    paper's tuning space (Section 5.3).  accuracy = measured / predicted, the
    paper's model-accuracy ratio (Section 6.3)."""
    if dtype not in ("f32", "f64"):
        return None
    n = inputs.coeff_count(ndim, shape, R)
    ops = (n - 1, 1, 0, 1 if post else 0)
    comp = (PAPER_FP64_NOMINAL_GFLOPS if dtype == "f64"
            else inrun["sms"] * 128 * 2 * inrun["sm_clock_mhz"] * 1e-3)
    dev = dict(peak_comp_gflops=comp, peak_gm_gbs=inrun["hbm_gbs"], peak_sm_gbs=inrun["smem_gbs"],
               sm_count=inrun["sms"], max_threads_per_sm=2048)
    w = bytes_per_cell(dtype)
    out = {"peaks": dev}
    try:
        r = an5d.an5d_paper_model(ndim, shape, R, w, ops, dims, bt, tile, hsn, dev)
        out["at_this_config"] = {"bT": bt, "bS": tile, "hSN": hsn, "gcells": r["gcells"],
                                 "bound": r["bound"], "accuracy": value / r["gcells"]}
    except an5d.An5dError:
        pass
    best = None
    bts = range(1, 17) if ndim == 2 else range(1, 9)
    bss = [[128], [256], [512], [1024]] if ndim == 2 else [[16, 16], [32, 16], [32, 32], [64, 16]]
    for b in bts:
        for bs in bss:
            for h in (128, 256, 512, 1024):
                try:
                    r = an5d.an5d_paper_model(ndim, shape, R, w, ops, dims, b, bs, h, dev)
                except an5d.An5dError:
                    continue
                if best is None or r["gcells"] > best["gcells"]:
                    best = {"bT": b, "bS": bs, "hSN": h, "gcells": r["gcells"], "bound": r["bound"]}
    if best:
        best["accuracy"] = value / best["gcells"]
        out["model_best"] = best
    return out


# ---------------------------------------------------------------------------
# Reference arm: the CPU oracle.

def oracle_time(ndim, shape, R, dtype, dims, budget_s=12.0, post=None, T_full=None, out=None):
    """Time the oracle on a bounded sample of the workload: the full grid for
    a number of steps chosen so that the run takes about budget_s.  When the
    workload's whole length T_full fits that budget, exactly T_full steps
    run; with `out` (the GPU's result of the same workload) the oracle's
    result is then compared with it bit for bit ("parity" in the result)."""
    import oracle
    c = workload_coeffs(ndim, shape, R, post)
    u0 = inputs.field(dims, R, 1, dtype)
    cells = float(np.prod(dims))

    def run(T):
        if post:
            t = np.float64 if dtype == "f64" else np.float32
            return oracle.run_div(dtype, ndim, shape, R, c.astype(t), DIVISOR,
                                  oracle.POST_DIV if post == "div" else oracle.POST_MUL_RCP, dims, u0, T)
        if dtype == "f64":
            return oracle.run_f64(ndim, shape, R, c, dims, u0, T)
        if dtype == "f16":
            return oracle.run_f16s(ndim, shape, R, c.astype(np.float32), dims, u0, T)
        if dtype == "f32c":
            return oracle.run_dot2(ndim, shape, R, c.astype(np.float32), dims, u0, T)
        return oracle.run_f32(ndim, shape, R, c.astype(np.float32), dims, u0, T)

    # per-step cost without the oracle's set-up copies: difference of two runs
    t0 = time.perf_counter()
    run(1)
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    run(3)
    t3 = time.perf_counter() - t0
    per_step = max((t3 - t1) / 2.0, 1e-4)
    T = max(1, min(1000, int(budget_s / per_step)))
    whole = T_full is not None and T >= T_full
    if whole:
        T = T_full
    t0 = time.perf_counter()
    res = run(T)
    dt = time.perf_counter() - t0
    line = {"value": cells * T / dt / 1e9, "unit": "GCell-updates/s", "cores": oracle.get_threads(),
            "kind": "oracle", "seconds": round(dt, 3),
            "sample": (f"full {'x'.join(map(str, dims))} grid, "
                       + (f"all T={T} steps of the workload" if whole else f"T={T} of the workload's steps")
                       + " (includes the oracle's two buffer copies)")}
    if whole and out is not None:
        g = np.ascontiguousarray(out).view(np.uint8)
        r = np.ascontiguousarray(res).view(np.uint8)
        same = g.shape == r.shape and bool(np.array_equal(g, r))
        line["parity"] = {"T": T, "cells": int(np.asarray(res).size), "bitwise_equal": same}
    return line


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    ndim, shape, R, dtype, dims, T, post = workload(args.workload)
    # each step is a bounded sample: the whole run stays within a few minutes
    budget = max(2.0, min(args.ref_budget, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(max(0, args.warmup)):
        oracle_time(ndim, shape, R, dtype, dims, budget_s=min(budget, 2.0), post=post)
    steps = [oracle_time(ndim, shape, R, dtype, dims, budget_s=budget, post=post)
             for _ in range(args.steps)]
    v = statistics.mean(s["value"] for s in steps)
    cpu = dict(steps[0])
    cpu["value"] = v
    line = {
        "impl": "reference", "metric": "GCell-updates/s", "value": v, "unit": "GCell-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(s["seconds"] for s in steps) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic", "config": workload_config(args.workload, world),
        "cpu_baseline": cpu,
        "e2e": {"value": v, "unit": "GCell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(name, world, flushed=False):
    ndim, shape, R, dtype, dims, T, post = workload(name)
    div = ""
    if post:
        div = (f", divided by {DIVISOR:g} every step "
               f"({'IEEE division' if post == 'div' else 'product with the rounded reciprocal'}; "
               f"coefficients scaled by {DIVISOR:g})")
    return {"workload": f"{name}: {'star' if shape == STAR else 'box'} radius {R}, "
                        f"{'x'.join(map(str, dims))} interior + {R}-cell Dirichlet halo, T={T}, "
                        f"seeded normalised coefficients, uniform [0,1) field{div}",
            "stencil": name, "dims": list(dims), "T": T, "radius": R,
            "parallelism": f"replicas{world}" if world > 1 else "single",
            "l2": ("grid inside L2: a 512 MB buffer is written between timed steps (L2 flush), "
                   "each step timed by its own CUDA events" if flushed else
                   "inputs larger than L2 (129 MB)")}


# ---------------------------------------------------------------------------
# Our arm.

def sweep_roofline(ndim, shape, R, dtype, post, cells, bt, launch_s, inrun, kernel, traffic=None):
    """Roofline object of one sweep launch of degree bt over `cells` interior
    cells taking launch_s seconds: the binding term of min(HBM, shared memory,
    ALU), the achieved rate in that term's unit, and the same throughput
    against the roof at the largest degree built for the stencil."""
    peaks, peak_src = load_measured_peaks()
    w = bytes_per_cell(dtype)
    hbm_bytes_launch = cells * 2 * w              # read once + write once per pass
    flops_launch = cells * bt * flops_per_cell(ndim, shape, R, dtype, post)
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    alu_fp32 = NOMINAL_SMS * NOMINAL_FP32_LANES * 2 * NOMINAL_MAX_MHZ * 1e6 / 1e12   # TFLOP/s
    alu_peak = alu_fp32 if dtype != "f64" else inrun["fp64_gflops"] / 1e3
    smem_peak = float(inrun["smem_gbs"])
    smem_b = smem_bytes_per_cell(ndim, shape, R, dtype, bt)
    terms = roof_terms(ndim, shape, R, dtype, bt, post, hbm_peak, smem_peak, alu_peak)
    bound = min(terms, key=terms.get)
    if bound == "hbm":
        achieved, peak, unit = hbm_bytes_launch / launch_s / 1e9, hbm_peak, "GB/s"
    elif bound == "smem":
        achieved, peak, unit = cells * bt * smem_b / launch_s / 1e9, smem_peak, "GB/s"
    else:
        achieved, peak, unit = flops_launch / launch_s / 1e12, alu_peak, "TFLOP/s"
    roof_gcells = terms[bound] / 1e9
    measured_gcells = cells * bt / launch_s / 1e9
    # the same throughput against the roof at the largest degree built for this
    # stencil: a lower-degree pick cannot hide throughput left on the table
    bt_top = max(built_degrees(ndim, shape, R, dtype, post) or [bt])
    terms_top = roof_terms(ndim, shape, R, dtype, bt_top, post, hbm_peak, smem_peak, alu_peak)
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": ({"hbm": f"{peak_src} MEASURED_PEAKS.json hbm_gbs",
                             "smem": "in-run shared-memory microbenchmark (LDS.128)",
                             "alu": ("152 SMs x 128 FP32 lanes x 2 x 2070 MHz" if dtype != "f64"
                                     else "in-run FP64 fma microbenchmark")}[bound]),
            "kernel": kernel,
            "algorithmic_bytes_per_launch": hbm_bytes_launch,
            "algorithmic_flops_per_launch": flops_launch,
            "smem_bytes_per_cell_update": smem_b,
            "roof_terms_gcells": {k: v / 1e9 for k, v in terms.items()},
            "temporal_roof_gcells": roof_gcells,
            "frac_of_temporal_roof": measured_gcells / roof_gcells,
            "largest_built_bT": bt_top,
            "roof_at_largest_bT_gcells": min(terms_top.values()) / 1e9,
            "roof_at_largest_bT_bound": min(terms_top, key=terms_top.get),
            "frac_of_roof_at_largest_bT": measured_gcells / (min(terms_top.values()) / 1e9)}


def run_ours(args, rank, world, local):
    import torch
    from paper_2001_01473_gb300 import an5d

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, "nccl")
    ndim, shape, R, dtype, dims, T, post = workload(args.workload)
    c = workload_coeffs(ndim, shape, R, post)
    u0 = inputs.field(dims, R, 1, dtype)
    cells = float(np.prod(dims))
    stream = torch.cuda.current_stream()

    inrun = an5d.an5d_measure_peaks(stream)        # copy / fma / smem microbenchmarks
    if post:
        plan = an5d.Plan(ndim, shape, R, c, dtype, dims, divisor=DIVISOR, post=post)
    else:
        plan = an5d.Plan(ndim, shape, R, c, dtype, dims)
    if args.config:
        fbt, fhsn, ftile = (int(v) for v in args.config.split(","))
        plan.set_config(fbt, fhsn)
        plan.set_tile(ftile)
    else:
        plan.tune(topk=args.topk, T_probe=args.tune_T, stream=stream)
    cfg = plan.config()
    bt = cfg["bT"]
    passes = T // bt + (1 if T % bt else 0)
    launches_per_step = plan.launches(T)            # passes (2 launches for a split 3D pass) + halo copies

    x = torch.from_numpy(u0).to(dev)
    y = torch.empty_like(x)

    # ---- device-resident timing ----
    for _ in range(args.warmup):
        plan.run(x, y, T, stream)
    torch.cuda.synchronize()
    barrier(dist, dev)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    # Grids that fit in L2 (the 512^2 case) are timed step by step, with a
    # write of a buffer larger than L2 between the timed steps; the others
    # are larger than L2 themselves and run back to back.
    flush = (torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
             if 3 * x.numel() * x.element_size() < L2_FLUSH_BYTES else None)
    torch.cuda.nvtx.range_push("timed")
    if flush is None:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            plan.run(x, y, T, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_local = ev0.elapsed_time(ev1)
    else:
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            plan.run(x, y, T, stream)
            e1.record(stream)
        torch.cuda.synchronize()
        ms_local = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    barrier(dist, dev)
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"device status {st}: {an5d.an5d_last_error()}")
    y_host = y.cpu().numpy() if x.numel() * x.element_size() <= (256 << 20) else None
    ms = reduce_max(ms_local, dist, dev)
    ms_step = ms / args.steps
    value = world * cells * T * args.steps / (ms * 1e-3) / 1e9

    # ---- end to end through the host-buffer entry point ----
    hin = torch.from_numpy(u0).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    hin_np, hout_np = hin.numpy(), hout.numpy()
    plan.run_host(hin_np, hout_np, T, stream)      # warm (allocates staging buffers)
    barrier(dist, dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        plan.run_host(hin_np, hout_np, T, stream)
    e2e_s = time.perf_counter() - t0
    e2e_s = reduce_max(e2e_s, dist, dev)
    e2e_value = world * cells * T * args.e2e_steps / e2e_s / 1e9
    nbytes = u0.nbytes

    # ---- roofline of the dominant kernel (the sweep pass) ----
    launch_s = ms_step * 1e-3 / passes            # halo copy (~us) included: conservative
    full_passes = T // bt
    traffic = committed_traffic(args.workload, bt, cfg["tile_x"])
    from paper_2001_01473_gb300 import kernels as K
    k9 = (ndim == 3 and shape == STAR and dtype == "f32" and post is None
          and any(r == R and bt in bts for r, bts, _nw, _rw in K.KERNELS_3D_STAR))
    kernel = (f"box1_kernel bT={bt}" if ndim == 3 and shape == BOX and R >= 2
              else f"star3d_kernel bT={bt} tile_x={cfg['tile_x']}" if k9
              else f"sweep{ndim}d_kernel bT={bt} tile_x={cfg['tile_x']}")
    roofline = sweep_roofline(ndim, shape, R, dtype, post, cells, bt, launch_s, inrun, kernel, traffic)
    roofline["passes_per_step"] = passes
    roofline["full_degree_launches"] = full_passes

    base = PAPER_V100_GCELLS.get(args.workload)
    line = {
        "metric": "GCell-updates/s", "value": value, "unit": "GCell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": (value / world / base) if base else None,
        "baseline_note": "paper's V100 SXM2 Tuned figure (Table 5) for this workload: context "
                         "from other hardware" if base else None,
        "dtype": dtype, "data": "synthetic",
        "config": dict(workload_config(args.workload, world, flushed=flush is not None), bT=bt, hsn=cfg["hsn"],
                       tile_x=cfg["tile_x"], ctas=cfg["ctas"],
                       model_gcells=cfg["model_gcells"], tuned_gcells=cfg["measured_gcells"]),
        "e2e": {"value": e2e_value, "unit": "GCell-updates/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roofline,
        "inrun_peaks": inrun,
        "paper_model": paper_model_report(an5d, ndim, shape, R, dtype, dims, post, bt, cfg["hsn"],
                                          [cfg["tile_x"]] + ([cfg["tile_y"]] if ndim == 3 else []),
                                          value, inrun),
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_time(ndim, shape, R, dtype, dims, budget_s=args.ref_budget,
                                            post=post, T_full=T, out=y_host)
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


PRECISION_WORKLOADS = {
    # name -> (ndim, shape, radius, coefficient recipe, dims, T)
    "heat3d": (3, STAR, 1, "heat", (512, 512, 512), 1000),
    "box2d1r": (2, BOX, 1, "normalised", (16384, 16384), 1000),
}


def run_precision(args, rank, world, local):
    """Precision forms: throughput of the FP32 plain, Dot2-compensated FP32 and
    binary16-storage forms next to their max / relative-L2 error against an
    FP64 evaluation of the same sweep from the same input.  The FP64
    evaluation is the library's FP64 plain method, which the parity tests
    show to be bit-identical to the FP64 CPU oracle."""
    import torch
    from paper_2001_01473_gb300 import an5d
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    names = [args.precision_workload] if args.precision_workload else list(PRECISION_WORKLOADS)
    inrun = an5d.an5d_measure_peaks(stream)
    for name in names:
        ndim, shape, R, recipe, dims, T = PRECISION_WORKLOADS[name]
        n = inputs.coeff_count(ndim, shape, R)
        c = inputs.heat_coeffs(ndim) if recipe == "heat" else inputs.normalised_coeffs(n, 0)
        c32 = c.astype(np.float32).astype(np.float64)
        cells = float(np.prod(dims))
        base32 = inputs.gaussian_bump(dims, R, 1, "f32")
        refs = {}
        seen = {}
        for form in ("f32", "f32c", "f16"):
            u0 = base32 if form != "f16" else base32.astype(np.float16)
            key = "f16" if form == "f16" else "f32"
            if key not in refs:                 # FP64 reference from this form's input
                r_in = torch.from_numpy(u0.astype(np.float64)).to(dev)
                r_out = torch.empty_like(r_in)
                with an5d.Plan(ndim, shape, R, c32, "f64", dims) as rp:
                    rp.run(r_in, r_out, T, stream)
                    torch.cuda.synchronize()
                    assert rp.status() == 0
                del r_in
                refs[key] = r_out
            x = torch.from_numpy(u0).to(dev)
            y = torch.empty_like(x)
            with an5d.Plan(ndim, shape, R, c, form, dims) as plan:
                plan.tune(topk=args.topk, T_probe=args.tune_T, stream=stream)
                cfg = plan.config()
                for _ in range(args.warmup):
                    plan.run(x, y, T, stream)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    plan.run(x, y, T, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                assert plan.status() == 0
                ms = e0.elapsed_time(e1) / args.steps
            err = an5d.an5d_error_norms(ndim, R, dims, form, y, refs[key], stream)
            umax = float(np.max(np.abs(u0.astype(np.float64))))
            bt = cfg["bT"]
            passes = T // bt + (1 if T % bt else 0)
            roofline = sweep_roofline(ndim, shape, R, form, None, cells, bt, ms * 1e-3 / passes, inrun,
                                      f"sweep{ndim}d_kernel bT={bt} tile_x={cfg['tile_x']} ({form})")
            roofline["passes_per_step"] = passes
            line = {"mode": "precision", "workload": name, "form": form,
                    "metric": "GCell-updates/s", "value": cells * T / (ms * 1e-3) / 1e9,
                    "unit": "GCell-updates/s", "ms_per_step": ms, "steps": args.steps,
                    "config": {"dims": list(dims), "T": T, "bT": cfg["bT"], "hsn": cfg["hsn"],
                               "init": "Gaussian bump (sigma n/8) + 0.01 U[0,1)",
                               "coefficients": recipe},
                    "error_vs_fp64": {"max_abs": err["max_abs"], "rel_l2": err["rel_l2"],
                                      "max_abs_over_max_u0": err["max_abs"] / umax},
                    "roofline": roofline}
            seen[form] = (line["value"], err["rel_l2"], err["max_abs"])
            if rank == 0:
                print(json.dumps(line), flush=True)
            del x, y
        # The chosen form of this workload: the one with the smallest relative
        # L2 error against the FP64 evaluation, stated next to the plain FP32
        # chain's speed and error.
        chosen = min(seen, key=lambda f: seen[f][1])
        v0, l0, m0 = seen["f32"]
        summary = {"mode": "precision-choice", "workload": name,
                   "rule": "form with the smallest relative L2 error vs the FP64 evaluation",
                   "chosen": chosen,
                   "chosen_gcells": seen[chosen][0], "plain_gcells": v0,
                   "speed_vs_plain": seen[chosen][0] / v0,
                   "chosen_rel_l2": seen[chosen][1], "plain_rel_l2": l0,
                   "chosen_max_abs": seen[chosen][2], "plain_max_abs": m0,
                   "error_vs_plain": seen[chosen][1] / l0 if l0 > 0 else None,
                   "forms": {f: {"gcells": v, "rel_l2": l, "max_abs": m} for f, (v, l, m) in seen.items()}}
        if rank == 0:
            print(json.dumps(summary), flush=True)
        refs.clear()
        torch.cuda.empty_cache()
    return 0


# degrees the batched kernel builds per radius, largest first
BATCH_MENU = {1: (8, 4, 1), 2: (4, 2, 1)}


def batch_roof(grids, class_bt):
    """Roof time of one batch step: for every grid, the larger of the HBM time
    of its passes (each reads and writes the grid once, 8 bytes per cell;
    the T mod bT remaining steps split greedily over the smaller built
    degrees, as the kernel runs them) and the time of its flops at the FP32
    peak, summed over the grids."""
    peaks, src = load_measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)) * 1e9
    alu = NOMINAL_SMS * NOMINAL_FP32_LANES * 2 * NOMINAL_MAX_MHZ * 1e6
    bt_of = {(STAR, 1): class_bt[0], (STAR, 2): class_bt[1], (BOX, 1): class_bt[2], (BOX, 2): class_bt[3]}
    tot = th = ta = 0.0
    for g in grids:
        bt = bt_of[(g[0], g[1])]
        left, passes = g[5] % bt, g[5] // bt
        for m in BATCH_MENU[g[1]]:
            if m < bt:
                passes += left // m
                left %= m
        t_h = passes * g[3] * g[4] * 8.0 / hbm
        t_a = g[3] * g[4] * g[5] * flops_per_cell(2, g[0], g[1], "f32") / alu
        tot += max(t_h, t_a)
        th += t_h
        ta += t_a
    return {"time_s": tot, "hbm_s": th, "alu_s": ta, "bound": "hbm" if th >= ta else "alu",
            "class_bt": list(class_bt),
            "peak_source": f"{src} MEASURED_PEAKS.json hbm_gbs; 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}


def run_batch(args, rank, world, local):
    """Batched form: 512 independent 2D FP32 grids (sides log-uniform in
    [128, 4096], star/box radius 1-2, T uniform in [10, 500]) advanced by one
    CUDA-graph launch of the persistent kernel per step."""
    import torch
    from paper_2001_01473_gb300 import an5d
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    descs = inputs.batch_descs(n=args.batch_n, side_hi=args.batch_side_hi, t_lo=args.batch_tlo,
                               t_hi=args.batch_thi)
    grids = []
    for i, d in enumerate(descs):
        n = inputs.coeff_count(2, d.shape, d.radius)
        grids.append((d.shape, d.radius, inputs.normalised_coeffs(n, 100 + i), d.ny, d.nx, d.T))
    xs = [torch.from_numpy(inputs.field((g[3], g[4]), g[1], 500 + i, "f32")).to(dev)
          for i, g in enumerate(grids)]
    ys = [torch.empty_like(x) for x in xs]
    with an5d.Batch(grids) as b:
        info = b.tune(stream, xs, ys)
        for _ in range(args.warmup):
            b.run(xs, ys, stream)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            b.run(xs, ys, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        assert b.status() == 0, an5d.an5d_batch_last_error()
        ms = e0.elapsed_time(e1) / args.steps
    cells = info["cell_updates"]
    roof = batch_roof(grids, info["class_bt"])
    top = batch_roof(grids, [BATCH_MENU[1][0], BATCH_MENU[2][0], BATCH_MENU[1][0], BATCH_MENU[2][0]])
    t = ms * 1e-3
    line = {"mode": "batch", "metric": "GCell-updates/s", "value": cells / t / 1e9,
            "unit": "GCell-updates/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
            "config": {"grids": len(grids), "cell_updates_per_step": cells, "items": info["items"],
                       "persistent_ctas": info["ctas"], "class_bt": info["class_bt"],
                       "class_tile_x": info["class_tile_x"],
                       "recipe": "sides log-uniform [128,4096], star/box R1-2, T U[10,500], seed 3"},
            "roofline": {"bound": roof["bound"], "roof_time_ms": roof["time_s"] * 1e3,
                         "hbm_time_ms": roof["hbm_s"] * 1e3, "alu_time_ms": roof["alu_s"] * 1e3,
                         "frac": roof["time_s"] / t,
                         "class_bt": info["class_bt"],
                         "largest_built_class_bt": top["class_bt"],
                         "roof_at_largest_bT_time_ms": top["time_s"] * 1e3,
                         "frac_of_roof_at_largest_bT": top["time_s"] / t,
                         "peak_source": roof["peak_source"],
                         "how": "per grid max(HBM time of its passes at 8 B per cell and pass, "
                                "flops at the FP32 peak), summed over the grids"},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


ADJ_NB = {1: 4, 2: 2}   # block degree of the batched adjoint per radius


def adjoint_roof(grids):
    """Roof time of one batched-adjoint step: per grid, the larger of its
    algorithmic HBM time and its flops at the FP32 peak, summed.  Per block
    of nb steps (M = ceil(T/nb) blocks) a grid's cells move: 8 B for the
    forward checkpoint pass (M - 1 of them), 4 + 4 (nb - 1) B for the
    recompute pass (read the checkpoint, write nb - 1 states; nb >= 2), and
    8 + 4 nb B for the transposed pass (read and write g, read the nb
    states); flops: (2n - 1) per cell and step of every forward, recompute
    and transposed step, and 2n per cell and step of the coefficient
    gradient."""
    peaks, src = load_measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)) * 1e9
    alu = NOMINAL_SMS * NOMINAL_FP32_LANES * 2 * NOMINAL_MAX_MHZ * 1e6
    tot = th = ta = 0.0
    for shape, R, _c, ny, nx, T in grids:
        cells = float(ny * nx)
        n = inputs.coeff_count(2, shape, R)
        nb = ADJ_NB[R]
        M = -(-T // nb)
        byt = 8.0 * max(M - 1, 0)
        fl = (2 * n - 1) * nb * max(M - 1, 0)
        for m in range(M):
            nbm = min(nb, T - m * nb)
            if nbm >= 2:
                byt += 4 + 4 * (nbm - 1)
                fl += (2 * n - 1) * (nbm - 1)
            byt += 8 + 4 * nbm
            fl += nbm * (2 * n - 1 + 2 * n)
        t_h, t_a = cells * byt / hbm, cells * fl / alu
        tot += max(t_h, t_a)
        th += t_h
        ta += t_a
    return {"time_s": tot, "hbm_s": th, "alu_s": ta, "bound": "hbm" if th >= ta else "alu",
            "peak_source": f"{src} MEASURED_PEAKS.json hbm_gbs; 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}


def run_adjoint_bench(args, rank, world, local):
    """Adjoint form on the batched workload: loss 0.5 ||u_T - target||^2 per
    grid (target uniform [0,1) from seed 2), gradients w.r.t. u_0 and the
    coefficients for all 512 grids by the batched adjoint (persistent
    launches in one CUDA graph), and for comparison by the single-grid
    adjoint driven per grid from host threads.  The CPU-baseline leg runs
    the FP64 oracle adjoint on a sample of the grids, timed, and reports the
    GPU result's error against it."""
    import torch
    from paper_2001_01473_gb300 import an5d
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    descs = inputs.batch_descs(n=args.batch_n, side_hi=args.batch_side_hi, t_lo=args.batch_tlo,
                               t_hi=args.batch_thi)
    grids, xs, gts = [], [], []
    for i, d in enumerate(descs):
        n = inputs.coeff_count(2, d.shape, d.radius)
        c = inputs.normalised_coeffs(n, 100 + i)
        grids.append((d.shape, d.radius, c, d.ny, d.nx, d.T))
    with an5d.Batch(grids) as b:
        b.tune(stream)
        for i, g in enumerate(grids):
            xs.append(torch.from_numpy(inputs.field((g[3], g[4]), g[1], 500 + i, "f32")).to(dev))
        ys = [torch.empty_like(x) for x in xs]
        b.run(xs, ys, stream)
        torch.cuda.synchronize()
        assert b.status() == 0
    targets = []
    for i, g in enumerate(grids):
        R = g[1]
        tg = torch.from_numpy(inputs.target_field((g[3], g[4]), R, 2, "f32")).to(dev)
        gt = torch.zeros_like(ys[i])
        gt[R:-R, R:-R] = ys[i][R:-R, R:-R] - tg[R:-R, R:-R]
        gts.append(gt)
        targets.append(tg)
    del ys
    gus = [torch.empty_like(x) for x in xs]
    cells = sum(float(g[3] * g[4] * g[5]) for g in grids)
    with an5d.AdjointBatch(grids, int(args.adjoint_budget_gib * (1 << 30))) as ab:
        info = ab.info()
        for _ in range(max(1, args.warmup)):
            dc = ab.run(xs, gts, gus, stream)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            dc = ab.run(xs, gts, gus, stream)      # synchronous: includes the dL/dc copy to the host
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        t = e0.elapsed_time(e1) * 1e-3 / args.steps
    # the single-grid adjoint (checkpointed level-storing passes and a
    # separate reduction per block) driven per grid from host threads, each
    # on its own stream, largest work first: the same gradients by another
    # schedule, timed for comparison
    per_grid = None
    if args.adjoint_streams > 0:
        import concurrent.futures
        import threading
        plans = [an5d.Plan(2, g[0], g[1], g[2], "f32", (g[3], g[4])) for g in grids]
        order = sorted(range(len(grids)), key=lambda i: -grids[i][3] * grids[i][4] * grids[i][5])
        streams = [torch.cuda.Stream(device=dev) for _ in range(args.adjoint_streams)]
        gus2 = [torch.empty_like(x) for x in xs]
        # A plan keeps the adjoint's work memory (ceil(T / bT) checkpoints and
        # 2 bT level grids, bT = min(plan degree, 4)) between calls.  All 512
        # plans' work memory together does not fit the device, so the grids
        # run in chunks that do (largest first), each timed after a first run
        # that grows its plans' work memory, and a chunk's plans are closed
        # before the next chunk starts.
        need = []
        for i, g in enumerate(grids):
            bt = min(plans[i].config()["bT"], 4)
            need.append((-(-g[5] // bt) + 2 * bt + 1) * (g[3] + 2 * g[1]) * (g[4] + 2 * g[1]) * 4)
        torch.cuda.empty_cache()
        cap = 0.8 * torch.cuda.mem_get_info(dev)[0]
        chunks, cur, acc = [], [], 0
        for i in order:
            if cur and acc + need[i] > cap:
                chunks.append(cur)
                cur, acc = [], 0
            cur.append(i)
            acc += need[i]
        if cur:
            chunks.append(cur)
        seconds = 0.0
        for chunk in chunks:
            times = []
            for _rep in range(2):  # the first run grows the plans' work memory
                torch.cuda.synchronize()
                nxt = iter(chunk)
                lock = threading.Lock()

                def worker(k):
                    torch.cuda.set_device(local)
                    while True:
                        with lock:
                            i = next(nxt, None)
                        if i is None:
                            return
                        an5d.an5d_run_adjoint(plans[i].handle, xs[i], gts[i], gus2[i], grids[i][5], streams[k])

                t0 = time.perf_counter()
                with concurrent.futures.ThreadPoolExecutor(len(streams)) as ex:
                    list(ex.map(worker, range(len(streams))))
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            seconds += times[-1]
            for i in chunk:
                plans[i].close()
        times = [seconds]
        same = all(torch.equal(a, b) for a, b in zip(gus, gus2))
        per_grid = {"value": cells / times[-1] / 1e9, "unit": "GCell-updates/s", "seconds_per_step": times[-1],
                    "streams": args.adjoint_streams, "chunks": len(chunks), "grad_u0_bit_identical_to_batched": same,
                    "how": "an5d_run_adjoint per grid from host threads, one CUDA stream each, largest first "
                           "(host wall clock)"}
        del gus2
    roof = adjoint_roof(grids)
    line = {"mode": "adjoint", "metric": "GCell-updates/s", "value": cells / t / 1e9,
            "unit": "GCell-updates/s", "seconds_per_step": t, "steps": args.steps, "warmup": args.warmup,
            "config": {"grids": len(grids), "cell_updates_per_step": cells, "items": info["items"],
                       "waves": info["waves"], "work_gib": info["work_bytes"] / (1 << 30),
                       "persistent_ctas": info["ctas"], "class_nb": info["class_nb"],
                       "loss": "0.5*||u_T - target||^2, target U[0,1) seed 2",
                       "schedule": "checkpoint every nb steps (nb 4 for radius 1, 2 for radius 2); "
                                   "per block: blocked recompute storing the block's states + blocked "
                                   "transposed pass accumulating dL/dc in registers; all grids in "
                                   "persistent launches of one CUDA graph"},
            "roofline": {"bound": roof["bound"], "roof_time_ms": roof["time_s"] * 1e3,
                         "hbm_time_ms": roof["hbm_s"] * 1e3, "alu_time_ms": roof["alu_s"] * 1e3,
                         "frac": roof["time_s"] / t, "peak_source": roof["peak_source"],
                         "how": "per grid max(algorithmic HBM bytes of its forward, recompute and "
                                "transposed passes, flops of those passes and of dL/dc at the FP32 "
                                "peak), summed over the grids"},
            "clocks": clk}
    if per_grid is not None:
        line["per_grid_host_driven"] = per_grid
    if not args.no_cpu_baseline and rank == 0:
        # CPU-baseline leg: the FP64 oracle adjoint on the grids with the
        # fewest cell-updates (a bounded sample), timed; the GPU gradients of
        # those grids against it
        import oracle
        order = sorted(range(len(grids)), key=lambda i: grids[i][3] * grids[i][4] * grids[i][5])
        sample, t_cpu, cells_cpu = [], 0.0, 0.0
        err_u, err_c = 0.0, 0.0
        for i in order:
            shape, R, c, ny, nx, T = grids[i]
            if t_cpu > args.ref_budget or len(sample) >= 24:
                break
            c32 = c.astype(np.float32).astype(np.float64)
            u0 = xs[i].cpu().numpy().astype(np.float64)
            tg = targets[i].cpu().numpy().astype(np.float64)
            t0 = time.perf_counter()
            _loss, ref_gu, ref_gc = oracle.adjoint_f64(2, shape, R, c32, (ny, nx), u0, tg, T)
            t_cpu += time.perf_counter() - t0
            cells_cpu += float(ny * nx * T)
            inner = (slice(R, R + ny), slice(R, R + nx))
            gu = gus[i].cpu().numpy()[inner].astype(np.float64)
            n = len(c)
            e_u = float(np.linalg.norm(gu - ref_gu[inner]) / max(np.linalg.norm(ref_gu[inner]), 1e-300))
            e_c = float(np.linalg.norm(dc[i][:n] - ref_gc) / max(np.linalg.norm(ref_gc), 1e-300))
            err_u, err_c = max(err_u, e_u), max(err_c, e_c)
            sample.append(i)
        line["cpu_baseline"] = {"value": cells_cpu / t_cpu / 1e9, "unit": "GCell-updates/s",
                                "cores": oracle.get_threads(), "kind": "oracle", "seconds": t_cpu,
                                "sample": f"FP64 oracle adjoint (forward + backward) of the {len(sample)} "
                                          f"grids with the fewest cell-updates ({cells_cpu:.3g} of them)"}
        line["error_vs_fp64_oracle"] = {"grids": len(sample), "max_rel_l2_grad_u0": err_u,
                                        "max_rel_l2_grad_coeffs": err_c,
                                        "note": "the oracle starts from the same FP32 inputs and the "
                                                "run's FP32-rounded coefficients"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS) + sorted(DIV_WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--topk", type=int, default=6)
    ap.add_argument("--tune-T", type=int, default=40)
    ap.add_argument("--config", default=None, metavar="BT,HSN,TILE",
                    help="force a blocking (degree, stream-block length, tile width; 0 = default) "
                         "instead of tuning, e.g. to profile the kernel the full-size run picks")
    ap.add_argument("--ref-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", action="store_true",
                    help="report the precision forms (throughput and error vs FP64)")
    ap.add_argument("--precision-workload", default=None, choices=sorted(PRECISION_WORKLOADS))
    ap.add_argument("--batch", action="store_true", help="report the batched form (512 grids)")
    ap.add_argument("--adjoint", action="store_true", help="report the adjoint form (512 grids)")
    ap.add_argument("--adjoint-streams", type=int, default=8,
                    help="host threads / streams of the per-grid adjoint leg (0: skip it)")
    ap.add_argument("--adjoint-budget-gib", type=float, default=200.0,
                    help="device work memory of the batched adjoint (grids beyond it run in later waves)")
    ap.add_argument("--batch-n", type=int, default=512)
    ap.add_argument("--batch-side-hi", type=int, default=4096)
    ap.add_argument("--batch-tlo", type=int, default=10)
    ap.add_argument("--batch-thi", type=int, default=500)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.precision:
        return run_precision(args, rank, world, local)
    if args.batch:
        return run_batch(args, rank, world, local)
    if args.adjoint:
        return run_adjoint_bench(args, rank, world, local)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
