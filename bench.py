#!/usr/bin/env python
"""Throughput of the FVLBM D2Q9 step on one or more GB300 GPUs.

Workload (default): a batched solve of 256 heterogeneous instances advanced by
one launch sequence per stage -- jittered Couette channels (64x16, 2048
triangles), tanh-stretched lid-driven cavities (128^2 quads, 1:20) and
cylinder hybrids (100x200 O-grid quads + 100 rings of triangles, 60,000 cells)
in thirds, Reynolds number log-uniform in [10, 1000] (seed 2018), RK2, FP32
arithmetic on the deviation g = f - w.  ~6.7 M cells; the f state alone is
~240 MB, larger than the 129 MB L2, so no L2 flush is needed between steps.

One JSON line on rank 0: MCUPS (million cell updates per second; an RK2 step
counts once), the same workload in FP64 for the mixed/FP64 ratio and its
error, the roofline of the stage kernels, the CPU oracle baseline, an
end-to-end number through the C ABI with host buffers, and the SM clocks seen.

--impl reference times the FP64 CPU oracle (the only reference this method
has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D2Q9 MCUPS mixed vs FP64 at fixed error, %HBM peak; p50/p99 solve latency"
HBM_FALLBACK_GBS = 6800.0


# ----------------------------------------------------------------------------- workload
def batch_instances(n_inst: int, seed: int = 2018, small: bool = False, rank: int = 0):
    """(meshgen meshes by variant, list of (variant key, tau, u0)) for the batch.

    Rank r of a multi-GPU run solves its own batch (seed + r): the same mix and
    cell count on every GPU, different Reynolds numbers (weak scaling)."""
    from paper_1812_00390_gb300 import meshgen as mg
    specs = mg.batch_specs(n_inst, seed=seed + rank)
    variants = {}
    out = []
    for k, sp in enumerate(specs):
        kind, re_ = sp["kind"], sp["re"]
        if kind == "couette":
            key = ("couette", k % 4)
            if key not in variants:
                variants[key] = mg.couette(nx=16 if small else 64, ny=4 if small else 16, U=0.1,
                                           seed=1812 + key[1])
            H = 4.0 if small else 16.0
            tau = 3.0 * 0.1 * H / re_
            u0 = (0.0, 0.0)
        elif kind == "cavity":
            key = ("cavity", 0)
            if key not in variants:
                variants[key] = mg.cavity(32 if small else 128, 20.0, U=0.1)
            tau = 3.0 * 0.1 * 1.0 / re_
            u0 = (0.0, 0.0)
        else:
            key = ("cylinder", k % 2)
            if key not in variants:
                variants[key] = (mg.cylinder_hybrid(n_rad=25, n_circ=50, n_tri_rings=25, seed=100 + key[1])
                                 if small else mg.cylinder_hybrid(seed=100 + key[1]))
            tau = 3.0 * 0.05 * 1.0 / re_
            u0 = (0.05, 0.0)
        out.append((key, tau, u0))
    return variants, out


def build_solver(fv, variants, inst, precision, scheme="rk2", handles=None, kernel=0):
    handles = handles or {k: fv.Mesh(m) for k, m in variants.items()}
    mesh = fv.Mesh.concat([handles[k] for k, _, _ in inst])
    params = [fv.make_params(tau, scheme=scheme, precision=precision, u0=u0, kernel=kernel)
              for _, tau, u0 in inst]
    return fv.Solver(mesh, params), handles


def tune_kernel(fv, handles, inst, precision, scheme="rk2", n_sample=64, steps=20):
    """Stage-kernel variant chosen by the library's autotuner on the first
    n_sample instances of the batch (all three kinds)."""
    sub = inst[:n_sample]
    mesh = fv.Mesh.concat([handles[k] for k, _, _ in sub])
    params = [fv.make_params(tau, scheme=scheme, precision=precision, u0=u0) for _, tau, u0 in sub]
    return fv.autotune(mesh, params, steps=steps)


def tile_plan_summary(fv, mesh, inst, kernel):
    """The fused stage's tile plan of the batch (fvlbm_plan_info, on the host):
    tiles, cells per tile, the 1-ring cells whose gradients each tile
    recomputes, and the modelled shared-memory wavefronts per warp access."""
    params = [fv.make_params(tau, scheme="rk2", precision="fp32", u0=u0, kernel=kernel) for _, tau, u0 in inst]
    i = fv.plan_info(mesh, params)
    keep = ("stage_kernel", "n_tiles", "mean_tile_cells", "mean_ring1_cells", "mean_local_cells",
            "max_local_cells", "max_faces", "face_table_waves", "gather_waves", "violations")
    return {k: i[k] for k in keep}


# ----------------------------------------------------------------------------- single configs
def config_runs(fv, torch, dev, steps: int = 30):
    """MCUPS of the single-mesh configurations.  Their state fits in L2, so every
    timed step is preceded by writing a 256 MB buffer (L2 flush) on the
    solver's stream, outside the timed events ("cold": device time of a step
    that starts from DRAM; the host enqueues the step while the flush runs);
    "from_idle_host" times the same from a synchronised host, so it adds the
    launch of one step (binding, C ABI, graph launch) to an idle GPU; "warm"
    is the same solver replaying its graphs with the mesh resident in L2."""
    from paper_1812_00390_gb300 import meshgen as mg
    cases = [
        ("couette_32x8_euler_fp64", mg.couette(), 3 * 0.1 * 8 / 10, "euler", "fp64", (0.0, 0.0)),
        ("cavity_128_re400_rk2_fp32", mg.cavity(128, 20.0), 3 * 0.1 / 400, "rk2", "fp32", (0.0, 0.0)),
        ("cavity_128_re400_rk2_fp64", mg.cavity(128, 20.0), 3 * 0.1 / 400, "rk2", "fp64", (0.0, 0.0)),
        ("cylinder_60k_re40_rk2_fp16split", mg.cylinder_hybrid(), 3 * 0.05 / 40, "rk2", "fp16", (0.05, 0.0)),
        ("cylinder_60k_re40_rk2_fp32", mg.cylinder_hybrid(), 3 * 0.05 / 40, "rk2", "fp32", (0.05, 0.0)),
    ]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
    out = {}
    for name, m, tau, scheme, prec, u0 in cases:
        h = fv.Mesh(m)
        best, tune = fv.autotune(h, fv.make_params(tau, scheme=scheme, precision=prec, u0=u0), steps=64)
        s = fv.Solver(h, fv.make_params(tau, scheme=scheme, precision=prec, u0=u0, kernel=best))
        s.step(5)
        s.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            with torch.cuda.stream(s.stream):
                flush.fill_(1)
            a.record(s.stream)
            s.step(1)
            b.record(s.stream)
        s.sync()
        cold = sum(a.elapsed_time(b) for a, b in ev) / steps
        for a, b in ev:
            flush.fill_(1)
            torch.cuda.current_stream(dev).synchronize()
            a.record(s.stream)
            s.step(1)
            b.record(s.stream)
        s.sync()
        idle = sum(a.elapsed_time(b) for a, b in ev) / steps
        a, b = ev[0]
        a.record(s.stream)
        s.step(10 * steps)
        b.record(s.stream)
        s.sync()
        warm = a.elapsed_time(b) / (10 * steps)
        out[name] = {"cells": m.n_cell, "stage_kernel": best,
                     "autotune_ms_per_step": {str(k): v for k, v in tune.items()},
                     "cold_l2_mcups": m.n_cell / (cold / 1e3) / 1e6,
                     "warm_l2_mcups": m.n_cell / (warm / 1e3) / 1e6, "cold_ms_per_step": cold,
                     "warm_ms_per_step": warm,
                     "from_idle_host_mcups": m.n_cell / (idle / 1e3) / 1e6, "from_idle_host_ms_per_step": idle}
        s.close()
    return out


def error_per_config(fv):
    """Mixed-precision error at fixed step counts on the single configurations,
    against the FP64 mode of the same configuration on the GPU (which the
    tests hold to the FP64 oracle within 1e-12): max relative |u| error (of
    the largest FP64 speed) and max |rho| error, per storage precision, each
    run with the automatic stage kernel."""
    from paper_1812_00390_gb300 import meshgen as mg
    cav, cyl = mg.cavity(128, 20.0), mg.cylinder_hybrid()
    cases = [("cavity_128_re400", cav, 3 * 0.1 / 400, (0.0, 0.0), 10_000),
             ("cavity_128_re1000", cav, 3 * 0.1 / 1000, (0.0, 0.0), 10_000),
             ("cylinder_60k_re20", cyl, 3 * 0.05 / 20, (0.05, 0.0), 2000),
             ("cylinder_60k_re40", cyl, 3 * 0.05 / 40, (0.05, 0.0), 10_000),
             ("cylinder_60k_re100", cyl, 3 * 0.05 / 100, (0.05, 0.0), 2000)]
    out = {}
    for name, m, tau, u0, n in cases:
        h = fv.Mesh(m)
        ref = fv.Solver(h, fv.make_params(tau, scheme="rk2", precision="fp64", u0=u0))
        ref.step(n)
        r64, u64 = ref.macros()
        ref.close()
        row = {"cells": m.n_cell, "steps": n, "scheme": "rk2"}
        for prec in ("fp32", "fp16", "bf16"):
            s = fv.Solver(h, fv.make_params(tau, scheme="rk2", precision=prec, u0=u0))
            s.step(n)
            r, u = s.macros()
            row[prec] = {"max_rel_velocity": float(np.abs(u - u64).max() / np.abs(u64).max()),
                         "max_abs_density": float(np.abs(r - r64).max()), "stage_kernel": s.stage_kernel()}
            s.close()
        out[name] = row
    return out


def roofline_synthetic(fv, torch, peak_gbs, steps: int = 20):
    """The interior-only roofline case: a fully periodic jittered-triangle domain
    of 2048 x 1024 x 2 = 4,194,304 cells (no boundary faces; state and geometry
    far larger than L2), uniform flow (the kernels do the same work for any
    state), RK2, in FP64, FP32 and FP16 split storage, each with the automatic
    stage kernel.  Per precision: MCUPS and the stage kernels' algorithmic HBM
    rate (state bytes only: 5 x the stored bytes per cell and RK2 step)."""
    from paper_1812_00390_gb300 import meshgen as mg
    m = mg.periodic_tri(2048, 1024, lx=2048.0, ly=1024.0, seed=2048)
    h = fv.Mesh(m)
    out = {"cells": m.n_cell, "mesh": "periodic jittered triangles 2048 x 1024 x 2", "scheme": "rk2"}
    for prec, sb in (("fp32", 36), ("fp16", 24), ("fp64", 72)):   # stored bytes per cell
        s = fv.Solver(h, fv.make_params(0.1, scheme="rk2", precision=prec, u0=(0.02, 0.01)))
        s.step(3)
        s.sync()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s.stream)
        s.step(steps)
        e.record(s.stream)
        s.sync()
        ms = a.elapsed_time(e) / steps
        kern, _ = s.profile(3)
        stage_ms = float(sum(kern))
        alg = 5 * sb / 2 * m.n_cell               # bytes per stage (mean of the two RK2 stages)
        out[prec] = {"mcups": m.n_cell / (ms / 1e3) / 1e6, "ms_per_step": ms, "stage_ms": stage_ms,
                     "stage_kernel": "two-kernel" if len(kern) == 2 else "fused 512",
                     "algorithmic_gbs": alg / (stage_ms / 1e3) / 1e9,
                     "frac_of_hbm_peak": alg / (stage_ms / 1e3) / 1e9 / peak_gbs}
        s.close()
    # the same mesh as a partitioned solve on this GPU (recursive bisection,
    # two ghost rings, one halo exchange per stage), FP32: the cost of the
    # partitioning itself (a multi-GPU run would place one part per GPU)
    out["partitioned_fp32"] = {}
    for parts in (2, 4):
        plan = fv.Partition(h, parts)
        dd = fv.DDSolver(plan, fv.make_params(0.1, scheme="rk2", precision="fp32", u0=(0.02, 0.01)))
        dd.step(3)
        dd.sync()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(dd.stream)
        dd.step(steps)
        e.record(dd.stream)
        dd.sync()
        ms = a.elapsed_time(e) / steps
        ghosts = sum(plan.info(p)["n_recv"] for p in range(parts))
        out["partitioned_fp32"][str(parts)] = {
            "mcups": m.n_cell / (ms / 1e3) / 1e6, "ms_per_step": ms,
            "relative_to_undivided": out["fp32"]["ms_per_step"] / ms,
            "ghost_cells": ghosts, "launches_per_step": dd.stage_kernel()[1]}
        dd.close()
        plan.close()
    return out


# ----------------------------------------------------------------------------- ranks
def reduce_max(x: float, dist, device=None) -> float:
    """Largest value over all ranks (the slowest rank's time); x itself at N = 1."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self._t.join(timeout=5)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- roofline inputs
GEOMETRY_BYTES_FP32 = 4 * (8 + 3 * 2 * 4)   # per cell and stage, 4 face slots


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except (ValueError, OSError):
            pass
    return HBM_FALLBACK_GBS, "fallback"


def kernel_source_sha() -> str:
    """Hash of the code (comments and blank space stripped) that decides what
    the stage kernels do and read: the kernels and the device storage (whole
    files), the shared-memory capacities and the host-side tile planner (their
    sections of the other files)."""
    csrc = os.path.join(ROOT, "paper_1812_00390_gb300", "csrc")

    def code(txt):
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        return re.sub(r"\s+", " ", txt).strip()

    h = hashlib.sha256()
    for f in ("fvlbm_stage.cuh", "fvlbm_device.cuh"):
        h.update(code(open(os.path.join(csrc, f)).read()).encode())
    for f, begin, end in (("fvlbm_internal.h", "struct TileDims", "};"),
                          ("fvlbm_solver.cpp", "struct TilePlan {", "// Offsets of every array")):
        txt = open(os.path.join(csrc, f)).read()
        a = txt.index(begin)
        h.update(code(txt[a:txt.index(end, a)]).encode())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str):
    """(DRAM bytes per cell and stage, where they come from) for the stage
    kernel of this workload from profiles/ncu_traffic.json (written by hand
    from an ncu capture, keyed by the kernel-source hash), or (None, reason)
    when it is missing or was taken on other kernel source."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))[workload]
    except (OSError, ValueError, KeyError):
        return None, "no ncu capture recorded for this workload"
    if d.get("kernel_source_sha") != kernel_source_sha():
        return None, "the recorded ncu capture is of other kernel source"
    return float(d["dram_bytes_per_cell_stage"]), d.get("capture", "")


# ----------------------------------------------------------------------------- oracle baseline
def oracle_mcups(variants, inst, budget_s: float, steps_cap: int = 100000, threads: int = 0):
    """The FP64 oracle, as it stands, on one instance of each kind, RK2, with
    `threads` OpenMP threads (0: all the host's cores)."""
    import oracle
    oracle.build()
    used = oracle.threads(threads if threads > 0 else (os.cpu_count() or 1))
    picked = {}
    for key, tau, u0 in inst:
        picked.setdefault(key[0], (key, tau, u0))
    runs = []
    for key, tau, u0 in picked.values():
        m = variants[key]
        o = oracle.Oracle(m)
        o.set_equilibrium(1.0, u0)
        dt = o.cfl_dt(0.5, max(0.1, abs(u0[0])), tau, "rk2")
        runs.append((o, m.n_cell, tau, dt))
    cells = sum(r[1] for r in runs)
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s and steps < steps_cap:
        for o, _, tau, dt in runs:
            o.run("rk2", tau, dt, 1)
        steps += 1
    el = time.perf_counter() - t0
    sample = (f"{len(runs)} instances ({'+'.join(k for k in picked)}, {cells} cells), "
              f"{steps} RK2 steps each, {el:.1f} s, {used} thread{'s' if used > 1 else ''}")
    return cells * steps / el / 1e6, used, sample, el, steps, cells


# ----------------------------------------------------------------------------- arms
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    small = args.workload == "batch256-small"
    variants, inst = batch_instances(256, small=small)
    import oracle
    oracle.build()
    picked = {}
    for key, tau, u0 in inst:
        picked.setdefault(key[0], (key, tau, u0))
    runs = []
    for key, tau, u0 in picked.values():
        o = oracle.Oracle(variants[key])
        o.set_equilibrium(1.0, u0)
        runs.append((o, variants[key].n_cell, tau, o.cfl_dt(0.5, max(0.1, abs(u0[0])), tau, "rk2")))
    cells = sum(r[1] for r in runs)
    for _ in range(args.warmup):
        for o, _, tau, dt in runs:
            o.run("rk2", tau, dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for o, _, tau, dt in runs:
            o.run("rk2", tau, dt, 1)
    el = time.perf_counter() - t0
    v = cells * args.steps / el / 1e6
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"one instance of each kind ({cells} cells) per step, RK2"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MCUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "sample": sample, "scheme": "rk2"},
            "cpu_baseline": {"value": v, "unit": "MCUPS", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "MCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = local if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1812_00390_gb300 import fvlbm as fv

    small = args.workload == "batch256-small"
    variants, inst = batch_instances(args.instances, small=small, rank=rank)

    # CPU oracle baseline first (rank 0 only), before any GPU work
    cpu = None
    if rank == 0 and not args.no_cpu:
        v, thr, sample, _, _, _ = oracle_mcups(variants, inst, args.cpu_seconds)
        v1, _, sample1, _, _, _ = oracle_mcups(variants, inst, args.cpu_seconds / 2, threads=1)
        cpu = {"value": v, "unit": "MCUPS", "cores": thr, "kind": "oracle", "sample": sample,
               "single_thread": {"value": v1, "unit": "MCUPS", "cores": 1, "sample": sample1}}

    handles = {k: fv.Mesh(m) for k, m in variants.items()}
    # the batch runs the library's automatic choice (or --kernel); the
    # autotuner's timings of every variant on a sample are reported beside it
    tune32, pick32 = {}, None
    if args.kernel is None:
        pick32, tune32 = tune_kernel(fv, handles, inst, "fp32")
    kernel32 = args.kernel if args.kernel is not None else 0
    s32, _ = build_solver(fv, variants, inst, "fp32", handles=handles, kernel=kernel32)
    kernel32 = s32.stage_kernel()
    n_cells = s32.n_cell
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def timed(solver, k):
        solver.step(args.warmup)
        solver.sync()
        barrier()
        with ClockSampler(dev) as clk:
            start.record(solver.stream)        # events on the stream the solver launches on
            for _ in range(k):
                solver.step(1)
            end.record(solver.stream)
            end.synchronize()
        ms = start.elapsed_time(end)
        solver.sync()
        barrier()
        ms = reduce_max(ms, dist, f"cuda:{dev}")
        return ms, clk.summary()

    ms32, clocks = timed(s32, args.steps)
    value = n_cells * world * args.steps / (ms32 / 1e3) / 1e6

    # per-kernel device times (events around each launch)
    kern_ms, _ = s32.profile(max(3, args.steps // 4))
    launches = s32.launches_per_step() * args.steps

    # FP64 on the same workload, and the mixed-mode error against it
    ms64 = None
    err = None
    fp64_peak = None
    if not args.no_fp64:
        fp64_peak = fv.fma_peak(dev, fp64=True)
        k64 = max(3, args.steps // 8)
        kernel64 = args.kernel if args.kernel is not None else 0
        s64, _ = build_solver(fv, variants, inst, "fp64", handles=handles, kernel=kernel64)
        kernel64 = s64.stage_kernel()
        ms64, _ = timed(s64, k64)
        ms64 /= k64
        # same number of steps from Step 0 in both modes
        n_cmp = args.warmup + args.steps + args.steps
        s64.close()
        s64, _ = build_solver(fv, variants, inst, "fp64", handles=handles, kernel=kernel64)
        s64.step(n_cmp)
        _, u64 = s64.macros()
        s64.close()
        ref32, _ = build_solver(fv, variants, inst, "fp32", handles=handles, kernel=kernel32)
        ref32.step(n_cmp)
        _, u32 = ref32.macros()
        ref32.close()
        err = float(np.abs(u32 - u64).max() / np.abs(u64).max())
        err_steps = n_cmp

    # FP16 split storage (FP32 rho, rho u; 16-bit non-equilibrium part) on the same workload
    fp16 = None
    if not args.no_fp16:
        s16, _ = build_solver(fv, variants, inst, "fp16", handles=handles, kernel=kernel32)
        ms16, _ = timed(s16, max(3, args.steps // 4))
        ms16 /= max(3, args.steps // 4)
        fp16 = {"value": n_cells * world / (ms16 / 1e3) / 1e6, "unit": "MCUPS", "ms_per_step": ms16,
                "storage": "rho-1, rho u in FP32 + 6 non-equilibrium components in FP16 (24 B/cell)"}
        if err is not None:
            s16.close()
            s16, _ = build_solver(fv, variants, inst, "fp16", handles=handles, kernel=kernel32)
            s16.step(err_steps)
            _, u16 = s16.macros()
            fp16["max_rel_velocity_error_vs_fp64"] = float(np.abs(u16 - u64).max() / np.abs(u64).max())
            fp16["steps"] = err_steps
        s16.close()

    # roofline of the stage kernels: algorithmic f traffic per RK2 stage,
    # stage 1 reads f0 and writes f1, stage 2 reads f1 and f0 and writes f
    bytes_store = 4
    alg_per_cell_stage = (2 + 3) * 9 * bytes_store / 2.0        # 90 B, mean over the 2 stages
    stage_ms = float(sum(kern_ms))
    achieved = alg_per_cell_stage * n_cells / (stage_ms / 1e3) / 1e9
    peak, peak_src = measured_peaks()
    traffic_pc, traffic_src = ncu_traffic(args.workload)
    names = ["stage_tile_kernel"] if len(kern_ms) == 1 else ["face_values_kernel", "update_kernel"]
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": (traffic_pc * n_cells if traffic_pc else None),
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per cell and stage, "
                               "profiles/ncu_traffic.json (%s), scaled to this launch's cells" % traffic_src
                               if traffic_pc else traffic_src),
            "kernel": ("stage_tile_kernel (one fused RK2 stage)" if len(kern_ms) == 1
                       else "one RK2 stage = face_values_kernel + update_kernel"),
            "kernel_ms": {n: float(t) for n, t in zip(names, kern_ms)},
            "algorithmic_bytes_per_launch": alg_per_cell_stage * n_cells,
            # the same with the per-slot geometry the stage reads (8-byte descriptor and three
            # FP32 2-vectors per slot, 4 slots): 90 + 128 B per cell and stage
            "with_geometry": {"bytes_per_launch": (alg_per_cell_stage + GEOMETRY_BYTES_FP32) * n_cells,
                              "achieved": (alg_per_cell_stage + GEOMETRY_BYTES_FP32) * n_cells
                              / (stage_ms / 1e3) / 1e9,
                              "frac": (alg_per_cell_stage + GEOMETRY_BYTES_FP32) * n_cells
                              / (stage_ms / 1e3) / 1e9 / peak},
            # ncu's DRAM bytes per launch over the live launch time
            "dram_frac": (traffic_pc * n_cells / (stage_ms / 1e3) / 1e9 / peak if traffic_pc else None),
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
            else f"{peak_src} {HBM_FALLBACK_GBS:.0f} GB/s"}
    if kernel32 != 1:
        roof["tile_plan"] = tile_plan_summary(fv, s32.mesh, inst, kernel32)

    # end to end through the C ABI with host buffers: each e2e step uploads the
    # state from host memory (set_f), advances e2e_inner time steps and reads
    # the solution back (macros: rho and u of every cell into host arrays).
    # The headline uses pinned host buffers; the same loop with pageable numpy
    # arrays is reported beside it.
    e2e_inner = args.e2e_inner
    e2e_val = e2e_pageable = None
    if args.e2e_steps > 0:
        f_host = s32.get_f()
        f_pinned = torch.empty(f_host.shape, dtype=torch.float64, pin_memory=True).numpy()
        f_pinned[...] = f_host
        rho_pinned = torch.empty(n_cells, dtype=torch.float64, pin_memory=True).numpy()
        u_pinned = torch.empty((n_cells, 2), dtype=torch.float64, pin_memory=True).numpy()
        rho_page, u_page = np.zeros(n_cells), np.zeros((n_cells, 2))

        def e2e_loop(buf, rho_out, u_out):
            s32.sync()
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                s32.set_f(buf)
                s32.step(e2e_inner)
                s32.macros_into(rho_out, u_out)
            torch.cuda.synchronize()
            return n_cells * world * e2e_inner * args.e2e_steps / (time.perf_counter() - t0) / 1e6

        e2e_pageable = e2e_loop(f_host, rho_page, u_page)
        e2e_val = e2e_loop(f_pinned, rho_pinned, u_pinned)
        # the read-back is the solution: it equals what macros() returns
        _, u_chk = s32.macros()
        e2e_readback_ok = bool(np.array_equal(u_chk, u_pinned))

    configs = config_runs(fv, torch, dev) if (args.configs and rank == 0) else None
    roof_syn = roofline_synthetic(fv, torch, peak) if (args.configs and rank == 0) else None
    errs = error_per_config(fv) if (args.configs and rank == 0) else None

    # serving stream (config 5): Poisson arrivals of tandem / single cylinder
    # solves, plus every fourth request a small cavity that converges, on the
    # continuous-batching server, swept over the arrival rate; the same
    # requests (meshes, Reynolds numbers, arrival order) at every rate, their
    # arrival times scaled by 1 / rate
    serving = None
    if args.serving > 0 and rank == 0:
        from paper_1812_00390_gb300 import serving as sv
        base = sv.request_mix(args.serving, seed=390, rate=1.0, cavity_every=4)
        meshes = [sv.build_mesh(sp) for sp in base]
        srv = fv.Server(int(args.serving_arena_gb * 1e9), device=dev, n_streams=8, max_active=32,
                        check_interval=1000, residual_tol=1e-8, max_steps=args.serving_steps)
        per_rate = []
        for rate in [float(x) for x in args.serving_rates.split(",")]:
            specs = [dataclasses.replace(sp, arrival=sp.arrival / rate) for sp in base]
            lat, infos, wall, cells = sv.run_poisson(srv, fv, specs, meshes)
            row = sv.summarize_rate(infos, specs, wall, cells, 1e-8)
            row["arrival_rate_per_s"] = rate
            per_rate.append(row)
        srv.close()
        serving = {"per_rate": per_rate, "precision": "fp32", "scheme": "rk2",
                   "requests_per_rate": args.serving,
                   "stop": f"residual <= 1e-8 (checked every 1000 steps) or {args.serving_steps} steps",
                   "mix": "3/8 tandem double-cylinder (50k-150k cells), 3/8 single cylinder (20k-60k), "
                          "1/4 cavity 16x16 at Re 5-10 (converges); cylinders Re U[20, 200]",
                   "cells_per_request": [int(m.n_cell) for m in meshes],
                   "latency": "p50/p99 of submission to completion over all requests; converged_*: over the "
                              "requests that reached the tolerance; queue_*: submission to admission",
                   "arena_gb": args.serving_arena_gb}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MCUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "n_instances": args.instances, "n_cells": n_cells,
                       "scheme": "rk2", "precision": "fp32 deviation (g = f - w)",
                       "l2": "inputs larger than L2 (f state %.0f MB per GPU)" % (n_cells * 9 * 4 / 1e6),
                       "parallelism": "instances replicated per GPU (weak scaling)" if world > 1 else "1 GPU",
                       "stage_kernel": kernel32,
                       "autotune_ms_per_step": {str(k): v for k, v in tune32.items()},
                       "autotune_pick": pick32},
            "fp64": {"value": (n_cells * world / (ms64 / 1e3) / 1e6) if ms64 else None, "unit": "MCUPS",
                     "ms_per_step": ms64, "stage_kernel": kernel64 if ms64 else None,
                     "fma_peak_tflops": fp64_peak,
                     "note": "FP64 stage is bound by the FP64 units, not HBM"},
            "fp16_split": fp16,
            "mixed_over_fp64": (value / (n_cells * world / (ms64 / 1e3) / 1e6)) if ms64 else None,
            "mixed_error_vs_fp64": ({"max_rel_velocity": err, "steps": err_steps} if err is not None else None),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": ({"value": e2e_val, "unit": "MCUPS", "h2d_bytes_per_step": n_cells * 9 * 8,
                     "d2h_bytes_per_step": n_cells * 3 * 8,
                     "definition": (f"per e2e step: set_f of the whole state from host memory (FP64, "
                                    f"caller order) + {e2e_inner} time steps + macros (rho, u of every cell "
                                    f"into host arrays); the byte counts are per e2e step"),
                     "host_memory": "pinned", "pageable_value": e2e_pageable,
                     "readback_equals_macros": e2e_readback_ok}
                    if e2e_val is not None else None),
            "serving": serving,
            "single_configs": configs,
            "error_per_config": errs,
            "roofline_synthetic": roof_syn,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch256", choices=["batch256", "batch256-small"])
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--e2e-inner", type=int, default=100)
    ap.add_argument("--serving", type=int, default=32, help="requests per arrival rate in the serving leg (0 = skip)")
    ap.add_argument("--serving-rates", default="1,2,4,8,16", help="Poisson arrival rates per second, swept")
    ap.add_argument("--serving-steps", type=int, default=20000)
    ap.add_argument("--serving-arena-gb", type=float, default=8.0)
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the single-mesh configurations")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-fp16", action="store_true")
    ap.add_argument("--kernel", type=int, default=None,
                    help="stage kernel variant (1, 128, 256, 512, 1024) instead of the autotuner's choice")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
