"""Serving workload: Poisson arrivals of cylinder solves on the continuous-
batching server (fvlbm_server_* in the C ABI).

A request is a tandem double-cylinder hybrid mesh (gap ratio L/D uniform in
[1.5, 5], 50k-150k cells) or a single-cylinder hybrid mesh (20k-60k cells),
half and half, with Re uniform in [20, 200], u_inf = 0.05, started from the
free stream and solved until the velocity residual of Sec. 3.2 reaches the
tolerance or the step cap.  Optionally a fraction of the requests are small
steady lid-driven cavities (16 x 16 quads, lid 0.1, Re uniform in [5, 10],
Sec. 3.2) that do reach e <= 1e-8 within the cap (about 9000 steps), so that
time-to-converged is measured as well: the cylinder wakes keep developing for
far longer than the cap allows.  Latency of a request = completion -
submission; queueing delay = admission - submission (wall clock of the
server).
"""
from __future__ import annotations

import dataclasses
import time
from typing import List, Optional

import numpy as np

from . import meshgen as mg


@dataclasses.dataclass
class RequestSpec:
    kind: str          # "tandem", "single" or "cavity"
    re: float
    gap: float
    target_cells: int
    seed: int
    arrival: float = 0.0


def request_mix(n: int, seed: int = 390, rate: float = 1.0, tandem_cells=(50_000, 150_000),
                single_cells=(20_000, 60_000), cavity_every: int = 0) -> List[RequestSpec]:
    """n requests, half tandem / half single cylinder, Poisson arrivals at `rate`
    per second; with cavity_every = m > 0, every m-th request is a small
    converging cavity instead."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for k in range(n):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        if cavity_every > 0 and k % cavity_every == cavity_every - 1:
            out.append(RequestSpec("cavity", float(rng.uniform(5, 10)), 0.0, 256, int(rng.integers(1 << 30)), t))
        elif k % 2 == 0:
            out.append(RequestSpec("tandem", float(rng.uniform(20, 200)), float(rng.uniform(1.5, 5.0)),
                                   int(rng.uniform(*tandem_cells)), int(rng.integers(1 << 30)), t))
        else:
            out.append(RequestSpec("single", float(rng.uniform(20, 200)), 0.0,
                                   int(rng.uniform(*single_cells)), int(rng.integers(1 << 30)), t))
    return out


def build_mesh(spec: RequestSpec) -> mg.Mesh:
    if spec.kind == "cavity":
        return mg.cavity(16, 1.0, U=0.1)
    if spec.kind == "tandem":
        n_circ = max(64, int(round((spec.target_cells - 12_000) / 256.0)))
        return mg.tandem_cylinders(gap_ratio=spec.gap, n_circ=n_circ, grade=0.06, seed=spec.seed % 1000)
    n_tri = max(1, int(round((spec.target_cells - 5_000) / 200.0)))
    return mg.cylinder_hybrid(n_rad=50, n_circ=100, n_tri_rings=n_tri, first=0.003, growth=1.08,
                              seed=spec.seed % 1000)


def request_params(fv, spec: RequestSpec, precision: str = "fp32", scheme: str = "rk2", u_inf: float = 0.05,
                   device: int = 0):
    if spec.kind == "cavity":                  # side 1, lid 0.1, at rest
        return fv.make_params(3.0 * 0.1 / spec.re, scheme=scheme, precision=precision, device=device)
    tau = 3.0 * u_inf * 1.0 / spec.re          # D = 1, tau = 3 nu
    return fv.make_params(tau, scheme=scheme, precision=precision, u0=(u_inf, 0.0), device=device)


def run_poisson(server, fv, specs: List[RequestSpec], meshes, precision: str = "fp32",
                time_limit: float = 600.0):
    """Submit each request at its arrival time, poll until all are done.
    Returns (latencies [s], per-request info, wall seconds, cell updates)."""
    handles = [fv.Mesh(m) for m in meshes]
    params = [request_params(fv, s, precision) for s in specs]
    ids = [None] * len(specs)
    t0 = time.perf_counter()
    start_cells = server.stats()["cell_steps"]
    nxt = 0
    done = 0
    while done < len(specs):
        now = time.perf_counter() - t0
        while nxt < len(specs) and specs[nxt].arrival <= now:
            ids[nxt] = server.submit(handles[nxt], params[nxt])
            nxt += 1
        if server.stats()["active"] == 0 and server.stats()["queued"] == 0:
            if nxt < len(specs):
                time.sleep(max(0.0, min(0.01, specs[nxt].arrival - now)))
            continue
        done += server.poll()
        if time.perf_counter() - t0 > time_limit:
            raise TimeoutError("serving run exceeded its time limit")
    wall = time.perf_counter() - t0
    infos = [server.request(i) for i in ids]
    lat = np.array([x["t_done"] - x["t_submit"] for x in infos])
    cells = server.stats()["cell_steps"] - start_cells
    return lat, infos, wall, cells


def summarize(lat: np.ndarray, wall: float, cells: int) -> dict:
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "requests": int(len(lat)), "wall_s": wall,
            "aggregate_mcups": cells / wall / 1e6}


def summarize_rate(infos, specs, wall: float, cells: int, tol: float) -> dict:
    """Per-rate figures: latency (submission to completion) and queueing delay
    (submission to admission) percentiles over all requests, the same latency
    over the requests that converged (time to e <= tol), and the aggregate
    MCUPS over the run's wall time."""
    lat = np.array([x["t_done"] - x["t_submit"] for x in infos])
    queue = np.array([x["t_admit"] - x["t_submit"] for x in infos])
    conv = np.array([x["t_done"] - x["t_submit"] for x in infos if x["residual"] <= tol])
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
    out = summarize(lat, wall, cells)
    out.update({"queue_p50_s": pct(queue, 50), "queue_p99_s": pct(queue, 99),
                "converged": int(len(conv)), "converged_p50_s": pct(conv, 50), "converged_p99_s": pct(conv, 99),
                "kinds": {k: sum(1 for s in specs if s.kind == k) for k in ("tandem", "single", "cavity")}})
    return out
