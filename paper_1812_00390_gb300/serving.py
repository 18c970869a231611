"""Serving workload: Poisson arrivals of cylinder solves on the continuous-
batching server (fvlbm_server_* in the C ABI).

A request is a tandem double-cylinder hybrid mesh (gap ratio L/D uniform in
[1.5, 5], 50k-150k cells) or a single-cylinder hybrid mesh (20k-60k cells),
half and half, with Re uniform in [20, 200], u_inf = 0.05, started from the
free stream and solved until the velocity residual of Sec. 3.2 reaches the
tolerance or the step cap.  Latency of a request = completion - submission
(wall clock of the server).
"""
from __future__ import annotations

import dataclasses
import time
from typing import List, Optional

import numpy as np

from . import meshgen as mg


@dataclasses.dataclass
class RequestSpec:
    kind: str          # "tandem" or "single"
    re: float
    gap: float
    target_cells: int
    seed: int
    arrival: float = 0.0


def request_mix(n: int, seed: int = 390, rate: float = 1.0, tandem_cells=(50_000, 150_000),
                single_cells=(20_000, 60_000)) -> List[RequestSpec]:
    """n requests, half tandem / half single cylinder, Poisson arrivals at `rate` per second."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for k in range(n):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        if k % 2 == 0:
            out.append(RequestSpec("tandem", float(rng.uniform(20, 200)), float(rng.uniform(1.5, 5.0)),
                                   int(rng.uniform(*tandem_cells)), int(rng.integers(1 << 30)), t))
        else:
            out.append(RequestSpec("single", float(rng.uniform(20, 200)), 0.0,
                                   int(rng.uniform(*single_cells)), int(rng.integers(1 << 30)), t))
    return out


def build_mesh(spec: RequestSpec) -> mg.Mesh:
    if spec.kind == "tandem":
        n_circ = max(64, int(round((spec.target_cells - 12_000) / 256.0)))
        return mg.tandem_cylinders(gap_ratio=spec.gap, n_circ=n_circ, grade=0.06, seed=spec.seed % 1000)
    n_tri = max(1, int(round((spec.target_cells - 5_000) / 200.0)))
    return mg.cylinder_hybrid(n_rad=50, n_circ=100, n_tri_rings=n_tri, first=0.003, growth=1.08,
                              seed=spec.seed % 1000)


def request_params(fv, spec: RequestSpec, precision: str = "fp32", scheme: str = "rk2", u_inf: float = 0.05,
                   device: int = 0):
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
