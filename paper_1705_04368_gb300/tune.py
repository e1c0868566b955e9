"""Autotuner for the neighbour-cell geometry of the MD step.

The step kernel's cost grows with the Verlet-list length (list radius = MD cell
width k g = rc + skin) while the re-sort + list rebuild cost falls with the
skin (fewer rebuilds).  The best trade-off depends on density, temperature and
system size, so it is measured: each candidate (grid g, skin) builds the
workload through the C ABI, runs a warm-up and then a timed stretch of MD steps
on the caller's stream, and the fastest candidate is kept.  Results are cached
in a JSON file keyed by a coarse description of the workload (particle count
and density to two significant digits, temperature, dt, rc), so a later run of
a similar workload reuses them without timing.
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import replace
from typing import Callable, Iterable, Optional

import numpy as np

from .binding import Params, Simulation

# (grid, skin) pairs giving MD cell widths (= list radii at rc = 2.5) of 2.75 ... 4.0,
# in steps of 0.25 and, on the 0.125 grid, 3.125 and 3.375 around the usual optimum
DEFAULT_CANDIDATES = ((0.25, 0.25), (0.5, 0.5), (0.125, 0.625), (0.25, 0.75), (0.125, 0.875),
                      (0.5, 1.0), (0.25, 1.25), (0.5, 1.5))


def cache_path() -> str:
    return os.environ.get("MDLG_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mdlg_gb300",
                                       "tune.json"))


def _sig(x: float) -> str:
    return f"{x:.2g}"


def workload_key(params: Params, temperature: float) -> str:
    box = (params.box, params.box) if np.isscalar(params.box) else params.box
    rho = params.n / (box[0] * box[1])
    return (f"n={_sig(params.n)} rho={_sig(rho)} T={_sig(temperature)} dt={params.dt:g} "
            f"rc={params.rcut:g} lags={','.join(str(l) for l in params.lag_steps)}")


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_candidate(params: Params, x0, v0, steps: int, warmup: int, stream=None) -> float:
    """Seconds per MD step of one candidate, CUDA events on the library's stream."""
    import torch
    s = stream if stream is not None else torch.cuda.Stream()
    with Simulation(params, x0, v0, stream=s) as sim:
        sim.step(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        sim.step(steps)
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps


def tune(params: Params, x0, v0, temperature: float,
         candidates: Iterable[tuple] = DEFAULT_CANDIDATES, steps: int = 140, warmup: int = 14,
         timer: Optional[Callable] = None, path: Optional[str] = None, refresh: bool = False,
         key: Optional[str] = None, extents: Optional[Iterable[float]] = None,
         keep_sort_every: bool = False):
    """Best (grid, skin) for this workload; returns (params with them set, report).

    ``timer(params, x0, v0, steps, warmup) -> seconds per step`` defaults to a
    CUDA-event measurement; candidates whose grid does not divide the lattice
    spacing and every box extent (``extents``, default the params' box), or that
    fail to build, are skipped.  ``key`` overrides the cache key;
    ``keep_sort_every`` keeps the caller's re-sort interval instead of letting
    the library derive one per candidate.
    """
    path = path or cache_path()
    key = key or workload_key(params, temperature)
    cache = _load(path)
    if key in cache and not refresh:
        g, sk = cache[key]["grid"], cache[key]["skin"]
        return replace(params, grid=g, skin=sk), {"key": key, "cached": True, **cache[key]}
    timer = timer or time_candidate
    if extents is None:
        extents = (params.box, params.box) if np.isscalar(params.box) else params.box
    extents = [float(v) for v in extents]
    results = []
    for g, sk in candidates:
        if any(abs(v / g - round(v / g)) > 1e-9 for v in (params.dx, *extents)):
            continue
        cand = replace(params, grid=float(g), skin=float(sk))
        if not keep_sort_every:
            cand = replace(cand, sort_every=0)
        try:
            sec = float(timer(cand, x0, v0, steps, warmup))
        except Exception as exc:       # a candidate that cannot be built is skipped
            results.append({"grid": g, "skin": sk, "error": str(exc)})
            continue
        results.append({"grid": g, "skin": sk, "sec_per_step": sec})
    timed = [r for r in results if "sec_per_step" in r]
    if not timed:
        raise RuntimeError(f"no tuning candidate could be timed: {results}")
    best = min(timed, key=lambda r: r["sec_per_step"])
    entry = {"grid": best["grid"], "skin": best["skin"], "sec_per_step": best["sec_per_step"],
             "candidates": results, "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    cache[key] = entry
    _store(path, cache)
    return replace(params, grid=best["grid"], skin=best["skin"]), {"key": key, "cached": False,
                                                                   **entry}


def time_batch_candidate(params: Params, ns, boxes, x0, v0, steps: int, warmup: int,
                         stream=None) -> float:
    """Seconds per MD step of a replica batch under one candidate geometry."""
    import torch
    from .binding import BatchSimulation
    s = stream if stream is not None else torch.cuda.Stream()
    with BatchSimulation(params, ns, boxes, x0, v0, stream=s) as bt:
        bt.step(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        bt.step(steps)
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps


def tune_batch(params: Params, ns, boxes, x0, v0, temperature: float,
               candidates: Iterable[tuple] = DEFAULT_CANDIDATES, steps: int = 140,
               warmup: int = 14, path: Optional[str] = None, refresh: bool = False):
    """Best (grid, skin) for a batch of replicas (every system shares the geometry);
    returns (params, report).  The caller's re-sort interval is kept (0: the library
    derives one per candidate)."""
    ns = np.asarray(ns)
    boxes = np.asarray(boxes, dtype=np.float64)
    rho = float(ns.sum() / np.prod(boxes, axis=1).sum())
    key = (f"batch nsys={len(ns)} n={_sig(float(ns.sum()))} rho={_sig(rho)} "
           f"T={_sig(temperature)} dt={params.dt:g} rc={params.rcut:g} "
           f"sort_every={params.sort_every}")

    def timer(cand, x0_, v0_, steps_, warmup_):
        return time_batch_candidate(cand, ns, boxes, x0_, v0_, steps_, warmup_)

    return tune(params, x0, v0, temperature, candidates, steps, warmup, timer=timer, path=path,
                refresh=refresh, key=key, extents=boxes.ravel(), keep_sort_every=True)
