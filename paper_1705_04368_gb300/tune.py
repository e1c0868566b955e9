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

# (grid, skin) pairs giving MD cell widths (= list radii at rc = 2.5) of 2.75 ... 4.0
DEFAULT_CANDIDATES = ((0.25, 0.25), (0.5, 0.5), (0.25, 0.75), (0.5, 1.0), (0.25, 1.25),
                      (0.5, 1.5))


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
         timer: Optional[Callable] = None, path: Optional[str] = None, refresh: bool = False):
    """Best (grid, skin) for this workload; returns (params with them set, report).

    ``timer(params, x0, v0, steps, warmup) -> seconds per step`` defaults to a
    CUDA-event measurement; candidates whose grid does not divide the lattice
    spacing and box, or that fail to build, are skipped.
    """
    path = path or cache_path()
    key = workload_key(params, temperature)
    cache = _load(path)
    if key in cache and not refresh:
        g, sk = cache[key]["grid"], cache[key]["skin"]
        return replace(params, grid=g, skin=sk), {"key": key, "cached": True, **cache[key]}
    timer = timer or time_candidate
    results = []
    for g, sk in candidates:
        box = (params.box, params.box) if np.isscalar(params.box) else params.box
        if any(abs(v / g - round(v / g)) > 1e-9 for v in (params.dx, *box)):
            continue
        cand = replace(params, grid=float(g), skin=float(sk), sort_every=0)
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
