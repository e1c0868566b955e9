"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This module holds input generation only -- none of the method's arithmetic (no
forces, no integration, no binning).  Both the FP64 oracle and the CUDA library
are fed from here, so neither ever produces the other's inputs.

Recipes (the paper's own trajectory is not available; these stand in for it):
  * Lennard-Jones gas: positions uniform in the periodic box (0, L]^2 with no
    pair closer than ``dmin`` (random sequential placement, place.c), Maxwell velocities at temperature T with the centre-of-mass
    velocity removed and rescaled so the kinetic energy is (N - 1) T (2N - 2
    degrees of freedom).  The paper starts from "a homogeneous distribution"
    with a kinetic energy for the target temperature.
  * Ideal gas: binary32 positions uniform in (0, L]^2, Maxwell velocities.
  * Binning snapshots: dyadic positions (multiples of 2^-bits) so that a value
    is exactly representable both as an FP64 coordinate and as integer base
    cell plus binary32 offset; a fraction of points sits exactly on cell
    boundaries to exercise the left-open / right-closed cell convention.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np


def box_for(n: int, rho: float, dx: float) -> float:
    """Box side sqrt(N / rho) rounded up to a multiple of the lattice spacing dx."""
    return math.ceil(math.sqrt(n / rho) / dx) * dx


def _uniform_open_closed(rng: np.random.Generator, size, L: float) -> np.ndarray:
    # rng.random is in [0, 1); L - L*u is in (0, L].
    return L - L * rng.random(size)


_HERE = os.path.dirname(os.path.abspath(__file__))
_PLACE_SRC = os.path.join(_HERE, "place.c")
_PLACE_LIB = os.path.join(_HERE, "_build", "libplace.so")
_place = None


def build(force: bool = False) -> str:
    """Compile the placement helper (plain C, gcc)."""
    os.makedirs(os.path.dirname(_PLACE_LIB), exist_ok=True)
    if force or not os.path.exists(_PLACE_LIB) or \
            os.path.getmtime(_PLACE_LIB) < os.path.getmtime(_PLACE_SRC):
        tmp = _PLACE_LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                        _PLACE_SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _PLACE_LIB)
    return _PLACE_LIB


def _nonoverlap(n: int, L: tuple, dmin: float, seed: int) -> np.ndarray:
    """Uniform positions in (0, L]^2 with every pair at least dmin apart (minimum image)."""
    global _place
    if _place is None:
        lib = ctypes.CDLL(build())
        lib.place_nonoverlap.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
                                         ctypes.c_void_p]
        lib.place_nonoverlap.restype = ctypes.c_int
        _place = lib
    x = np.empty((n, 2))
    rc = _place.place_nonoverlap(n, float(L[0]), float(L[1]), float(dmin),
                                 ctypes.c_uint64(seed & (2**64 - 1)), 100000,
                                 x.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise RuntimeError("non-overlapping placement failed (density too high for dmin)")
    return x


def maxwell_velocities(n: int, temperature: float, rng: np.random.Generator,
                       mass: float = 1.0) -> np.ndarray:
    """Maxwell velocities, zero total momentum, kinetic energy exactly (N-1) T."""
    v = rng.normal(0.0, math.sqrt(temperature / mass), size=(n, 2))
    if n > 1:
        v -= v.mean(axis=0)
        ke = 0.5 * mass * float((v * v).sum())
        v *= math.sqrt((n - 1) * temperature / ke)
    return v


def lj_initial_state(n: int, box, temperature: float, seed: int, dmin: float = 0.9,
                     mass: float = 1.0, quantum: float | None = None):
    """(x, v): (n, 2) FP64 positions in (0, L] and velocities for the LJ gas.

    ``quantum`` (a power of two, e.g. 2**-20) rounds positions to its multiples
    so that they are exactly representable as integer cell origin + binary32
    offset: both sides of a force comparison then see identical positions.
    """
    L = (float(box), float(box)) if np.isscalar(box) else (float(box[0]), float(box[1]))
    x = _nonoverlap(n, L, dmin, seed)
    if quantum is not None:
        x = np.round(x / quantum) * quantum
        for a in (0, 1):
            x[:, a] = np.where(x[:, a] <= 0, L[a], x[:, a])
    v = maxwell_velocities(n, temperature, np.random.default_rng(seed), mass)
    return x, v


def idealgas_state(n: int, box: float, temperature: float, seed: int):
    """(pos, vel) binary32 (n, 2): uniform positions in (0, L], Maxwell velocities."""
    rng = np.random.default_rng(seed)
    pos = _uniform_open_closed(rng, (n, 2), float(box)).astype(np.float32)
    # binary32 rounding may land exactly on 0 only if L*u underflows; it cannot
    # for L >= 1, but clamp defensively into (0, L].
    pos[pos <= 0] = np.float32(box)
    vel = rng.normal(0.0, math.sqrt(temperature), size=(n, 2)).astype(np.float32)
    return pos, vel


def dyadic_positions(n: int, box: float, seed: int, bits: int = 16,
                     boundary_frac: float = 0.05) -> np.ndarray:
    """(n, 2) FP64 positions in (0, L] that are multiples of 2^-bits.

    A fraction ``boundary_frac`` of coordinates is an exact integer (a base
    cell boundary).  Exactly representable as integer + binary32 offset for
    L <= 2^(24 - bits).
    """
    rng = np.random.default_rng(seed)
    scale = 1 << bits
    k = rng.integers(1, int(box) * scale + 1, size=(n, 2))   # (0, L] in units of 2^-bits
    x = k.astype(np.float64) / scale
    on_edge = rng.random((n, 2)) < boundary_frac
    x[on_edge] = rng.integers(1, int(box) + 1, size=int(on_edge.sum())).astype(np.float64)
    return x


def displaced(x: np.ndarray, box: float, seed: int, scale: float, bits: int = 16,
              boundary_frac: float = 0.05) -> np.ndarray:
    """Second snapshot: x plus a Gaussian step of std ``scale``, kept dyadic, in (0, L]."""
    rng = np.random.default_rng(seed)
    s = 1 << bits
    step = np.round(rng.normal(0.0, scale, size=x.shape) * s) / s
    y = np.mod(x + step, box)
    on_edge = rng.random(x.shape) < boundary_frac
    y[on_edge] = np.ceil(y[on_edge])
    y[y <= 0] = box
    return y


@dataclass
class LJConfig:
    """A Lennard-Jones MD + MDLG workload (units eps = sigma = m = 1)."""
    name: str
    n: int
    rho: float
    temperature: float
    dx: float = 4.0
    dt: float = 0.005
    rc: float = 2.5
    lags: tuple = (50,)
    vmax: int = 3
    steps: int = 2000
    box: float = field(default=0.0)

    def __post_init__(self):
        if not self.box:
            self.box = box_for(self.n, self.rho, self.dx)


# Small LJ system (the oracle finishes it in seconds): N = 1024, L = 64, dx = 4.
SMALL_LJ = LJConfig("lj2d_n1024_L64", n=1024, rho=0.25, temperature=1.0, dx=4.0,
                    lags=(50,), steps=2000, box=64.0)
# Production LJ gas: N = 4 194 304 at rho = 0.3, T = 1 (L rounded up to 3740).
PRODUCTION_LJ = LJConfig("lj2d_n4194304_rho0.3_T1", n=4_194_304, rho=0.3, temperature=1.0,
                         dx=4.0, lags=(10, 20, 50, 100, 200), steps=10_000)
# Dense production case: rho = 0.6, T = 0.8 (L rounded up to 2644).
PRODUCTION_LJ_DENSE = LJConfig("lj2d_n4194304_rho0.6_T0.8", n=4_194_304, rho=0.6,
                               temperature=0.8, dx=4.0, lags=(10, 20, 50, 100, 200),
                               steps=10_000)
# The paper's own state point (hot dilute gas): N = 100 000 in L = 1000 sigma
# (packing fraction 0.0785), T = 50, dt = 1e-4 tau, 3e6 steps of which the first
# 1e6 are discarded.  dx = 10 sigma here (the paper sweeps dx).
PAPER_STATE_POINT = LJConfig("lj2d_n100000_L1000_T50", n=100_000, rho=0.1, temperature=50.0,
                             dx=10.0, dt=1e-4, lags=(100, 300, 1000, 3000, 7000, 10000, 20000,
                                                     50000),
                             vmax=7, steps=3_000_000, box=1000.0)
# Ideal gas: N = 2^22 in L = 2048, all (dx, dt) in {1,2,4} x {0.5,1,2}.
IDEALGAS_N = 1 << 22
IDEALGAS_BOX = 2048.0
IDEALGAS_COMBOS = tuple((dx, dt) for dx in (1.0, 2.0, 4.0) for dt in (0.5, 1.0, 2.0))


def batch_recipe(nsys: int = 256, seed: int = 4, n_lo: int = 1000, n_hi: int = 65536,
                 rho_lo: float = 0.1, rho_hi: float = 0.6, dx: float = 4.0):
    """Replica ensemble: N log-uniform in [n_lo, n_hi], rho uniform in [rho_lo, rho_hi].

    Returns (ns, boxes, seeds); each box is sqrt(N / rho) rounded up to a multiple of dx.
    """
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), nsys)).astype(np.int64)
    rhos = rng.uniform(rho_lo, rho_hi, nsys)
    boxes = np.array([[box_for(int(n), float(r), dx)] * 2 for n, r in zip(ns, rhos)])
    seeds = 1000 + np.arange(nsys)
    return ns, boxes, seeds


def batch_states(ns, boxes, seeds, temperature: float = 1.0):
    """Concatenated initial states of a replica ensemble."""
    xs, vs = [], []
    for n, b, sd in zip(ns, boxes, seeds):
        x, v = lj_initial_state(int(n), float(b[0]), temperature, int(sd))
        xs.append(x)
        vs.append(v)
    return np.concatenate(xs), np.concatenate(vs)
