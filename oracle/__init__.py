"""FP64 CPU oracle for the MDLG hot path (arXiv:1705.04368).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library in ``paper_1705_04368_gb300``; neither
imports the other.

Contents
  mdlg_oracle.c  plain C, FP64: direct O(N^2) and linked-cell Lennard-Jones
                 forces, velocity-Verlet, MDLG occupation numbers (Eq. MDni),
                 the binary32 ideal-gas stream-and-bin, FP64 reductions, the
                 moving lattice of Sec. IV, the collision operator Xi_i (Eq.
                 Xi), the mean-square displacement and the velocity
                 correlation (Sec. IV-A).
  closed_form.py the Gaussian/wedge equilibrium of Eq. fialpha.

Parity status per function (what pins it, see tests/test_oracle_*.py):
  lj_forces_direct   pinned: hand-computed two-particle force and energy,
                     Newton's third law, finite-difference gradient of the
                     potential energy.
  lj_forces_cells    pinned: equal to the direct sum on random systems.
  vv                 pinned: energy drift bound, time reversal, exact free
                     flight when the potential is switched off.
  mdlg_bin           pinned: Fig. 2 worked example (tests/golden), brute-force
                     recount, partition of unity N = sum_i n_i, mass
                     conservation across intervals, boundary convention.
  stream_bin_f32     pinned: equal to mdlg_bin on the same binary32 points; its
                     totals match the closed form within sampling error.
  mdlg_bin (shifted) pinned: equal to binning the shifted, wrapped positions;
                     whole-box shifts change nothing; a gas at rest seen from
                     the moving lattice matches the closed form at mean
                     velocity u (chi-square).
  stream_bin_f32 us  pinned: equal to boosting the binary32 velocities first;
                     closed form at u (chi-square).
  collision          pinned: particle-by-particle tracking (brute force), mass
                     conservation without overflow, the Fig. 2 worked example.
  msd                pinned: exact dyadic free flight across the boundary; the
                     ballistic value T dt^2 within sampling error.
  half_velocity      pinned: equal to v_n + F(x_n) dt / 2m from the oracle's own
                     forces after a velocity-Verlet step; exact in free flight.
  vacf               pinned: free flight gives <v_a^2> exactly; the correlation
                     of the one-step velocities with themselves, times dt^2,
                     equals msd over that step.
  closed_form        pinned: numerical quadrature of the wedge integral (Eq.
                     fieqW), Monte-Carlo binning, normalisation and first
                     moment identities, the second-moment offset of Sec. VI.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdlg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_threaded = False


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle C file into a shared library with gcc (FP64, no fast-math).

    openmp: the same source built with -fopenmp (the threaded timing build of the
    benchmark's CPU baseline); the default build is serial."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _LIB_OMP_PATH if openmp else _LIB_PATH
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", *(["-fopenmp"] if openmp else []), _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return path


def use_threads(threads: int) -> int:
    """Switch this process to the threaded build with `threads` host threads (0: all
    cores); returns the thread count in use.  Call before the first oracle call."""
    global _threaded
    with _lock:
        if _lib is not None and not _threaded:
            raise RuntimeError("oracle.use_threads must come before the first oracle call")
        _threaded = True
    lib = _load()
    lib.oracle_set_threads(int(threads) if threads > 0 else (os.cpu_count() or 1))
    return int(lib.oracle_threads())


def threads() -> int:
    """Host threads the loaded oracle build uses (1 for the serial build)."""
    return int(_load().oracle_threads())


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB: an alternative build of the same source (the sanitizer test)
            lib = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build(openmp=_threaded))
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            D = ctypes.c_double
            lib.oracle_lj_forces_direct.argtypes = [I64, P, P, D, D, D, P, P, P]
            lib.oracle_lj_forces_cells.argtypes = [I64, P, P, D, D, D, P, P, P]
            lib.oracle_lj_forces_sample.argtypes = [I64, P, P, D, D, D, I64, P, P, P]
            lib.oracle_vv.argtypes = [I64, P, P, P, ctypes.c_int, P, D, D, D, D, D, I64,
                                      ctypes.c_int, P]
            lib.oracle_free_stream.argtypes = [I64, P, P, P, D, I64]
            lib.oracle_mdlg_bin.argtypes = [I64, P, P, D, P, ctypes.c_int, P, P, P, P]
            lib.oracle_stream_bin_f32.argtypes = [I64, P, P, ctypes.c_int, P, P, P, ctypes.c_int, P]
            lib.oracle_mdlg_bin_shifted.argtypes = [I64, P, P, D, P, ctypes.c_int, P, P, P, P, P, P]
            lib.oracle_collision.argtypes = [P, ctypes.c_int, P, P, P]
            lib.oracle_msd.argtypes = [I64, P, P, P, P]
            lib.oracle_half_velocity.argtypes = [I64, P, P, P, D, P]
            lib.oracle_vacf.argtypes = [I64, P, P, P]
            lib.oracle_kinetic.argtypes = [I64, P, D, P]
            lib.oracle_set_shifted_force.argtypes = [ctypes.c_int]
            lib.oracle_set_shifted_force.restype = None
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = None
            lib.oracle_threads.argtypes = []
            lib.oracle_threads.restype = ctypes.c_int
            for name in ("oracle_lj_forces_direct", "oracle_lj_forces_cells",
                         "oracle_lj_forces_sample", "oracle_vv", "oracle_free_stream",
                         "oracle_mdlg_bin", "oracle_stream_bin_f32", "oracle_kinetic",
                         "oracle_mdlg_bin_shifted", "oracle_collision", "oracle_msd",
                         "oracle_half_velocity", "oracle_vacf"):
                getattr(lib, name).restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def lj_forces(x, box, eps=1.0, sigma=1.0, rc=2.5, cells=False, shifted_force=False):
    """Lennard-Jones forces, the per-particle error scale sum_j (|F_rep,ij| + |F_att,ij|),
    potential energy and virial.

    x: (n, 2) positions.  Returns (F (n,2), fscale (n,), pe, virial).
    shifted_force: F(r) - F(rc) instead of the force truncated at rc.
    """
    lib = _load()
    lib.oracle_set_shifted_force(int(shifted_force))
    x = _f64(x)
    n = x.shape[0]
    L = _f64(box)
    f = np.zeros((n, 2))
    fs = np.zeros(n)
    out = np.zeros(2)
    fn = lib.oracle_lj_forces_cells if cells else lib.oracle_lj_forces_direct
    fn(n, _p(x), _p(L), eps, sigma, rc, _p(f), _p(fs), _p(out))
    return f, fs, float(out[0]), float(out[1])


def lj_forces_sample(x, box, which, eps=1.0, sigma=1.0, rc=2.5, shifted_force=False):
    """Direct-sum forces for the particles listed in ``which`` only."""
    lib = _load()
    lib.oracle_set_shifted_force(int(shifted_force))
    x = _f64(x)
    w = np.ascontiguousarray(which, dtype=np.int64)
    f = np.zeros((w.size, 2))
    fs = np.zeros(w.size)
    lib.oracle_lj_forces_sample(x.shape[0], _p(x), _p(_f64(box)), eps, sigma, rc,
                                w.size, _p(w), _p(f), _p(fs))
    return f, fs


class VV:
    """Velocity-Verlet state (x, v, F) advanced by the oracle (FP64)."""

    def __init__(self, x, v, box, dt, mass=1.0, eps=1.0, sigma=1.0, rc=2.5, cells=None,
                 shifted_force=False):
        self.x = _f64(x).copy()
        self.v = _f64(v).copy()
        self.f = np.zeros_like(self.x)
        self.box = _f64(box)
        self.dt, self.mass, self.eps, self.sigma, self.rc = dt, mass, eps, sigma, rc
        n = self.x.shape[0]
        self.cells = (n > 2048) if cells is None else cells
        self.shifted_force = bool(shifted_force)
        self.have_force = 0
        self.pe = 0.0
        self.virial = 0.0
        self.steps = 0

    def run(self, nsteps: int):
        lib = _load()
        lib.oracle_set_shifted_force(int(self.shifted_force))
        out = np.zeros(2)
        lib.oracle_vv(self.x.shape[0], _p(self.x), _p(self.v), _p(self.f), self.have_force,
                      _p(self.box), self.mass, self.eps, self.sigma, self.rc, self.dt,
                      int(nsteps), int(self.cells), _p(out))
        self.have_force = 1
        self.pe, self.virial = float(out[0]), float(out[1])
        self.steps += int(nsteps)
        return self

    def kinetic(self):
        """[kinetic energy, momentum_x, momentum_y] in FP64."""
        out = np.zeros(3)
        _load().oracle_kinetic(self.x.shape[0], _p(self.v), self.mass, _p(out))
        return out

    def energy(self):
        """Total energy KE + PE (the force routine's PE of the current state)."""
        if not self.have_force:
            _, _, self.pe, self.virial = lj_forces(self.x, self.box, self.eps, self.sigma,
                                                   self.rc, self.cells, self.shifted_force)
        return float(self.kinetic()[0]) + self.pe


def free_stream(x, v, box, dt, nsteps=1):
    lib = _load()
    x = _f64(x).copy()
    lib.oracle_free_stream(x.shape[0], _p(x), _p(_f64(v)), _p(_f64(box)), dt, int(nsteps))
    return x


def mdlg_bin(xprev, xcur, dx, cells, vmax, field=False, counts=None, ncell=None, fld=None,
             shift_prev=None, shift_cur=None):
    """Occupation numbers of Eq. MDni for one pair of snapshots.

    Returns (counts (Q+1,) uint64, ncell (Cy*Cx,) uint32, field (Cy*Cx, Q+1) uint32
    or None, vsum (2,) int64).  Passing arrays accumulates into them.
    """
    lib = _load()
    xp, xc = _f64(xprev), _f64(xcur)
    C = np.ascontiguousarray(cells, dtype=np.int64)
    q1 = (2 * vmax + 1) ** 2 + 1
    counts = np.zeros(q1, np.uint64) if counts is None else counts
    ncell = np.zeros(int(C[0] * C[1]), np.uint32) if ncell is None else ncell
    if field and fld is None:
        fld = np.zeros((int(C[0] * C[1]), q1), np.uint32)
    vsum = np.zeros(2, np.int64)
    sp = _f64(shift_prev) if shift_prev is not None else None
    sc = _f64(shift_cur) if shift_cur is not None else None
    lib.oracle_mdlg_bin_shifted(xp.shape[0], _p(xp), _p(xc), float(dx), _p(C), int(vmax),
                                _p(sp) if sp is not None else None,
                                _p(sc) if sc is not None else None,
                                _p(counts), _p(ncell), _p(fld) if fld is not None else None,
                                _p(vsum))
    return counts, ncell, fld, vsum


def stream_bin_f32(pos, vel, dxs, dts, vmax, us=None):
    """Ideal-gas stream + bin in binary32 decisions; returns (ncombo, Q+1) uint64.

    us: optional (ncombo, 2) lattice velocities U (velocities boosted by U)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    vel = np.ascontiguousarray(vel, dtype=np.float32)
    dxs = np.ascontiguousarray(dxs, dtype=np.float32)
    dts = np.ascontiguousarray(dts, dtype=np.float32)
    q1 = (2 * vmax + 1) ** 2 + 1
    counts = np.zeros((dxs.size, q1), np.uint64)
    u = np.ascontiguousarray(us, dtype=np.float32).reshape(-1, 2) if us is not None else None
    lib.oracle_stream_bin_f32(pos.shape[0], _p(pos), _p(vel), dxs.size, _p(dxs), _p(dts),
                              _p(u) if u is not None else None, int(vmax), _p(counts))
    return counts


def collision(cells, vmax, field_prev, field_cur):
    """Xi_i(x) = n_i(x + v_i, t+dt) - n_i(x, t) (Eq. Xi); (C_y*C_x, Q) int64."""
    lib = _load()
    C = np.ascontiguousarray(cells, dtype=np.int64)
    q = (2 * vmax + 1) ** 2
    fp = np.ascontiguousarray(field_prev, dtype=np.uint32)
    fc = np.ascontiguousarray(field_cur, dtype=np.uint32)
    xi = np.zeros((int(C[0] * C[1]), q), np.int64)
    lib.oracle_collision(_p(C), int(vmax), _p(fp), _p(fc), _p(xi))
    return xi


def msd(xprev, xcur, box):
    """<dx_a^2> per axis between two snapshots (minimum image)."""
    lib = _load()
    xp, xc = _f64(xprev), _f64(xcur)
    out = np.zeros(2)
    lib.oracle_msd(xp.shape[0], _p(xp), _p(xc), _p(_f64(box)), _p(out))
    return out


def half_velocity(xprev, xcur, box, dt):
    """Leapfrog half-step velocity of the step from xprev to xcur: the
    minimum-image displacement over dt."""
    xp, xc = _f64(xprev), _f64(xcur)
    out = np.zeros_like(xc)
    _load().oracle_half_velocity(xp.shape[0], _p(xp), _p(xc), _p(_f64(box)), float(dt), _p(out))
    return out


def initial_half_velocity(x0, v0, box, dt, mass=1.0, eps=1.0, sigma=1.0, rc=2.5,
                          shifted_force=False):
    """v_{-1/2} = v_0 - F(x_0) dt / (2m): the half-step velocity before the first step."""
    f, _, _, _ = lj_forces(x0, box, eps, sigma, rc, cells=_f64(x0).shape[0] > 2048,
                           shifted_force=shifted_force)
    return _f64(v0) - f * (dt / (2.0 * mass))


def vacf(vprev, vcur):
    """Per axis, the mean over particles of v_a(now) v_a(before) (Sec. IV-A)."""
    vp, vc = _f64(vprev), _f64(vcur)
    out = np.zeros(2)
    _load().oracle_vacf(vp.shape[0], _p(vp), _p(vc), _p(out))
    return out


def velocity_table(vmax):
    """(Q, 2) integer lattice velocities in the index order i = (vy+V)(2V+1)+(vx+V)."""
    r = np.arange(-vmax, vmax + 1)
    vy, vx = np.meshgrid(r, r, indexing="ij")
    return np.stack([vx.ravel(), vy.ravel()], axis=1)
