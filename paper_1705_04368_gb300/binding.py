"""Thin ctypes binding of libmdlg (include/mdlg.h).

Argument marshalling only: every step of the MD + MDLG path runs in the CUDA
kernels behind the C ABI.  PyTorch supplies device memory (through the
allocator callback) and streams.  There is no CPU fallback: if the library
cannot be built or loaded, the import of the first entry point raises.
"""
from __future__ import annotations

import ctypes
import re
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

from . import _build

MAX_LAGS = 8
MAX_VMAX = 15
MAX_COMBOS = 16
STATIC_MAX_N = 65536      # mdlg_forces_static particle limit (MDLG_STATIC_MAX_N)
POT_NONE = 0
POT_LJ_TS = 1
POT_LJ_SF = 2
SITES_FIELD = 1
SITES_ACCUM = 2
SITES_XI = 4

ERRORS = {0: "MDLG_OK", -1: "MDLG_EINVAL", -2: "MDLG_ENOMEM", -3: "MDLG_ECUDA",
          -4: "MDLG_EOVERFLOW", -5: "MDLG_ENONFINITE", -6: "MDLG_ETIMEOUT", -7: "MDLG_ENOTIMPL"}


class MdlgError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({lib().mdlg_strerror(code).decode()})")


class _Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int64), ("box", ctypes.c_double * 2),
                ("potential", ctypes.c_int32), ("eps", ctypes.c_double),
                ("sigma", ctypes.c_double), ("mass", ctypes.c_double),
                ("rcut", ctypes.c_double), ("dt", ctypes.c_double), ("grid", ctypes.c_double),
                ("skin", ctypes.c_double), ("sort_every", ctypes.c_int32),
                ("dx", ctypes.c_double), ("nlags", ctypes.c_int32),
                ("lag_steps", ctypes.c_int32 * MAX_LAGS), ("vmax", ctypes.c_int32),
                ("site_mode", ctypes.c_int32), ("stats_every", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("lattice_u", ctypes.c_double * 2),
                ("msd", ctypes.c_int32), ("vacf", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("stats_step", ctypes.c_int64),
                ("kinetic", ctypes.c_double), ("potential", ctypes.c_double),
                ("virial", ctypes.c_double), ("momentum", ctypes.c_double * 2),
                ("temperature", ctypes.c_double), ("pressure", ctypes.c_double),
                ("intervals", ctypes.c_int64 * MAX_LAGS), ("status", ctypes.c_int32),
                ("msd", (ctypes.c_double * 2) * MAX_LAGS), ("lattice_u", ctypes.c_double * 2),
                ("stale_steps", ctypes.c_int64), ("sort_every", ctypes.c_int32),
                ("vacf", (ctypes.c_double * 2) * MAX_LAGS)]


class _Lattice(ctypes.Structure):
    _fields_ = [("base", ctypes.c_int32 * 2), ("ratio", ctypes.c_int32), ("vmax", ctypes.c_int32)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()

# Every function the header declares, with its ctypes signature.
_P = ctypes.c_void_p
_SIGNATURES = {
    "mdlg_create": (ctypes.c_int, [ctypes.POINTER(_Params), _P, _P, ctypes.POINTER(_Allocator), _P,
                                   ctypes.POINTER(_P)]),
    "mdlg_create_batch": (ctypes.c_int, [ctypes.POINTER(_Params), ctypes.c_int32, _P, _P, _P, _P,
                                         ctypes.POINTER(_Allocator), _P, ctypes.POINTER(_P)]),
    "mdlg_stats_system": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_Stats), _P, _P]),
    "mdlg_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "mdlg_stats": (ctypes.c_int, [_P, ctypes.POINTER(_Stats), _P, _P]),
    "mdlg_get_state": (ctypes.c_int, [_P, _P, _P, _P]),
    "mdlg_get_sites": (ctypes.c_int, [_P, _P, _P]),
    "mdlg_get_collision": (ctypes.c_int, [_P, _P, _P, _P]),
    "mdlg_collision": (ctypes.c_int, [ctypes.POINTER(_Lattice), _P, _P, _P, _P, _P, _P]),
    "mdlg_reset_counts": (ctypes.c_int, [_P]),
    "mdlg_adjoint": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, _P, _P,
                                    _P, _P, _P, _P, _P]),
    "mdlg_profile": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "mdlg_checkpoint_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "mdlg_save": (ctypes.c_int, [_P, _P, ctypes.c_uint64]),
    "mdlg_load": (ctypes.c_int, [_P, _P, ctypes.c_uint64]),
    "mdlg_destroy": (None, [_P]),
    "mdlg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mdlg_bin": (ctypes.c_int, [ctypes.POINTER(_Lattice), ctypes.c_int64, _P, _P, _P, _P, _P, _P]),
    "mdlg_idealgas_bin": (ctypes.c_int, [ctypes.c_int64, _P, _P, ctypes.c_int32, _P, _P, _P,
                                         ctypes.c_int32, _P, _P]),
    "mdlg_forces_static": (ctypes.c_int, [ctypes.POINTER(_Params), _P, _P, _P, _P, _P, _P]),
    "mdlg_probe_fma": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P,
                                      ctypes.POINTER(ctypes.c_double), _P]),
    "mdlg_probe_copy": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
}


def lib():
    """Load (building if needed) libmdlg.so; raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            h = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _lib = h
    return _lib


def header_functions(path: str) -> list[str]:
    """Names of the functions declared in a C header (for export checks)."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mdlg_\w+)\s*\(", text,
                                 flags=re.M)))


def _check(rc: int, where: str):
    if rc != 0:
        raise MdlgError(rc, where)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, handed to the library."""

    def __init__(self, device: int, stream: int):
        import torch
        self._torch = torch
        self.device = device
        self.stream = stream

        def _alloc(nbytes, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
            except Exception:
                return None

        def _free(ptr, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.c_alloc = _ALLOC_FN(_alloc)
        self.c_free = _FREE_FN(_free)
        self.struct = _Allocator(self.c_alloc, self.c_free, None)


@dataclass
class Params:
    """Parameters of mdlg_create (see include/mdlg.h, mdlg_params)."""
    n: int
    box: float | tuple
    dx: float
    dt: float = 0.005
    lag_steps: Sequence[int] = (50,)
    potential: int = POT_LJ_TS
    eps: float = 1.0
    sigma: float = 1.0
    mass: float = 1.0
    rcut: float = 2.5
    grid: float = 0.5
    skin: float = 0.5
    sort_every: int = 0
    vmax: int = 3
    site_mode: int = 0
    stats_every: int = 0
    use_graphs: bool = False
    lattice_u: tuple = (0.0, 0.0)
    msd: bool = False
    vacf: bool = False

    def to_c(self) -> _Params:
        p = _Params()
        p.dim = 2
        p.n = int(self.n)
        box = (self.box, self.box) if np.isscalar(self.box) else self.box
        p.box[0], p.box[1] = float(box[0]), float(box[1])
        p.potential = int(self.potential)
        p.eps, p.sigma, p.mass, p.rcut = float(self.eps), float(self.sigma), float(self.mass), float(self.rcut)
        p.dt, p.grid, p.skin = float(self.dt), float(self.grid), float(self.skin)
        p.sort_every = int(self.sort_every)
        p.dx = float(self.dx)
        lags = list(self.lag_steps)
        if not 1 <= len(lags) <= MAX_LAGS:
            raise ValueError("between 1 and 8 lags")
        p.nlags = len(lags)
        for i, l in enumerate(lags):
            p.lag_steps[i] = int(l)
        p.vmax = int(self.vmax)
        p.site_mode = int(self.site_mode)
        p.stats_every = int(self.stats_every)
        p.use_graphs = int(bool(self.use_graphs))
        p.lattice_u[0], p.lattice_u[1] = float(self.lattice_u[0]), float(self.lattice_u[1])
        p.msd = int(bool(self.msd))
        p.vacf = int(bool(self.vacf))
        return p

    @property
    def q1(self) -> int:
        return (2 * self.vmax + 1) ** 2 + 1

    @property
    def lattice_cells(self) -> tuple:
        box = (self.box, self.box) if np.isscalar(self.box) else self.box
        return (int(round(box[0] / self.dx)), int(round(box[1] / self.dx)))


class Simulation:
    """One MD + MDLG context (mdlg_create ... mdlg_destroy)."""

    def __init__(self, params: Params, x0: np.ndarray, v0: np.ndarray, stream=None,
                 device: int = 0, torch_memory: bool = True):
        self.params = params
        self._lib = lib()
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        v0 = np.ascontiguousarray(v0, dtype=np.float64)
        if x0.shape != (params.n, 2) or v0.shape != (params.n, 2):
            raise ValueError("x0 and v0 must be (n, 2)")
        self._stream = _stream_handle(stream)
        self._alloc = _TorchAllocator(device, self._stream) if torch_memory else None
        self._cparams = params.to_c()
        h = ctypes.c_void_p()
        rc = self._lib.mdlg_create(ctypes.byref(self._cparams), x0.ctypes.data, v0.ctypes.data,
                                   ctypes.byref(self._alloc.struct) if self._alloc else None,
                                   self._stream, ctypes.byref(h))
        _check(rc, "mdlg_create")
        self._h = h

    def step(self, nsteps: int):
        _check(self._lib.mdlg_step(self._h, int(nsteps)), "mdlg_step")

    def stats(self):
        """(dict of FP64 observables, counts (nlags, Q+1) uint64, f_i (nlags, Q+1))."""
        out = _Stats()
        nl, q1 = len(self.params.lag_steps), self.params.q1
        counts = np.zeros((nl, q1), np.uint64)
        fi = np.zeros((nl, q1), np.float64)
        _check(self._lib.mdlg_stats(self._h, ctypes.byref(out), counts.ctypes.data, fi.ctypes.data),
               "mdlg_stats")
        d = {k: getattr(out, k) for k in ("step", "stats_step", "kinetic", "potential", "virial",
                                          "temperature", "pressure", "status", "stale_steps",
                                          "sort_every")}
        d["momentum"] = (out.momentum[0], out.momentum[1])
        d["intervals"] = [out.intervals[i] for i in range(nl)]
        d["msd"] = [(out.msd[i][0], out.msd[i][1]) for i in range(nl)]
        d["vacf"] = [(out.vacf[i][0], out.vacf[i][1]) for i in range(nl)]
        d["lattice_u"] = (out.lattice_u[0], out.lattice_u[1])
        return d, counts, fi

    def get_state(self, want_force: bool = False):
        n = self.params.n
        x = np.empty((n, 2))
        v = np.empty((n, 2))
        f = np.empty((n, 2)) if want_force else None
        _check(self._lib.mdlg_get_state(self._h, x.ctypes.data, v.ctypes.data,
                                        f.ctypes.data if f is not None else None), "mdlg_get_state")
        return (x, v, f) if want_force else (x, v)

    def get_sites(self):
        cx, cy = self.params.lattice_cells
        sc = np.zeros((cy * cx, self.params.q1), np.uint32)
        nc = np.zeros(cy * cx, np.uint32)
        _check(self._lib.mdlg_get_sites(self._h, sc.ctypes.data, nc.ctypes.data), "mdlg_get_sites")
        return sc, nc

    def get_collision(self):
        """Xi_i(x) (sites, Q) int32 of the last two lag-0 intervals, with the
        per-site mass (sites,) and momentum (sites, 2) sums (mdlg_get_collision)."""
        cx, cy = self.params.lattice_cells
        q = self.params.q1 - 1
        xi = np.zeros((cy * cx, q), np.int32)
        dm = np.zeros(cy * cx, np.int32)
        dj = np.zeros((cy * cx, 2), np.int32)
        _check(self._lib.mdlg_get_collision(self._h, xi.ctypes.data, dm.ctypes.data, dj.ctypes.data),
               "mdlg_get_collision")
        return xi, dm, dj

    def adjoint(self, nsteps: int, ckpt_every: int, width: float, dloss=None):
        """mdlg_adjoint: advance nsteps and differentiate the soft-binned loss.

        Returns {"ftilde": (Q,), "loss": float} and, when ``dloss`` (Q weights)
        is given, "grad_eps", "grad_sigma", "grad_x0" (n, 2), "grad_v0" (n, 2).
        """
        q = (2 * self.params.vmax + 1) ** 2
        ft = np.zeros(q)
        loss = ctypes.c_double(0.0)
        out = {"ftilde": ft}
        if dloss is None:
            _check(self._lib.mdlg_adjoint(self._h, int(nsteps), int(ckpt_every), float(width),
                                          None, ft.ctypes.data, ctypes.byref(loss), None, None,
                                          None, None), "mdlg_adjoint")
        else:
            w = np.ascontiguousarray(dloss, dtype=np.float64).reshape(q)
            ge, gs = ctypes.c_double(0.0), ctypes.c_double(0.0)
            gx = np.zeros((self.params.n, 2))
            gv = np.zeros((self.params.n, 2))
            _check(self._lib.mdlg_adjoint(self._h, int(nsteps), int(ckpt_every), float(width),
                                          w.ctypes.data, ft.ctypes.data, ctypes.byref(loss),
                                          ctypes.byref(ge), ctypes.byref(gs), gx.ctypes.data,
                                          gv.ctypes.data), "mdlg_adjoint")
            out.update(grad_eps=ge.value, grad_sigma=gs.value, grad_x0=gx, grad_v0=gv)
        out["loss"] = loss.value
        return out

    PROF_KINDS = ("step", "sort", "bin", "sync")

    def profile(self, enable: bool):
        """Start (True) or stop (False) per-kernel event timing; stop returns
        {kind: (milliseconds, launches)}."""
        ms = np.zeros(4)
        ln = np.zeros(4, np.int64)
        _check(self._lib.mdlg_profile(self._h, int(enable), ms.ctypes.data, ln.ctypes.data),
               "mdlg_profile")
        if enable:
            return None
        return {k: (float(ms[i]), int(ln[i])) for i, k in enumerate(self.PROF_KINDS)}

    def reset_counts(self):
        _check(self._lib.mdlg_reset_counts(self._h), "mdlg_reset_counts")

    def save(self) -> bytes:
        """mdlg_save: the complete run state as bytes (see mdlg_checkpoint_size)."""
        size = ctypes.c_uint64()
        _check(self._lib.mdlg_checkpoint_size(self._h, ctypes.byref(size)), "mdlg_checkpoint_size")
        buf = ctypes.create_string_buffer(size.value)
        _check(self._lib.mdlg_save(self._h, buf, size.value), "mdlg_save")
        return buf.raw

    def load(self, data: bytes):
        """mdlg_load: continue from a checkpoint of a context with the same parameters."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        _check(self._lib.mdlg_load(self._h, buf, len(data)), "mdlg_load")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mdlg_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSimulation(Simulation):
    """Several independent systems advanced together (mdlg_create_batch).

    ``ns`` particle counts, ``boxes`` (nsys, 2) box sides, ``x0``/``v0`` the
    concatenated (sum ns, 2) initial states.  ``params.n``/``params.box`` are
    ignored.  ``stats()`` adds all systems; ``stats_system(k)`` reports one.
    """

    def __init__(self, params: Params, ns, boxes, x0, v0, stream=None, device: int = 0,
                 torch_memory: bool = True):
        self.ns = np.ascontiguousarray(ns, dtype=np.int64)
        self.boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 2)
        total = int(self.ns.sum())
        self.params = Params(**{**params.__dict__, "n": total})
        self._lib = lib()
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        v0 = np.ascontiguousarray(v0, dtype=np.float64)
        if x0.shape != (total, 2) or v0.shape != (total, 2):
            raise ValueError("x0 and v0 must be (sum ns, 2)")
        self._stream = _stream_handle(stream)
        self._alloc = _TorchAllocator(device, self._stream) if torch_memory else None
        self._cparams = self.params.to_c()
        h = ctypes.c_void_p()
        rc = self._lib.mdlg_create_batch(ctypes.byref(self._cparams), len(self.ns),
                                         self.ns.ctypes.data, self.boxes.ctypes.data,
                                         x0.ctypes.data, v0.ctypes.data,
                                         ctypes.byref(self._alloc.struct) if self._alloc else None,
                                         self._stream, ctypes.byref(h))
        _check(rc, "mdlg_create_batch")
        self._h = h

    def stats_system(self, k: int):
        out = _Stats()
        nl, q1 = len(self.params.lag_steps), self.params.q1
        counts = np.zeros((nl, q1), np.uint64)
        fi = np.zeros((nl, q1), np.float64)
        _check(self._lib.mdlg_stats_system(self._h, int(k), ctypes.byref(out), counts.ctypes.data,
                                           fi.ctypes.data), "mdlg_stats_system")
        d = {k2: getattr(out, k2) for k2 in ("step", "stats_step", "kinetic", "potential",
                                             "virial", "temperature", "pressure", "status")}
        d["momentum"] = (out.momentum[0], out.momentum[1])
        d["intervals"] = [out.intervals[i] for i in range(nl)]
        return d, counts, fi


def bin_snapshots(base: Sequence[int], ratio: int, vmax: int, idx_prev, idx_cur, counts,
                  ncell=None, field=None, stream=None):
    """mdlg_bin: tensors on the GPU; idx_* int32 (n, 2); counts int64 (Q+1,) (added to)."""
    lat = _Lattice()
    lat.base[0], lat.base[1] = int(base[0]), int(base[1])
    lat.ratio, lat.vmax = int(ratio), int(vmax)
    n = 0 if idx_cur is None else int(idx_cur.shape[0])
    _check(lib().mdlg_bin(ctypes.byref(lat), n, _ptr(idx_prev), _ptr(idx_cur), _ptr(counts),
                          _ptr(ncell), _ptr(field), _stream_handle(stream)), "mdlg_bin")


def idealgas_bin(pos, vel, combos: Sequence[tuple], vmax: int, counts, stream=None, us=None):
    """mdlg_idealgas_bin: pos/vel float32 (n, 2) on the GPU; counts int64 (ncombo, Q+1);
    us: optional (ncombo, 2) lattice drifts."""
    dxs = np.ascontiguousarray([c[0] for c in combos], dtype=np.float32)
    dts = np.ascontiguousarray([c[1] for c in combos], dtype=np.float32)
    u = None
    if us is not None:
        u = np.ascontiguousarray(us, dtype=np.float32).reshape(len(combos), 2)
    n = int(pos.shape[0])
    _check(lib().mdlg_idealgas_bin(n, _ptr(pos), _ptr(vel), len(combos), dxs.ctypes.data,
                                   dts.ctypes.data, u.ctypes.data if u is not None else None,
                                   int(vmax), _ptr(counts), _stream_handle(stream)),
           "mdlg_idealgas_bin")


def collision(lattice_cells: Sequence[int], vmax: int, field_prev, field_cur, xi=None, dmass=None,
              dmom=None, stream=None):
    """mdlg_collision: fields uint32/int32 (sites, Q+1) on the GPU; outputs int32
    xi (sites, Q), dmass (sites,), dmom (sites, 2), each optional."""
    lat = _Lattice()
    lat.base[0], lat.base[1] = int(lattice_cells[0]), int(lattice_cells[1])
    lat.ratio, lat.vmax = 1, int(vmax)
    _check(lib().mdlg_collision(ctypes.byref(lat), _ptr(field_prev), _ptr(field_cur), _ptr(xi),
                                _ptr(dmass), _ptr(dmom), _stream_handle(stream)), "mdlg_collision")
