"""Host-side checks of the C ABI: the library builds for sm_103a, loads without a
GPU, exports every function include/mdlg.h declares, and validates arguments
before touching the device."""
import ctypes
import os

import numpy as np
import pytest

import paper_1705_04368_gb300 as m
from paper_1705_04368_gb300 import binding as b

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "mdlg.h")


def test_exports_every_declared_function():
    names = m.header_functions(HEADER)
    assert {"mdlg_create", "mdlg_step", "mdlg_bin", "mdlg_stats", "mdlg_adjoint",
            "mdlg_get_state", "mdlg_destroy", "mdlg_strerror",
            "mdlg_idealgas_bin"} <= set(names)
    h = ctypes.CDLL(m.binding._build.build())
    for name in names:
        assert hasattr(h, name), name
    assert set(b._SIGNATURES) == set(names)


def test_strerror_names_every_code():
    L = m.lib()
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert L.mdlg_strerror(code) != b"unknown error"
    assert L.mdlg_strerror(-99) == b"unknown error"


def _params(**kw):
    raw = {k: kw.pop(k) for k in ("msd", "vacf") if k in kw}   # set on the C struct unchecked
    base = dict(n=16, box=16.0, dx=4.0, grid=0.5, lag_steps=(5,))
    base.update(kw)
    p = m.Params(**base).to_c()
    for k, v in raw.items():
        setattr(p, k, v)
    return p


BAD = [
    dict(n=0), dict(dx=3.0, box=16.0), dict(grid=0.3), dict(dx=0.75, grid=0.5),
    dict(vmax=0), dict(vmax=16), dict(lag_steps=()), dict(lag_steps=(0,)), dict(dt=0.0),
    dict(rcut=9.0), dict(box=8.0, dx=4.0), dict(potential=7), dict(site_mode=3),
    dict(skin=-1.0), dict(sort_every=-2), dict(mass=0.0),
    dict(site_mode=4), dict(site_mode=6), dict(msd=2), dict(vacf=2),
    dict(lattice_u=(float("nan"), 0.0)),
    dict(lattice_u=(0.0, 1e9)),
]


@pytest.mark.parametrize("kw", BAD, ids=[str(k) for k in BAD])
def test_create_rejects_bad_parameters(kw):
    if kw.get("lag_steps") == ():
        p = _params()
        p.nlags = 0
    else:
        p = _params(**kw)
    x = np.full((max(p.n, 1), 2), 1.0)
    h = ctypes.c_void_p()
    rc = m.lib().mdlg_create(ctypes.byref(p), x.ctypes.data, x.ctypes.data, None, None,
                             ctypes.byref(h))
    assert rc == -1 and not h.value


def test_create_limits_particles_to_what_list_entries_hold():
    # Verlet-list entries hold slot numbers in 28 bits: with a potential, 2^28
    # particles are rejected while the parameters are checked, before any device
    # work and before the inputs are read (a one-particle buffer stands in for
    # them); 2^28 - 1 passes the check (and fails only at allocation without a
    # GPU, or is not tried with one), and without a potential 2^28 passes too
    import torch
    if torch.cuda.is_available():
        pytest.skip("the passing sizes would allocate and read a 4 GB input")
    x = np.zeros((1, 2))

    def rc_for(n, pot):
        p = _params(n=n, box=12000.0, dx=4.0, grid=0.5, potential=pot)
        h = ctypes.c_void_p()
        rc = m.lib().mdlg_create(ctypes.byref(p), x.ctypes.data, x.ctypes.data, None, None,
                                 ctypes.byref(h))
        assert not h.value
        return rc

    for pot in (m.POT_LJ_TS, m.POT_LJ_SF):
        assert rc_for(1 << 28, pot) == -1
        assert rc_for((1 << 28) - 1, pot) != -1
    assert rc_for(1 << 28, m.POT_NONE) != -1


def test_create_rejects_null_state():
    p = _params()
    h = ctypes.c_void_p()
    assert m.lib().mdlg_create(ctypes.byref(p), None, None, None, None, ctypes.byref(h)) == -1


def test_allocation_failure_is_reported_and_nothing_leaks():
    # host-side fault injection: an allocator that fails on its 5th request
    calls = {"alloc": 0, "free": 0, "live": set()}
    store = []

    def alloc(nbytes, user):
        calls["alloc"] += 1
        if calls["alloc"] == 5:
            return None
        buf = ctypes.create_string_buffer(int(nbytes) + 256)
        store.append(buf)
        p = ctypes.addressof(buf)
        calls["live"].add(p)
        return p

    def free(ptr, user):
        calls["free"] += 1
        calls["live"].discard(ptr)

    A = b._Allocator(b._ALLOC_FN(alloc), b._FREE_FN(free), None)
    p = _params()
    x = np.full((16, 2), 1.0)
    h = ctypes.c_void_p()
    rc = m.lib().mdlg_create(ctypes.byref(p), x.ctypes.data, x.ctypes.data, ctypes.byref(A), None,
                             ctypes.byref(h))
    assert rc == -2 and not h.value
    assert calls["alloc"] == 5 and calls["free"] == 4 and not calls["live"]


def test_context_free_entry_points_validate():
    L = m.lib()
    lat = b._Lattice()
    lat.base[0], lat.base[1], lat.ratio, lat.vmax = 16, 16, 3, 3    # 16 not a multiple of 3
    buf = ctypes.c_void_p(1)
    assert L.mdlg_bin(ctypes.byref(lat), 4, buf, buf, buf, None, None, None) == -1
    lat.ratio = 4
    assert L.mdlg_bin(ctypes.byref(lat), 4, buf, buf, None, None, None, None) == -1
    assert L.mdlg_bin(ctypes.byref(lat), 0, None, None, buf, None, None, None) == 0  # empty: no-op
    d = np.array([1.0], np.float32)
    assert L.mdlg_idealgas_bin(4, buf, buf, 0, d.ctypes.data, d.ctypes.data, None, 3, buf, None) == -1
    assert L.mdlg_idealgas_bin(4, buf, buf, 1, d.ctypes.data, d.ctypes.data, None, 16, buf, None) == -1
    z = np.array([0.0], np.float32)
    assert L.mdlg_idealgas_bin(4, buf, buf, 1, z.ctypes.data, d.ctypes.data, None, 3, buf, None) == -1
    assert L.mdlg_idealgas_bin(0, None, None, 1, d.ctypes.data, d.ctypes.data, None, 3, buf, None) == 0
    nan = np.array([np.nan, 0.0], np.float32)
    assert L.mdlg_idealgas_bin(4, buf, buf, 1, d.ctypes.data, d.ctypes.data, nan.ctypes.data, 3, buf,
                               None) == -1
    # collision operator: lattice and fields are checked before any launch
    assert L.mdlg_collision(ctypes.byref(lat), None, buf, buf, None, None, None) == -1
    lat.base[0] = 0
    assert L.mdlg_collision(ctypes.byref(lat), buf, buf, buf, None, None, None) == -1
    lat.base[0], lat.vmax = 16, 16
    assert L.mdlg_collision(ctypes.byref(lat), buf, buf, buf, None, None, None) == -1
    lat.vmax = 3
    assert L.mdlg_collision(ctypes.byref(lat), buf, buf, None, None, None, None) == 0  # nothing asked


def test_batch_rejects_single_system_analyses():
    # the moving lattice, displacement and velocity sums and per-site outputs are
    # single-system only
    x = np.full((32, 2), 1.0)
    ns = np.array([16, 16], np.int64)
    boxes = np.array([[16.0, 16.0], [16.0, 16.0]])
    for kw in (dict(msd=1), dict(vacf=1), dict(lattice_u=(0.5, 0.0)), dict(site_mode=1)):
        p = _params(**kw)
        h = ctypes.c_void_p()
        rc = m.lib().mdlg_create_batch(ctypes.byref(p), 2, ns.ctypes.data, boxes.ctypes.data,
                                       x.ctypes.data, x.ctypes.data, None, None, ctypes.byref(h))
        assert rc == -1 and not h.value, kw


def test_batch_rejects_slot_count_past_list_index_range():
    # list entries hold a slot index in 28 bits; systems are padded to whole
    # 128-slot chunks, so 2^28 - 64 particles in two systems take 2^28 slots
    x = np.full((1, 2), 1.0)
    ns = np.array([1 << 27, (1 << 27) - 64], np.int64)
    boxes = np.array([[16.0, 16.0], [16.0, 16.0]])
    h = ctypes.c_void_p()
    rc = m.lib().mdlg_create_batch(ctypes.byref(_params()), 2, ns.ctypes.data, boxes.ctypes.data,
                                   x.ctypes.data, x.ctypes.data, None, None, ctypes.byref(h))
    assert rc == -1 and not h.value


def test_get_collision_rejects_null_context():
    assert m.lib().mdlg_get_collision(None, None, None, None) == -1


def test_checkpoint_entry_points_validate():
    L = m.lib()
    size = ctypes.c_uint64()
    buf = ctypes.create_string_buffer(64)
    assert L.mdlg_checkpoint_size(None, ctypes.byref(size)) == -1
    assert L.mdlg_save(None, buf, 64) == -1
    assert L.mdlg_load(None, buf, 64) == -1


def test_adjoint_rejects_null_context():
    assert m.lib().mdlg_adjoint(None, 10, 10, 1.0, None, None, None, None, None, None, None) == -1


def test_probes_validate_arguments_before_launching():
    L = m.lib()
    buf = ctypes.c_void_p(16)
    assert L.mdlg_probe_fma(0, 256, 10, buf, None, None) == -1
    assert L.mdlg_probe_fma(4, 48, 10, buf, None, None) == -1      # not a multiple of 32
    assert L.mdlg_probe_fma(4, 512, 10, buf, None, None) == -1     # above 256
    assert L.mdlg_probe_fma(4, 256, 0, buf, None, None) == -1
    assert L.mdlg_probe_fma(4, 256, 10, None, None, None) == -1
    assert L.mdlg_probe_copy(buf, buf, 24, None) == -1             # not a multiple of 16
    assert L.mdlg_probe_copy(ctypes.c_void_p(8), buf, 32, None) == -1   # misaligned
    assert L.mdlg_probe_copy(buf, buf, 0, None) == 0
