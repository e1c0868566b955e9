"""GPU parity: MDLG occupation numbers (Eq. MDni) and the ideal-gas pass are
bit-exact against the oracle on identical snapshots."""
import math

import numpy as np
import pytest

import mdlg_inputs as mi
import oracle
from oracle import closed_form as cf
import paper_1705_04368_gb300 as m

pytestmark = pytest.mark.gpu


def _base_index(x, g):
    # storage convention of the library's snapshots: base cell b with b g < x <= (b+1) g
    return (np.ceil(x / g) - 1).astype(np.int32)


def _run_bin(cuda, xp, xc, L, dx, g, vmax, with_sites=True):
    import torch
    q1 = (2 * vmax + 1) ** 2 + 1
    C = (int(L / dx), int(L / dx))
    ip = torch.from_numpy(_base_index(xp, g)).to(cuda)
    ic = torch.from_numpy(_base_index(xc, g)).to(cuda)
    counts = torch.zeros(q1, dtype=torch.int64, device=cuda)
    ncell = torch.zeros(C[0] * C[1], dtype=torch.int32, device=cuda) if with_sites else None
    field = torch.zeros(C[0] * C[1] * q1, dtype=torch.int32, device=cuda) if with_sites else None
    base = (int(L / g), int(L / g))
    m.bin_snapshots(base, int(round(dx / g)), vmax, ip, ic, counts, ncell, field)
    torch.cuda.synchronize()
    out = counts.cpu().numpy().view(np.uint64)
    if with_sites:
        return out, ncell.cpu().numpy().view(np.uint32), field.cpu().numpy().view(np.uint32).reshape(-1, q1)
    return out, None, None


CASES = [
    # n, L, dx, g, vmax, step scale, boundary fraction
    (5000, 64.0, 4.0, 0.5, 3, 3.0, 0.05),      # several blocks, ragged tail
    (777, 48.0, 2.0, 1.0, 3, 2.0, 0.5),        # half the coordinates on cell boundaries
    (1, 16.0, 4.0, 0.5, 3, 1.0, 0.0),
    (20000, 96.0, 3.0, 1.0, 3, 4.0, 0.1),      # ratio 3: non power of two
    (20000, 64.0, 1.0, 0.25, 1, 1.5, 0.1),     # narrow window, overflow-heavy
    (20000, 64.0, 2.0, 0.5, 15, 9.0, 0.1),     # widest window
    (30000, 40.0, 4.0, 1.0, 3, 30.0, 0.05),    # steps comparable to the box: wrap-around
]


@pytest.mark.parametrize("case", CASES, ids=[f"n{c[0]}_L{c[1]}_dx{c[2]}_g{c[3]}_V{c[4]}" for c in CASES])
def test_bin_snapshots_bit_exact(cuda, case):
    n, L, dx, g, vmax, scale, bf = case
    xp = mi.dyadic_positions(n, L, seed=n, bits=12, boundary_frac=bf)
    xc = mi.displaced(xp, L, seed=n + 1, scale=scale, bits=12, boundary_frac=bf)
    got_c, got_n, got_f = _run_bin(cuda, xp, xc, L, dx, g, vmax)
    ref_c, ref_n, ref_f, _ = oracle.mdlg_bin(xp, xc, dx, (int(L / dx),) * 2, vmax, field=True)
    assert np.array_equal(got_c, ref_c)
    assert np.array_equal(got_n, ref_n)
    assert np.array_equal(got_f, ref_f)


def test_bin_snapshots_accumulates_and_empty(cuda):
    import torch
    xp = mi.dyadic_positions(3000, 32.0, seed=1, bits=12)
    xc = mi.displaced(xp, 32.0, seed=2, scale=2.0, bits=12)
    ip = torch.from_numpy(_base_index(xp, 0.5)).to(cuda)
    ic = torch.from_numpy(_base_index(xc, 0.5)).to(cuda)
    counts = torch.zeros(50, dtype=torch.int64, device=cuda)
    m.bin_snapshots((64, 64), 8, 3, ip, ic, counts)
    m.bin_snapshots((64, 64), 8, 3, ip, ic, counts)
    m.bin_snapshots((64, 64), 8, 3, ip[:0], ic[:0], counts)
    torch.cuda.synchronize()
    ref, _, _, _ = oracle.mdlg_bin(xp, xc, 4.0, (8, 8), 3)
    assert np.array_equal(counts.cpu().numpy().view(np.uint64), 2 * ref)


def test_bin_snapshots_full_size(cuda):
    # 4 194 304 particles in L = 3740 at dx = 4 (935 x 935 lattice), g = 0.5
    n, L = mi.PRODUCTION_LJ.n, mi.PRODUCTION_LJ.box
    xp = mi.dyadic_positions(n, L, seed=3, bits=10, boundary_frac=0.02)
    xc = mi.displaced(xp, L, seed=4, scale=2.5, bits=10, boundary_frac=0.02)
    got_c, got_n, got_f = _run_bin(cuda, xp, xc, L, 4.0, 0.5, 3)
    ref_c, ref_n, ref_f, _ = oracle.mdlg_bin(xp, xc, 4.0, (935, 935), 3, field=True)
    assert np.array_equal(got_c, ref_c)
    assert np.array_equal(got_n, ref_n)
    assert np.array_equal(got_f, ref_f)


def _idealgas(cuda, pos, vel, combos, vmax):
    import torch
    q1 = (2 * vmax + 1) ** 2 + 1
    p = torch.from_numpy(pos).to(cuda)
    v = torch.from_numpy(vel).to(cuda)
    counts = torch.zeros((len(combos), q1), dtype=torch.int64, device=cuda)
    m.idealgas_bin(p, v, combos, vmax, counts)
    torch.cuda.synchronize()
    return counts.cpu().numpy().view(np.uint64)


def test_idealgas_bit_exact_small(cuda):
    pos, vel = mi.idealgas_state(300_001, 512.0, 1.0, seed=5)
    combos = list(mi.IDEALGAS_COMBOS) + [(3.0, 0.7), (1.5, 1.3)]   # last two: division path
    got = _idealgas(cuda, pos, vel, combos, 3)
    ref = oracle.stream_bin_f32(pos, vel, [c[0] for c in combos], [c[1] for c in combos], 3)
    assert np.array_equal(got, ref)


def test_idealgas_bit_exact_full_size(cuda):
    pos, vel = mi.idealgas_state(mi.IDEALGAS_N, mi.IDEALGAS_BOX, 1.0, seed=6)
    combos = list(mi.IDEALGAS_COMBOS)
    got = _idealgas(cuda, pos, vel, combos, 3)
    ref = oracle.stream_bin_f32(pos, vel, [c[0] for c in combos], [c[1] for c in combos], 3)
    assert np.array_equal(got, ref)
    assert np.all(got.sum(axis=1) == mi.IDEALGAS_N)


def test_idealgas_matches_closed_form(cuda):
    # Ballistic gas (Sec. IV-A): f_i / rho^eq of Eq. fialpha at a = sqrt(T) dt / dx;
    # each bin within 4 standard errors of the multinomial count.
    pos, vel = mi.idealgas_state(mi.IDEALGAS_N, mi.IDEALGAS_BOX, 1.0, seed=7)
    combos = list(mi.IDEALGAS_COMBOS)
    got = _idealgas(cuda, pos, vel, combos, 3)
    n = mi.IDEALGAS_N
    for k, (dx, dt) in enumerate(combos):
        p = cf.feq_window(3, cf.a_ballistic(1.0, dt, dx))
        se = np.sqrt(np.maximum(p * (1 - p), 1e-300) / n)
        z = np.abs(got[k] / n - p) / se
        assert np.all(z[p > 1e-6] < 4.0), (dx, dt, z.max())


def test_idealgas_largest_window_and_pair_count(cuda):
    # 16 (dx, dt) pairs with the V = 15 window: 16 x 962 histogram bins (61.6 KB of
    # shared memory, above the default 48 KB), non-power-of-two dx among them
    pos, vel = mi.idealgas_state(200_003, 256.0, 1.0, seed=12)
    combos = [(dx, dt) for dx in (1.0, 2.0, 4.0, 0.5) for dt in (0.25, 1.0, 3.0, 6.0)]
    combos[5] = (3.0, 1.5)
    got = _idealgas(cuda, pos, vel, combos, 15)
    ref = oracle.stream_bin_f32(pos, vel, [c[0] for c in combos], [c[1] for c in combos], 15)
    assert np.array_equal(got, ref)
    assert np.all(got.sum(axis=1) == 200_003)



@pytest.mark.parametrize("boost", [False, True])
@pytest.mark.parametrize("offset", [0, 1])
def test_idealgas_pow2_groups_bit_exact(cuda, boost, offset):
    # Every dx a power of two (0.5 ... 8), pairs given out of (dt, dx) order, dt
    # values shared by non-adjacent pairs, an odd particle count; with drifts,
    # pairs that share dt but not U.  offset = 1 starts both arrays 8 bytes into
    # a buffer (no 16-byte loads).
    import torch
    n = 100_003
    pos, vel = mi.idealgas_state(n + offset, 512.0, 1.0, seed=31)
    combos = [(2.0, 1.0), (0.5, 0.25), (8.0, 1.0), (1.0, 0.25), (2.0, 0.25), (4.0, 1.5),
              (1.0, 1.0), (0.5, 1.5), (2.0, 1.0)]
    us = None
    if boost:
        us = np.array([[0.4, 0.0], [0.0, 0.0], [0.4, 0.0], [-0.3, 0.2], [0.0, 0.0], [1.1, -0.9],
                       [0.4, 0.0], [0.0, 0.0], [0.0, 0.5]], np.float32)
    pb = torch.from_numpy(pos).to(cuda)
    vb = torch.from_numpy(vel).to(cuda)
    p, v = pb[offset:], vb[offset:]
    counts = torch.zeros((len(combos), 50), dtype=torch.int64, device=cuda)
    m.idealgas_bin(p, v, combos, 3, counts, us=us)
    torch.cuda.synchronize()
    got = counts.cpu().numpy().view(np.uint64)
    ref = oracle.stream_bin_f32(pos[offset:], vel[offset:], [c[0] for c in combos],
                                [c[1] for c in combos], 3, us=us)
    assert np.array_equal(got, ref)
    assert np.all(got.sum(axis=1) == n)


GRID_LAYOUTS = {
    # (dx values, dt values, drift per dt or None): pairs (dx, dt) for every dt and dx
    "ns2": ((0.5, 1.0), (0.25, 1.0, 2.0), None),
    "ns3": ((1.0, 2.0, 4.0), (0.5, 1.0, 2.0), None),
    "ns4": ((1.0, 2.0, 4.0, 8.0), (0.5, 2.0), None),
    "ns3_drift": ((1.0, 2.0, 4.0), (0.5, 1.0), ((0.4, -0.2), (0.0, 0.7))),
}


@pytest.mark.parametrize("layout", sorted(GRID_LAYOUTS) + ["near_grid"])
def test_idealgas_full_grid_layouts_bit_exact(cuda, layout):
    # Pair lists that form a full (dt, U) x dx grid run with the shifts as
    # compile-time constants (2, 3 or 4 dx per group); a list that is almost a
    # grid (the second group's largest dx differs) keeps the runtime shifts.
    # Pairs are given out of order and the particle count is odd; every layout is
    # bit-exact against the oracle.
    import torch
    n = 100_003
    pos, vel = mi.idealgas_state(n, 512.0, 1.0, seed=41)
    if layout == "near_grid":
        pairs = [(dx, 0.5) for dx in (1.0, 2.0, 4.0)] + [(dx, 1.0) for dx in (1.0, 2.0, 8.0)]
        drift = [None] * len(pairs)
    else:
        dxs, dts, us_ = GRID_LAYOUTS[layout]
        pairs, drift = [], []
        for g, dt in enumerate(dts):
            for dx in dxs:
                pairs.append((dx, dt))
                drift.append(None if us_ is None else us_[g])
    order = np.random.default_rng(7).permutation(len(pairs))
    combos = [pairs[i] for i in order]
    us = None
    if any(d is not None for d in drift):
        us = np.array([drift[i] for i in order], np.float32)
    counts = torch.zeros((len(combos), 50), dtype=torch.int64, device=cuda)
    m.idealgas_bin(torch.from_numpy(pos).to(cuda), torch.from_numpy(vel).to(cuda), combos, 3,
                   counts, us=us)
    torch.cuda.synchronize()
    got = counts.cpu().numpy().view(np.uint64)
    ref = oracle.stream_bin_f32(pos, vel, [c[0] for c in combos], [c[1] for c in combos], 3, us=us)
    assert np.array_equal(got, ref)
    assert np.all(got.sum(axis=1) == n)
