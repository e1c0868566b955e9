"""Pins for the oracle's MDLG occupation numbers (Eq. MDni) and ideal-gas binning."""
import math
import os

import numpy as np
import pytest

import mdlg_inputs as mi
import oracle
from oracle import closed_form as cf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
V = 3
W = 2 * V + 1
Q = W * W


def _idx(vx, vy):
    return (vy + V) * W + (vx + V)


def test_fig2_worked_example():
    # Fig. 2 (Sec. III): a particle at x(t) = 1.1 + t/3 (dx = 1) in a 1D row.
    rows = [tuple(int(v) for v in ln.split()) for ln in open(os.path.join(GOLDEN,
            "fig2_lattice_momentum.txt")) if ln.strip() and not ln.startswith("#")]
    table = {(t, x): (f0, f1) for t, x, f0, f1 in rows}
    C = (8, 8)
    mom = 0
    for t in range(1, 7):
        xp = np.array([[1.1 + (t - 1) / 3, 0.5]])
        xc = np.array([[1.1 + t / 3, 0.5]])
        counts, ncell, field, vsum = oracle.mdlg_bin(xp, xc, 1.0, C, V, field=True)
        mom += vsum[0]
        for x in (1, 2, 3):
            f0 = field[0 * C[0] + x, _idx(0, 0)]
            f1 = field[0 * C[0] + x, _idx(1, 0)]
            assert (f0, f1) == table[(t, x)], (t, x)
    # the lattice momentum averages to the particle's 1/3 cell per step
    assert mom == 2


def _brute_force(xprev, xcur, dx, C):
    # Eq. MDni with the cell indicator written out as interval tests:
    # Delta_x(x') = 1 iff x_a < x'_a <= x_a + dx for every axis, with the
    # periodic images of the site considered.
    L = (C[0] * dx, C[1] * dx)
    vr = range(-V, V + 1)

    def inside(site, p):
        ok = True
        for a in (0, 1):
            lo = site[a] * dx
            hit = any(lo + m * L[a] < p[a] <= lo + dx + m * L[a] for m in (-1, 0, 1))
            ok &= hit
        return ok

    n = np.zeros((C[1] * C[0], Q + 1), np.int64)
    for sy in range(C[1]):
        for sx in range(C[0]):
            for j in range(xcur.shape[0]):
                if not inside((sx, sy), xcur[j]):
                    continue
                found = False
                for vy in vr:
                    for vx in vr:
                        if inside((sx - vx, sy - vy), xprev[j]):
                            n[sy * C[0] + sx, _idx(vx, vy)] += 1
                            found = True
                if not found:
                    n[sy * C[0] + sx, Q] += 1
    return n


def test_brute_force_recount():
    C, dx = (9, 8), 2.0
    L = C[0] * dx
    # 9 x 8 cells of side 2; dyadic points, 20% exactly on base-grid lines
    xp = mi.dyadic_positions(60, L, seed=1, bits=4, boundary_frac=0.2)
    xp[:, 1] = np.minimum(xp[:, 1], C[1] * dx)
    xc = mi.displaced(xp, L, seed=2, scale=2.5, bits=4, boundary_frac=0.2)
    xc[:, 1] = np.where(xc[:, 1] > C[1] * dx, xc[:, 1] - 2.0, xc[:, 1])
    counts, ncell, field, _ = oracle.mdlg_bin(xp, xc, dx, C, V, field=True)
    ref = _brute_force(xp, xc, dx, C)
    assert np.array_equal(field.astype(np.int64), ref)
    assert np.array_equal(counts.astype(np.int64), ref.sum(axis=0))


def test_partition_of_unity_and_boundaries():
    L, dx = 64.0, 4.0
    C = (16, 16)
    xp = mi.dyadic_positions(5000, L, seed=3)
    xc = mi.displaced(xp, L, seed=4, scale=3.0)
    counts, ncell, field, _ = oracle.mdlg_bin(xp, xc, dx, C, V, field=True)
    assert np.array_equal(field.sum(axis=1), ncell)          # N = sum_i n_i
    assert int(ncell.sum()) == 5000 and int(counts.sum()) == 5000
    # a point exactly on x = dx is in cell 0; x = L is in the last cell
    e = np.array([[4.0, 4.0], [64.0, 64.0], [4.0 + 2 ** -16, 0.5]])
    _, nc, _, _ = oracle.mdlg_bin(e, e, dx, C, V)
    assert nc[0] == 1 and nc[16 * 16 - 1] == 1 and nc[1] == 1


def test_mass_conservation_across_intervals():
    # Sec. III (Eq. Mom0): the particles in cell x at t are the particles that
    # leave x by t + dt, so sum_i n_i(x + v_i, t + dt) = N(x, t).
    L, dx, C = 48.0, 4.0, (12, 12)
    x0 = mi.dyadic_positions(3000, L, seed=5)
    x1 = mi.displaced(x0, L, seed=6, scale=2.0)
    x2 = mi.displaced(x1, L, seed=7, scale=2.0)
    _, n1, _, _ = oracle.mdlg_bin(x0, x1, dx, C, V, field=True)
    c2, _, f2, _ = oracle.mdlg_bin(x1, x2, dx, C, V, field=True)
    assert c2[Q] == 0
    vel = oracle.velocity_table(V)
    back = np.zeros(C[0] * C[1], np.int64)
    for s in range(C[0] * C[1]):
        sx, sy = s % C[0], s // C[0]
        for i, (vx, vy) in enumerate(vel):
            back[s] += f2[((sy + vy) % C[1]) * C[0] + (sx + vx) % C[0], i]
    assert np.array_equal(back, n1.astype(np.int64))


def test_stream_bin_equals_snapshot_bin():
    pos, vel = mi.idealgas_state(20000, 64.0, 1.0, seed=8)
    combos = [(1.0, 0.5), (2.0, 1.0), (4.0, 2.0), (2.0, 2.0)]
    got = oracle.stream_bin_f32(pos, vel, [c[0] for c in combos], [c[1] for c in combos], V)
    for k, (dx, dt) in enumerate(combos):
        moved = (pos + vel * np.float32(dt)).astype(np.float32)       # binary32, two roundings
        moved = np.where(moved <= 0, moved + np.float32(64.0), moved)
        moved = np.where(moved > 64, moved - np.float32(64.0), moved)
        C = (int(64 / dx),) * 2
        ref, _, _, _ = oracle.mdlg_bin(pos.astype(np.float64), moved.astype(np.float64), dx, C, V)
        # wrapping a binary32 value can shift it across a boundary by rounding;
        # allow those few particles only
        diff = np.abs(got[k].astype(np.int64) - ref.astype(np.int64)).sum()
        assert diff <= 4, (dx, dt, diff)


def test_ideal_gas_matches_closed_form():
    # Ballistic gas: counts are multinomial with the closed-form probabilities
    # of Eq. fialpha at a = sqrt(T) dt / dx; chi-square over the 50 bins.
    pos, vel = mi.idealgas_state(400_000, 256.0, 1.0, seed=9)
    combos = [(1.0, 0.5), (2.0, 1.0), (1.0, 2.0), (4.0, 1.0)]
    got = oracle.stream_bin_f32(pos, vel, [c[0] for c in combos], [c[1] for c in combos], V)
    for k, (dx, dt) in enumerate(combos):
        p = cf.feq_window(V, cf.a_ballistic(1.0, dt, dx))
        n = got[k].sum()
        e = n * p
        m = e > 5
        chi2 = float((((got[k] - e) ** 2)[m] / e[m]).sum())
        dof = int(m.sum()) - 1
        assert chi2 < dof + 5 * math.sqrt(2 * dof), (dx, dt, chi2, dof)
