"""Pins for the oracle's paper analyses: the moving lattice (Sec. IV, u-sweep of
Fig. wi_u), the MDLG collision operator Xi_i (Eq. Xi) and the mean-square
displacement over a coarse time step (Sec. IV-A)."""
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
VEL = oracle.velocity_table(V)


def _wrap(x, L):
    """Map into (0, L] (exact for dyadic values)."""
    y = np.mod(x, L)
    return np.where(y == 0.0, L, y)


def _chi2_ok(got, p):
    n = got.sum()
    e = n * p
    m = e > 5
    chi2 = float((((got - e) ** 2)[m] / e[m]).sum())
    dof = int(m.sum()) - 1
    return chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


# ---- moving lattice -------------------------------------------------------

def test_moving_lattice_bins_the_shifted_positions():
    # Each snapshot is binned at x + S of its own time (Galilean-transformed
    # positions); shifts that carry points across the box edge wrap.
    C, dx = (12, 10), 2.0
    L = (C[0] * dx, C[1] * dx)
    xp = mi.dyadic_positions(4000, L[0], seed=11, bits=6, boundary_frac=0.2)
    xp[:, 1] = _wrap(xp[:, 1], L[1])
    xc = mi.displaced(xp, L[0], seed=12, scale=3.0, bits=6, boundary_frac=0.2)
    xc[:, 1] = _wrap(xc[:, 1], L[1])
    s_prev = np.array([17.375, -3.5])
    s_cur = np.array([18.0625, -2.75])
    got = oracle.mdlg_bin(xp, xc, dx, C, V, field=True, shift_prev=s_prev, shift_cur=s_cur)
    ref = oracle.mdlg_bin(np.stack([_wrap(xp[:, a] + s_prev[a], L[a]) for a in (0, 1)], 1),
                          np.stack([_wrap(xc[:, a] + s_cur[a], L[a]) for a in (0, 1)], 1),
                          dx, C, V, field=True)
    for g, r in zip(got[:3], ref[:3]):
        assert np.array_equal(g, r)
    # a shift by whole boxes changes nothing
    whole = oracle.mdlg_bin(xp, xc, dx, C, V, field=True, shift_prev=(L[0], -2 * L[1]),
                            shift_cur=(3 * L[0], L[1]))
    plain = oracle.mdlg_bin(xp, xc, dx, C, V, field=True)
    assert np.array_equal(whole[2], plain[2])
    # the shift must move the lattice against the particles: a positive S
    # with S_cur - S_prev = dx adds one lattice velocity in x to everybody
    sh = oracle.mdlg_bin(xp, xp, dx, C, V, shift_prev=(0.25, 0.0), shift_cur=(0.25 + dx, 0.0))
    assert sh[0][(0 + V) * W + (1 + V)] == xp.shape[0]


@pytest.mark.parametrize("u", [(0.0, 0.0), (0.1, 0.0), (0.3, -0.2), (0.5, 0.5)])
def test_moving_lattice_matches_closed_form_at_mean_velocity(u):
    # A gas at rest seen from a lattice moved by -U t has the equilibrium of
    # Eq. feqfull at mean velocity u = U dt / dx (Sec. IV, Fig. wi_u).
    L, dx, dt, T = 256.0, 2.0, 1.0, 1.0
    C = (int(L / dx),) * 2
    rng = np.random.default_rng(21)
    n = 300_000
    x0 = rng.uniform(0.0, L, size=(n, 2))
    v = rng.normal(0.0, math.sqrt(T), size=(n, 2))
    x1 = _wrap(x0 + v * dt, L)
    U = np.array(u) * dx / dt
    t0 = 37.0
    got = oracle.mdlg_bin(x0, x1, dx, C, V, shift_prev=U * t0, shift_cur=U * (t0 + dt))[0]
    p = cf.feq_window(V, cf.a_ballistic(T, dt, dx), u)
    ok, info = _chi2_ok(got.astype(np.float64), p)
    assert ok, info


def test_idealgas_boost_equals_boosted_velocities():
    pos, vel = mi.idealgas_state(30000, 64.0, 1.0, seed=31)
    dxs, dts = [1.0, 2.0, 4.0], [0.5, 1.0, 1.5]
    us = np.array([[0.25, -0.125], [1.0, 0.0], [-0.375, 0.5]], np.float32)
    got = oracle.stream_bin_f32(pos, vel, dxs, dts, V, us=us)
    for k in range(3):
        vb = (vel + us[k]).astype(np.float32)            # fl(v + U), binary32
        ref = oracle.stream_bin_f32(pos, vb, [dxs[k]], [dts[k]], V)
        assert np.array_equal(got[k], ref[0])
    assert np.array_equal(oracle.stream_bin_f32(pos, vel, dxs, dts, V, us=np.zeros((3, 2))),
                          oracle.stream_bin_f32(pos, vel, dxs, dts, V))


def test_idealgas_boost_matches_closed_form():
    pos, vel = mi.idealgas_state(400_000, 256.0, 1.0, seed=32)
    combos = [(2.0, 1.0, (0.2, 0.0)), (1.0, 0.5, (-0.3, 0.4))]
    us = np.array([[c[2][0] * c[0] / c[1], c[2][1] * c[0] / c[1]] for c in combos], np.float32)
    got = oracle.stream_bin_f32(pos, vel, [c[0] for c in combos], [c[1] for c in combos], V, us=us)
    for k, (dx, dt, u) in enumerate(combos):
        ok, info = _chi2_ok(got[k].astype(np.float64), cf.feq_window(V, cf.a_ballistic(1.0, dt, dx), u))
        assert ok, (k, info)


# ---- collision operator -----------------------------------------------------

def _cells(x, dx, C):
    c = np.ceil(x / dx).astype(np.int64) - 1
    return np.stack([c[:, 0] % C[0], c[:, 1] % C[1]], 1)


def _disp(d, C):
    r = d % C
    return np.where(r > C // 2, r - C, r)


def test_collision_by_particle_tracking():
    # Xi_i(x) = (particles in x at t that move by v_i next) - (particles in x at
    # t that arrived by v_i): counted particle by particle, with the overflow
    # (out-of-window) moves left out on both sides.
    C, dx = (9, 7), 2.0
    L = C[0] * dx
    x0 = mi.dyadic_positions(400, L, seed=41, bits=4, boundary_frac=0.2)
    x0[:, 1] = _wrap(x0[:, 1], C[1] * dx)
    x1 = mi.displaced(x0, L, seed=42, scale=5.0, bits=4, boundary_frac=0.2)
    x1[:, 1] = _wrap(x1[:, 1], C[1] * dx)
    x2 = mi.displaced(x1, L, seed=43, scale=5.0, bits=4, boundary_frac=0.2)
    x2[:, 1] = _wrap(x2[:, 1], C[1] * dx)
    f1 = oracle.mdlg_bin(x0, x1, dx, C, V, field=True)[2]
    f2 = oracle.mdlg_bin(x1, x2, dx, C, V, field=True)[2]
    xi = oracle.collision(C, V, f1, f2)
    c0, c1, c2 = (_cells(x, dx, C) for x in (x0, x1, x2))
    ref = np.zeros_like(xi)
    Ca = np.array(C)
    for j in range(x0.shape[0]):
        site = c1[j, 1] * C[0] + c1[j, 0]
        for d, sign in ((_disp(c2[j] - c1[j], Ca), 1), (_disp(c1[j] - c0[j], Ca), -1)):
            if abs(d[0]) <= V and abs(d[1]) <= V:
                ref[site, (d[1] + V) * W + d[0] + V] += sign
    assert np.array_equal(xi, ref)
    # overflow moves do happen in this case, so the check is not vacuous
    assert f1[:, Q].sum() > 0 and f2[:, Q].sum() > 0


def test_collision_conserves_mass_not_momentum():
    # Eq. masscons holds exactly when no move leaves the window; Eq.
    # momentumcons does not hold in general (Sec. III).
    L, dx, C = 48.0, 4.0, (12, 12)
    x0 = mi.dyadic_positions(3000, L, seed=44)
    x1 = mi.displaced(x0, L, seed=45, scale=2.0)
    x2 = mi.displaced(x1, L, seed=46, scale=2.0)
    f1 = oracle.mdlg_bin(x0, x1, dx, C, V, field=True)[2]
    f2 = oracle.mdlg_bin(x1, x2, dx, C, V, field=True)[2]
    assert f1[:, Q].sum() == 0 and f2[:, Q].sum() == 0
    xi = oracle.collision(C, V, f1, f2)
    assert not xi.sum(axis=1).any()
    mom = xi @ VEL
    assert np.abs(mom).sum() > 0
    # the momentum change summed over the lattice is the change of the total
    # lattice momentum between the two intervals
    assert np.array_equal(mom.sum(axis=0),
                          f2[:, :Q].sum(axis=0) @ VEL - f1[:, :Q].sum(axis=0) @ VEL)


def test_collision_of_fig2_example():
    # Fig. 2 (Sec. III): the tabulated f_0, f_1 of the single particle give
    # Xi_0(x,t) = f_0(x,t+1) - f_0(x,t) and Xi_1(x,t) = f_1(x+1,t+1) - f_1(x,t).
    rows = [tuple(int(v) for v in ln.split()) for ln in open(os.path.join(
            GOLDEN, "fig2_lattice_momentum.txt")) if ln.strip() and not ln.startswith("#")]
    tab = {(t, x): (f0, f1) for t, x, f0, f1 in rows}
    C = (8, 8)
    fields = {}
    for t in range(1, 7):
        xp = np.array([[1.1 + (t - 1) / 3, 0.5]])
        xc = np.array([[1.1 + t / 3, 0.5]])
        fields[t] = oracle.mdlg_bin(xp, xc, 1.0, C, V, field=True)[2]
    i0, i1 = V * W + V, V * W + V + 1
    checked = 0
    for t in range(1, 6):
        xi = oracle.collision(C, V, fields[t], fields[t + 1])
        for x in (1, 2, 3):
            assert xi[x, i0] == tab[(t + 1, x)][0] - tab[(t, x)][0], (t, x)
            checked += 1
            if (t + 1, x + 1) in tab:
                assert xi[x, i1] == tab[(t + 1, x + 1)][1] - tab[(t, x)][1], (t, x)
                checked += 1
    assert checked == 25
    # the particle turns from resting to moving at x = 1 between t = 2 and 3
    xi = oracle.collision(C, V, fields[2], fields[3])
    assert xi[1, i0] == -1 and xi[1, i1] == 1


# ---- mean-square displacement -----------------------------------------------

def test_msd_free_flight_exact():
    # dyadic free flight: every displacement is v dt exactly, also for the
    # particles that cross the periodic boundary (minimum image)
    L = 32.0
    rng = np.random.default_rng(51)
    x0 = mi.dyadic_positions(5000, L, seed=52)
    v = np.round(rng.normal(0.0, 3.0, size=(5000, 2)) * 256) / 256
    dt = 0.5
    x1 = _wrap(x0 + v * dt, L)
    assert ((x0 + v * dt) > L).any() and ((x0 + v * dt) <= 0).any()
    got = oracle.msd(x0, x1, (L, L))
    ref = ((v * dt) ** 2).mean(axis=0)
    assert np.array_equal(got, ref)
    assert np.array_equal(oracle.msd(x0, x0, (L, L)), np.zeros(2))


def test_msd_ballistic_expectation():
    # <dx_a^2> = T dt^2 for a ballistic gas at temperature T, unit mass (Sec. IV-A)
    L, T, dt, n = 100.0, 2.0, 0.7, 200_000
    rng = np.random.default_rng(53)
    x0 = rng.uniform(0.0, L, size=(n, 2))
    v = rng.normal(0.0, math.sqrt(T), size=(n, 2))
    got = oracle.msd(x0, _wrap(x0 + v * dt, L), (L, L))
    want = T * dt * dt
    assert np.allclose(got, want, rtol=5 * math.sqrt(2.0 / n))
