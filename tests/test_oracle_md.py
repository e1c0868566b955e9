"""Pins for the oracle's Lennard-Jones forces and velocity-Verlet integrator."""
import math

import numpy as np
import pytest

import mdlg_inputs as mi
import oracle

BOX = (20.0, 20.0)


def _pair(r, angle=0.3):
    c = np.array([10.0, 10.0])
    d = r * np.array([math.cos(angle), math.sin(angle)])
    return np.stack([c, c + d])


def test_pair_textbook_points():
    # V(sigma) = 0 and the minimum V(2^(1/6) sigma) = -eps with zero force;
    # the energy is shifted so that V(rc) = 0.
    vrc = 4.0 * (2.5 ** -12 - 2.5 ** -6)
    _, _, pe, _ = oracle.lj_forces(_pair(1.0), BOX)
    assert pe == pytest.approx(-vrc, abs=1e-12)
    f, _, pe, _ = oracle.lj_forces(_pair(2 ** (1 / 6)), BOX)
    assert pe == pytest.approx(-1.0 - vrc, abs=1e-13)
    assert np.abs(f).max() < 1e-12
    f, _, pe, vir = oracle.lj_forces(_pair(2.5000001), BOX)
    assert pe == 0 and vir == 0 and np.abs(f).max() == 0


def test_pair_repulsive_inside_attractive_outside():
    f, _, _, _ = oracle.lj_forces(_pair(1.0, 0.0), BOX)
    assert f[1, 0] > 0 and f[0, 0] < 0          # pushed apart
    f, _, _, _ = oracle.lj_forces(_pair(1.5, 0.0), BOX)
    assert f[1, 0] < 0 and f[0, 0] > 0          # pulled together


def _pe(x, box):
    return oracle.lj_forces(x, box)[2]


def test_force_is_minus_gradient_of_energy():
    x, _ = mi.lj_initial_state(60, 12.0, 1.0, seed=3)
    box = (12.0, 12.0)
    f, _, _, _ = oracle.lj_forces(x, box)
    h = 1e-6
    for i in (0, 7, 33):
        for a in (0, 1):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            g = (_pe(xp, box) - _pe(xm, box)) / (2 * h)
            assert -g == pytest.approx(f[i, a], rel=1e-6, abs=1e-6)


def test_virial_is_scaling_derivative():
    # W = sum_{i<j} r_ij . F_ij = -d/dl PE(l x) at l = 1 (box scaled with x).
    x, _ = mi.lj_initial_state(80, 14.0, 1.0, seed=4)
    _, _, _, vir = oracle.lj_forces(x, (14.0, 14.0))
    h = 1e-6
    pp = oracle.lj_forces(x * (1 + h), (14.0 * (1 + h),) * 2)[2]
    pm = oracle.lj_forces(x * (1 - h), (14.0 * (1 - h),) * 2)[2]
    assert vir == pytest.approx(-(pp - pm) / (2 * h), rel=1e-6)


def test_newton_third_law_and_periodic_images():
    x, _ = mi.lj_initial_state(300, 20.0, 1.0, seed=5)
    f, _, _, _ = oracle.lj_forces(x, BOX)
    assert np.abs(f.sum(axis=0)).max() < 1e-10 * np.abs(f).max()
    # shifting every particle by a box length changes nothing
    f2, _, _, _ = oracle.lj_forces(x + np.array([20.0, -20.0]), BOX)
    assert np.abs(f - f2).max() < 1e-10


def test_cells_equal_direct():
    for n, L, seed in ((400, 24.0, 1), (2000, 80.0, 2), (700, 30.0, 3)):
        x, _ = mi.lj_initial_state(n, L, 1.0, seed)
        fd, sd, ped, vd = oracle.lj_forces(x, (L, L))
        fc, sc, pec, vc = oracle.lj_forces(x, (L, L), cells=True)
        assert np.abs(fd - fc).max() < 1e-11
        assert np.abs(sd - sc).max() < 1e-11
        assert ped == pytest.approx(pec, rel=1e-12)
        assert vd == pytest.approx(vc, rel=1e-12)


def test_sample_forces_equal_full():
    x, _ = mi.lj_initial_state(500, 30.0, 1.0, seed=9)
    f, fs, _, _ = oracle.lj_forces(x, (30.0, 30.0))
    which = np.array([0, 17, 499, 250])
    g, gs = oracle.lj_forces_sample(x, (30.0, 30.0), which)
    assert np.array_equal(g, f[which]) and np.array_equal(gs, fs[which])


def test_free_flight_exact():
    # eps = 0 switches the potential off: x(t) = x0 + v t exactly (mod L).
    x, v = mi.lj_initial_state(50, 10.0, 1.0, seed=6)
    s = oracle.VV(x, v, (10.0, 10.0), dt=0.01, eps=0.0)
    s.run(100)
    ref = x + v * 1.0
    d = s.x - ref
    d -= 10.0 * np.round(d / 10.0)
    assert np.abs(d).max() < 1e-11
    assert np.array_equal(s.v, v)


def test_momentum_conserved_and_time_reversible():
    x, v = mi.lj_initial_state(256, 32.0, 1.0, seed=8)
    s = oracle.VV(x, v, (32.0, 32.0), dt=0.005)
    p0 = s.kinetic()[1:]
    s.run(100)
    assert np.abs(s.kinetic()[1:] - p0).max() < 1e-10
    s.v = -s.v
    s.run(100)
    d = s.x - x
    d -= 32.0 * np.round(d / 32.0)
    assert np.abs(d).max() < 1e-9
    assert np.abs(s.v + v).max() < 1e-9


def test_energy_error_second_order_in_dt():
    # Velocity Verlet is second order: the energy fluctuation over a fixed time
    # falls by ~4x when dt halves (the truncated force adds a small floor).
    x, v = mi.lj_initial_state(200, 28.0, 1.0, seed=11)

    def max_dev(dt):
        s = oracle.VV(x, v, (28.0, 28.0), dt=dt)
        e0 = s.energy()
        dev = 0.0
        for _ in range(20):
            s.run(int(round(0.05 / dt)))
            dev = max(dev, abs(s.energy() - e0))
        return dev

    d1, d2 = max_dev(0.004), max_dev(0.002)
    assert 2.5 < d1 / d2 < 6.0, (d1, d2)


def test_small_config_energy_drift():
    # 2000 steps of the N = 1024, L = 64 gas at dt = 0.005: total energy per
    # particle stays within 2e-3 of its start (truncated force at rc included).
    c = mi.SMALL_LJ
    x, v = mi.lj_initial_state(c.n, c.box, c.temperature, seed=1)
    s = oracle.VV(x, v, (c.box, c.box), dt=c.dt, cells=True)
    e0 = s.energy()
    s.run(2000)
    assert abs(s.energy() - e0) / c.n < 2e-3


def test_shifted_force_vanishes_continuously_at_cutoff():
    # shifted force: F(rc-) = 0 and the pair energy is 0 at rc, with no jump
    f_in, _, pe_in, _ = oracle.lj_forces(_pair(2.5 - 1e-7), BOX, shifted_force=True)
    f_out, _, pe_out, _ = oracle.lj_forces(_pair(2.5 + 1e-7), BOX, shifted_force=True)
    assert np.abs(f_in).max() < 1e-6 and abs(pe_in) < 1e-12 and pe_out == 0   # F ~ F'(rc) 1e-7
    # truncated force: a jump of |F(rc)| = 24 (2 rc^-13 - rc^-7) at the cutoff
    f_ts, _, _, _ = oracle.lj_forces(_pair(2.5 - 1e-9, 0.0), BOX)
    assert abs(np.hypot(*f_ts[0])) == pytest.approx(abs(24 * (2 * 2.5 ** -13 - 2.5 ** -7)),
                                                    rel=1e-6)


@pytest.mark.parametrize("sf", [False, True])
def test_force_is_minus_gradient_both_cutoffs(sf):
    x, _ = mi.lj_initial_state(60, 12.0, 1.0, seed=13)
    box = (12.0, 12.0)
    f, _, _, _ = oracle.lj_forces(x, box, shifted_force=sf)
    h = 1e-6
    for i in (1, 22, 50):
        for a in (0, 1):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            g = (oracle.lj_forces(xp, box, shifted_force=sf)[2]
                 - oracle.lj_forces(xm, box, shifted_force=sf)[2]) / (2 * h)
            assert -g == pytest.approx(f[i, a], rel=1e-6, abs=1e-6)


def test_shifted_force_conserves_energy_tightly():
    # continuous forces: VV energy error is second order without cutoff kicks
    x, v = mi.lj_initial_state(200, 28.0, 1.0, seed=11)
    s = oracle.VV(x, v, (28.0, 28.0), dt=0.002, shifted_force=True)
    e0 = s.energy()
    s.run(500)
    assert abs(s.energy() - e0) / 200 < 2e-4
