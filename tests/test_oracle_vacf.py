"""Pins of the oracle's half-step velocity and velocity correlation (Sec. IV-A,
Fig. VD(a)) against what kinematics fixes: free flight, the velocity-Verlet
kick, and the one-step mean-square displacement."""
import numpy as np
import pytest

import mdlg_inputs as mi
import oracle


def test_free_flight_correlation_is_the_mean_square_velocity():
    # no forces: every half-step velocity is the initial one, so the correlation
    # over any lag is <v_a^2>, computed here directly (dyadic values: exact)
    rng = np.random.default_rng(3)
    n, L, dt = 500, 64.0, 0.125
    x0 = mi.dyadic_positions(n, L, seed=5, bits=12)
    v = np.round(rng.normal(0.0, 1.5, size=(n, 2)) * 256) / 256
    x1 = oracle.free_stream(x0, v, (L, L), dt, 7)
    x2 = oracle.free_stream(x1, v, (L, L), dt, 1)
    x3 = oracle.free_stream(x2, v, (L, L), dt, 13)
    x4 = oracle.free_stream(x3, v, (L, L), dt, 1)
    va = oracle.half_velocity(x1, x2, (L, L), dt)
    vb = oracle.half_velocity(x3, x4, (L, L), dt)
    assert np.array_equal(va, v) and np.array_equal(vb, v)
    c = oracle.vacf(va, vb)
    assert c[0] == np.mean(v[:, 0] ** 2) and c[1] == np.mean(v[:, 1] ** 2)


def test_half_velocity_is_the_verlet_kick():
    # after a velocity-Verlet step x' = x + v dt + F dt^2 / 2m, so the half-step
    # velocity (x' - x) / dt equals v + F dt / 2m from the forces at x
    n = 1024
    L = mi.box_for(n, 0.3, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=7)
    dt = 0.005
    f0, _, _, _ = oracle.lj_forces(x0, (L, L))
    vv = oracle.VV(x0, v0, (L, L), dt).run(1)
    vh = oracle.half_velocity(x0, vv.x, (L, L), dt)
    np.testing.assert_allclose(vh, v0 + f0 * dt / 2.0, rtol=0, atol=1e-9)
    np.testing.assert_allclose(oracle.initial_half_velocity(x0, v0, (L, L), dt),
                               v0 - f0 * dt / 2.0, rtol=0, atol=0)


def test_self_correlation_matches_the_one_step_msd():
    # one step moves each particle by v_half dt, so <v_a v_a> of that velocity
    # with itself, times dt^2, is the mean-square displacement of the step
    n = 2048
    L = mi.box_for(n, 0.45, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.2, seed=8)
    dt = 0.005
    vv = oracle.VV(x0, v0, (L, L), dt).run(20)
    x20 = vv.x.copy()
    vv.run(1)
    vh = oracle.half_velocity(x20, vv.x, (L, L), dt)
    c = oracle.vacf(vh, vh)
    m = oracle.msd(x20, vv.x, (L, L))
    np.testing.assert_allclose(c * dt * dt, m, rtol=1e-12)
    # the axes are not mixed: the cross product is a different number
    assert abs(np.mean(vh[:, 0] * vh[:, 1]) - c[0]) > 1e-3


def test_correlation_decays_from_the_temperature():
    # equipartition: at a small lag the correlation per axis is close to T, and
    # at a lag of several collision times it has decayed well below it
    n = 4096
    L = mi.box_for(n, 0.3, 4.0)
    T, dt = 1.0, 0.005
    x0, v0 = mi.lj_initial_state(n, L, T, seed=9)
    vv = oracle.VV(x0, v0, (L, L), dt, cells=True).run(200)
    x = vv.x.copy()
    vv.run(1)
    v_a = oracle.half_velocity(x, vv.x, (L, L), dt)
    x = vv.x.copy()
    vv.run(1)
    v_b = oracle.half_velocity(x, vv.x, (L, L), dt)
    near = oracle.vacf(v_a, v_b).mean()
    x = vv.x.copy()
    vv.run(400)
    xp = vv.x.copy()
    vv.run(1)
    v_c = oracle.half_velocity(xp, vv.x, (L, L), dt)
    far = oracle.vacf(v_a, v_c).mean()
    temp = vv.kinetic()[0] / (n - 1)
    assert near == pytest.approx(temp, rel=0.06)
    assert abs(far) < 0.25 * temp
