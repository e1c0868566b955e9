"""Host analyses of the equilibrium (moments Psi, Phi, theta_2, theta_3 and the
consistent (dx, dt) solve of Secs. V-VI) against the oracle's independent
closed form and the statements the paper makes about them."""
import itertools
import math

import numpy as np
import pytest

from oracle import closed_form as cf
from paper_1705_04368_gb300 import analysis as an


@pytest.mark.parametrize("vmax,a,u", [(3, 0.4, (0.0, 0.0)), (3, 0.2, (0.3, -0.1)),
                                      (7, 1.5, (0.5, 0.25)), (15, 4.0, (-0.2, 0.0)),
                                      (1, 0.05, (0.0, 0.4))])
def test_feq_matches_oracle_closed_form(vmax, a, u):
    assert np.allclose(an.feq(vmax, a, u), cf.feq_window(vmax, a, u), rtol=1e-13, atol=1e-16)


def test_moments_by_brute_force():
    rng = np.random.default_rng(3)
    V = 2
    f = rng.random((2 * V + 1) ** 2 + 1)
    u = (0.13, -0.31)
    out = an.moments(f, V, u, a=0.7)
    rho = m2 = m3 = 0.0
    m2 = np.zeros((2, 2))
    m3 = np.zeros((2, 2, 2))
    mean = np.zeros(2)
    for vy in range(-V, V + 1):
        for vx in range(-V, V + 1):
            fi = f[(vy + V) * (2 * V + 1) + vx + V]
            rho += fi
            c = (vx - u[0], vy - u[1])
            mean += fi * np.array([vx, vy])
            for p, q in itertools.product(range(2), repeat=2):
                m2[p, q] += fi * c[p] * c[q]
                for r in range(2):
                    m3[p, q, r] += fi * c[p] * c[q] * c[r]
    assert out["rho"] == pytest.approx(rho, rel=1e-14)
    assert np.allclose(out["mean"], mean / rho, rtol=1e-13)
    assert np.allclose(out["Psi"], m2 / rho / 0.49, rtol=1e-13)
    assert np.allclose(out["Phi"], m3 / rho / 0.343, rtol=1e-13)


def test_d2q9_weights_have_lattice_boltzmann_moments():
    # Sec. V: the D2Q9 weights carry theta = 1/3 and no third moment at u = 0
    f = np.zeros(10)
    for vy in (-1, 0, 1):
        for vx in (-1, 0, 1):
            key = (abs(vx), abs(vy)) if abs(vx) >= abs(vy) else (abs(vy), abs(vx))
            f[(vy + 1) * 3 + vx + 1] = an.D2Q9[key]
    out = an.moments(f, 1)
    assert out["rho"] == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(out["M2"], np.eye(2) / 3.0, atol=1e-15)
    assert np.allclose(out["M3"], 0.0, atol=1e-15)


def test_second_moment_offset_one_sixth():
    # Sec. VI (Fig. m2): the discrete second moment exceeds a^2 by 1/6 once
    # a^2 > 0.2 (1/12 from the cell width, 1/12 from the discrete moment)
    for a2, tol in ((0.5, 1e-5), (1.0, 1e-8), (4.0, 1e-8)):
        th = an.theta2(an.feq(15, math.sqrt(a2)), 15)
        assert th - a2 == pytest.approx(1.0 / 6.0, abs=tol), a2
    assert abs(an.theta2(an.feq(15, math.sqrt(0.05)), 15) - 0.05 - 1.0 / 6.0) > 0.01


def test_psi_galilean_invariance_only_for_wide_distributions():
    # Fig. Psi: Psi_xx is independent of u for large a^2 and strongly u-dependent
    # below a^2 = 0.1
    def psi(a2, ux):
        a = math.sqrt(a2)
        return an.moments(an.feq(15, a, (ux, 0.0)), 15, (ux, 0.0), a=a)["Psi"][0, 0]
    assert abs(psi(4.0, 0.5) - psi(4.0, 0.0)) < 1e-6
    assert abs(psi(0.05, 0.5) / psi(0.05, 0.0) - 1.0) > 0.3


def _one_shell_crossing(fn):
    grid = np.linspace(0.10, 0.30, 201)
    vals = [fn(a2) for a2 in grid]
    for k in range(len(grid) - 1):
        if (vals[k] > 0) != (vals[k + 1] > 0):
            return grid[k]
    return None


def test_one_shell_third_moment_vanishes_near_a2_one_sixth():
    # Fig. f3: restricted to one shell, Phi_xxx collapses to zero at a^2 ~ 1/6
    def phi(a2):
        a = math.sqrt(a2)
        return an.moments(an.feq(3, a, (0.001, 0.0)), 3, (0.001, 0.0), a=a, shells=1)["Phi"][0, 0, 0]
    x = _one_shell_crossing(phi)
    assert x is not None and abs(x - 1.0 / 6.0) < 0.02


def test_one_shell_temperatures_agree_at_one_third():
    # Fig. tet: one-shell theta_2 and theta_3 agree at one point, theta ~ 1/3,
    # a^2 ~ 1/6; with the full set they agree only for large a^2
    du = 1e-4

    def diff(a2, shells=1, V=7):
        a = math.sqrt(a2)
        t2 = an.theta2(an.feq(V, a), V, shells=shells)
        t3 = an.theta3(an.feq(V, a, (du, 0.0)), an.feq(V, a, (-du, 0.0)), du, V, shells=shells)
        return t2 - t3, t2
    x = _one_shell_crossing(lambda a2: diff(a2)[0])
    assert x is not None and abs(x - 1.0 / 6.0) < 0.02
    assert diff(x)[1] == pytest.approx(1.0 / 3.0, abs=0.02)
    assert abs(diff(0.15, None, 15)[0]) > 0.02 and abs(diff(3.0, None, 15)[0]) < 1e-6


def test_msd_model_limits():
    # Eq. vca: ballistic T t^2 for t << tau, diffusive 2 T tau t for t >> tau
    T, tau = 50.0, 0.5
    assert an.msd_exponential(T, tau, 1e-4) == pytest.approx(T * 1e-8, rel=1e-3)
    assert an.msd_exponential(T, tau, 500.0) == pytest.approx(2 * T * tau * 500.0, rel=2e-3)
    for t in (0.01, 0.3, 2.0, 40.0):
        assert an.msd_exponential(T, tau, t) == pytest.approx(cf.msd_exponential_vacf(T, tau, t),
                                                              rel=1e-12)


def test_consistent_dt_regimes():
    # Fig. dtdx: dt ~ dx in the ballistic regime, dt ~ dx^2 in the diffusive one,
    # and the three D2Q9 weights give nearly the same a^2 (close to 1/6)
    T, tau = 50.0, 0.5
    small = [an.consistent_dt(dx, T, tau)[(0, 0)][1] for dx in (0.01, 0.02)]
    large = [an.consistent_dt(dx, T, tau)[(0, 0)][1] for dx in (1000.0, 2000.0)]
    assert small[1] / small[0] == pytest.approx(2.0, rel=1e-3)
    assert large[1] / large[0] == pytest.approx(4.0, rel=1e-2)
    sol = an.consistent_dt(100.0, T, tau)
    a2s = [v[0] for v in sol.values()]
    assert max(a2s) - min(a2s) < 0.01 and all(abs(a - 1.0 / 6.0) < 0.02 for a in a2s)
    for v, (a2, dt) in sol.items():
        a = math.sqrt(a2)
        w = an.D2Q9[v]
        assert cf.feq_over_rho(v, a) == pytest.approx(w, rel=1e-9)
        assert an.msd_exponential(T, tau, dt) == pytest.approx(a2 * 1e4, rel=1e-9)


def test_lb_equilibrium_moments():
    # Eq. f0lb with theta = 1/3 reproduces Eqs. mom0-tet exactly (to second order
    # in u) and carries the third moment rho u u u on one shell (Sec. V)
    u = (0.07, -0.04)
    f = an.lb_equilibrium(u, vmax=2)
    out = an.moments(f, 2, u)
    assert out["rho"] == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(out["mean"], u, atol=1e-15)
    assert np.allclose(out["M2"], np.eye(2) / 3.0, atol=1e-14)
    # one shell has v^3 = v, so the central third moment is -rho u_x^3: of the
    # size rho u u u the paper calls small for u < 0.1
    assert out["M3"][0, 0, 0] == pytest.approx(-u[0] ** 3, abs=1e-15)
    assert np.allclose(an.lb_equilibrium((0.0, 0.0))[:9],
                       [1 / 36, 1 / 9, 1 / 36, 1 / 9, 4 / 9, 1 / 9, 1 / 36, 1 / 9, 1 / 36])
