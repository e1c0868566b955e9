"""Pins for the closed-form equilibrium (Eq. fialpha) against independent computations."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

from oracle import closed_form as cf


def _quad_axis(k, u, a):
    # Eq. fgen, one axis, integrated numerically: int P(d + k) W(d) dd with P the
    # Gaussian of mean u and variance a^2 and W(d) = (1 - |d|)_+.
    def integrand(d):
        s = d + k - u
        return math.exp(-s * s / (2 * a * a)) / (math.sqrt(2 * math.pi) * a) * (1 - abs(d))
    val, _ = integrate.quad(integrand, -1.0, 1.0, points=[0.0], epsabs=1e-14, epsrel=1e-12,
                            limit=200)
    return val


@pytest.mark.parametrize("a2", [0.01, 1 / 16, 1 / 6, 0.25, 1.0, 4.0])
@pytest.mark.parametrize("u", [0.0, 0.17, -0.4])
def test_axis_factor_matches_quadrature(a2, u):
    a = math.sqrt(a2)
    for k in range(-4, 5):
        assert cf.f_axis(k - u, a) == pytest.approx(_quad_axis(k, u, a), abs=1e-11)


def test_matches_monte_carlo_binning():
    # Physical meaning: a point uniform in its cell, moved by a Gaussian step,
    # lands k cells away with probability f_k.  Sample it directly.
    rng = np.random.default_rng(7)
    n, a, u = 2_000_000, 0.6, 0.25
    x = 1.0 - rng.random(n)                       # (0, 1]: inside cell 0
    y = x + u + a * rng.standard_normal(n)
    k = np.ceil(y).astype(np.int64) - 1           # cell (k, k+1]
    for kk in range(-3, 4):
        p = cf.f_axis(kk - u, a)
        emp = np.mean(k == kk)
        se = math.sqrt(max(p * (1 - p), 1e-12) / n)
        assert abs(emp - p) < 5 * se + 1e-9, (kk, emp, p)


@pytest.mark.parametrize("a2", [0.003, 0.1, 1 / 6, 1.0, 9.0])
@pytest.mark.parametrize("u", [0.0, 0.3, -0.45])
def test_normalisation_and_first_moment(a2, u):
    # The axis factors are a probability distribution over integer k with mean u
    # (the Gaussian step has mean u; the wedge is symmetric).
    a = math.sqrt(a2)
    ks = np.arange(-40, 41)
    f = np.array([cf.f_axis(k - u, a) for k in ks])
    assert f.min() >= -1e-15
    assert f.sum() == pytest.approx(1.0, abs=1e-12)
    assert (ks * f).sum() == pytest.approx(u, abs=1e-12)


def test_second_moment_offset_one_sixth():
    # Sec. VI (Eq. m2): the discrete second moment approaches a^2 + 1/6 once a^2
    # is large; the 1/6 is the variance of the difference of two independent
    # uniform in-cell offsets.
    for a2 in (2.0, 4.0, 9.0):
        a = math.sqrt(a2)
        ks = np.arange(-60, 61)
        f = np.array([cf.f_axis(k, a) for k in ks])
        assert (ks * ks * f).sum() - a2 == pytest.approx(1 / 6, abs=1e-9)


def test_zero_width_limit_is_wedge():
    # P -> delta: f_k = W(k - u), the linear overlap of the shifted cell.
    for u in (0.0, 0.3, -0.7):
        for k in range(-2, 3):
            w = max(0.0, 1 - abs(k - u))
            assert cf.f_axis(k - u, 1e-7) == pytest.approx(w, abs=1e-7)  # O(a) at the kinks
            assert cf.f_axis(k - u, 0.0) == pytest.approx(w, abs=0)


def test_window_and_overflow():
    f = cf.feq_window(3, 2.0)
    assert f.shape == (50,)
    assert f.sum() == pytest.approx(1.0, abs=1e-12)
    fx = np.array([cf.f_axis(k, 2.0) for k in range(-3, 4)])
    assert f[49] == pytest.approx(1 - fx.sum() ** 2, abs=1e-12)
    # the window is ordered i = (v_y + V)(2V+1) + (v_x + V)
    assert f[3 * 7 + 4] == pytest.approx(cf.f_axis(1, 2.0) * cf.f_axis(0, 2.0))


def test_d2q9_match_near_one_sixth():
    # Sec. V (Eq. wif0eqn): each D2Q9 weight is met by f_i^eq/rho at a^2 close
    # to 1/6, and the three solutions nearly coincide.  The roots are solved
    # twice: from the closed form, and from the wedge integral of Eq. fgen
    # evaluated by quadrature (independent of the erf algebra); both must give
    # 0.1771 (rest), 0.1836 (axis) and 0.1801 (diagonal) to 1e-4.
    def feq(a2, v):
        return cf.feq_over_rho(v, math.sqrt(a2))

    def feq_quad(a2, v):
        a = math.sqrt(a2)
        return _quad_axis(v[0], 0.0, a) * _quad_axis(v[1], 0.0, a)

    cases = (((0, 0), 4 / 9, 0.1771), ((1, 0), 1 / 9, 0.1836), ((1, 1), 1 / 36, 0.1801))
    roots = []
    for v, w, expect in cases:
        r = optimize.brentq(lambda a2: feq(a2, v) - w, 0.05, 0.5, xtol=1e-14)
        rq = optimize.brentq(lambda a2: feq_quad(a2, v) - w, 0.05, 0.5, xtol=1e-12)
        assert r == pytest.approx(expect, abs=1e-4), (v, r)
        assert rq == pytest.approx(r, abs=1e-9), (v, rq, r)
        roots.append(r)
    assert max(roots) - min(roots) < 0.01, roots


def test_ballistic_width_and_vacf_limits():
    # Sec. IV-A: <dx^2> = T dt^2 for free flight; Eq. vca has the same short-time
    # limit and the diffusive long-time limit 2 T tau t.
    assert cf.a_ballistic(1.0, 2.0, 4.0) == pytest.approx(0.5)
    t, tau, T = 1e-4, 0.5, 50.0
    assert cf.msd_exponential_vacf(T, tau, t) == pytest.approx(T * t * t, rel=1e-3)
    t = 1e3
    assert cf.msd_exponential_vacf(T, tau, t) == pytest.approx(2 * T * tau * t, rel=1e-3)
