"""Pins for the soft-binned MDLG occupations (the adjoint's loss)."""
import numpy as np
import pytest

import mdlg_inputs as mi
import oracle
from oracle import closed_form as cf


def test_soft_tends_to_hard_counts():
    # s -> 0: the smoothed boxes become the cell indicators of Sec. III, so the
    # soft f_i equal Eq. MDni's counts / N (points kept off cell boundaries).
    L, dx = 64.0, 4.0
    xp = mi.dyadic_positions(3000, L, seed=1, bits=12, boundary_frac=0.0)
    xc = mi.displaced(xp, L, seed=2, scale=2.0, bits=12, boundary_frac=0.0)
    xp = np.where(np.abs(xp / dx - np.round(xp / dx)) < 1e-3, xp + 0.01, xp)
    xc = np.where(np.abs(xc / dx - np.round(xc / dx)) < 1e-3, xc + 0.01, xc)
    hard, _, _, _ = oracle.mdlg_bin(xp, xc, dx, (16, 16), 3)
    soft = cf.soft_fi(xc, xp, (L, L), dx, 1e-6, 3)
    assert np.allclose(soft, hard[:49] / 3000.0, atol=1e-12)


def test_soft_partition_of_unity_and_symmetry():
    # sum_c u_c = 1, so over a window wide enough the soft f_i sum to one;
    # swapping the two snapshots mirrors the velocities.
    L = 48.0
    xp = 48.0 - 48.0 * np.random.default_rng(3).random((500, 2))
    xc = np.mod(xp + np.random.default_rng(4).normal(0, 1.5, xp.shape), L)
    xc[xc <= 0] = L
    f = cf.soft_fi(xc, xp, (L, L), 4.0, 2.0, 6)
    assert f.sum() == pytest.approx(1.0, abs=1e-9)
    g = cf.soft_fi(xp, xc, (L, L), 4.0, 2.0, 6)
    assert np.allclose(g.reshape(13, 13), f.reshape(13, 13)[::-1, ::-1], atol=1e-14)


def test_soft_of_static_particles_is_closed_form_at_width():
    # No displacement: for a point uniform in its cell, the soft kernel gives the
    # displacement law of a Gaussian of variance 2 s^2 convolved with the wedge,
    # i.e. the closed form of Eq. fialpha at a^2 = 2 s^2 / dx^2 (averaged over
    # many uniformly placed particles).
    rng = np.random.default_rng(5)
    L, dx, s = 400.0, 4.0, 0.5 * 4.0
    x = L - L * rng.random((40000, 2))
    f = cf.soft_fi(x, x, (L, L), dx, s, 3)
    ref = cf.feq_window(3, np.sqrt(2.0) * s / dx)[:49]
    assert np.allclose(f, ref, atol=5e-3)
