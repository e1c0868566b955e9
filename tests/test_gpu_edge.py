"""Degenerate and boundary cases of the MD path against the oracle: one
particle, one pair, the smallest periodic box (three neighbour cells per axis,
every neighbour cell a periodic image), a list that overflows its capacity
(cell-stencil fallback), lists exactly at their capacity, and the largest
velocity window."""
import numpy as np
import pytest

import mdlg_inputs as mi
import oracle
import paper_1705_04368_gb300 as m

pytestmark = pytest.mark.gpu

Q = 2.0 ** -20


def test_single_particle_free_flight(cuda):
    x0 = np.array([[3.0, 5.5]])
    v0 = np.array([[1.25, -0.5]])
    p = m.Params(n=1, box=16.0, dx=4.0, lag_steps=(4,), sort_every=3)
    with m.Simulation(p, x0, v0) as s:
        s.step(40)
        x, v, f = s.get_state(want_force=True)
        st, counts, _ = s.stats()
    assert np.array_equal(f, np.zeros((1, 2))) and np.array_equal(v, v0)
    ref = oracle.free_stream(x0, v0, (16.0, 16.0), 0.005, 40)
    assert np.abs(x - ref).max() < 1e-5
    assert int(counts[0].sum()) == 10 and st["status"] == 0


def test_one_pair_force(cuda):
    x0 = np.array([[2.0, 2.0], [3.25, 2.5]])
    v0 = np.zeros((2, 2))
    p = m.Params(n=2, box=16.0, dx=4.0)
    with m.Simulation(p, x0, v0) as s:
        _, _, f = s.get_state(want_force=True)
    f_ref, scale, _, _ = oracle.lj_forces(x0, (16.0, 16.0))
    assert np.abs(f - f_ref).max() <= 1e-5 * scale.max()
    assert np.abs(f.sum(axis=0)).max() < 1e-6          # Newton's third law


@pytest.mark.parametrize("box,n", [(10.0, 24), (12.0, 40)])
def test_smallest_periodic_box(cuda, box, n):
    # 3 neighbour cells per axis: every stencil wraps, pairs across every edge
    x0, v0 = mi.lj_initial_state(n, box, 1.0, seed=n, quantum=Q)
    p = m.Params(n=n, box=box, dx=2.0 if box == 10.0 else 4.0, skin=0.5, sort_every=2)
    with m.Simulation(p, x0, v0) as s:
        _, _, f = s.get_state(want_force=True)
        s.step(20)
        x, _ = s.get_state()
    f_ref, scale, _, _ = oracle.lj_forces(x0, (box, box))
    assert np.all(np.abs(f - f_ref).max(axis=1) <= 1e-5 * np.maximum(scale, 1e-3))
    ref = oracle.VV(x0, v0, (box, box), 0.005).run(20)
    d = x - ref.x
    d -= box * np.round(d / box)
    assert np.abs(d).max() < 1e-4


def test_dense_lists_overflow_to_cell_stencil(cuda):
    # a tight cluster: more neighbours than the list holds for some particles;
    # those take the cell-stencil path and still get the exact forces
    L = 128.0
    g = np.stack(np.meshgrid(np.arange(11), np.arange(11)), -1).reshape(-1, 2) * 0.85 + 40.0
    others, vo = mi.lj_initial_state(3000, L, 1.0, seed=6, quantum=Q)
    far = np.any((others < 38.0) | (others > 50.5), axis=1)
    x0 = np.round(np.concatenate([g, others[far][:2500]]) / Q) * Q
    n = x0.shape[0]
    v0 = np.concatenate([np.zeros((g.shape[0], 2)), vo[far][:2500]])
    p = m.Params(n=n, box=L, dx=4.0)
    with m.Simulation(p, x0, v0) as s:
        _, _, f = s.get_state(want_force=True)
        st, _, _ = s.stats()
    f_ref, scale, _, _ = oracle.lj_forces(x0, (L, L))
    assert np.all(np.abs(f - f_ref).max(axis=1) <= 1e-5 * np.maximum(scale, 1e-3))
    assert st["status"] == 0


def test_lists_at_and_around_capacity(cuda):
    # rectangular patches of spacings (0.80 + 0.02 k, 0.98 - 0.02 k) give list
    # lengths (pairs closer than the list radius, the MD cell width) on both
    # sides of the capacity, including lists exactly full: those are used, the
    # longer ones overflow to the cell stencil; every force matches the oracle
    L = 128.0
    pts = []
    for k in range(10):
        sp = np.array([0.80 + 0.02 * k, 0.98 - 0.02 * k])
        g = np.stack(np.meshgrid(np.arange(9), np.arange(9)), -1).reshape(-1, 2) * sp
        pts.append(g + np.array([4.0 + 12.0 * k, 20.0]))
    x0 = np.round(np.concatenate(pts) / Q) * Q
    n = x0.shape[0]
    p = m.Params(n=n, box=L, dx=4.0)
    rl = p.grid * np.ceil((p.rcut + p.skin) / p.grid)
    mean = n / (L * L) * np.pi * rl * rl
    cap = int(np.ceil((3.0 * mean + 16.0) / 4.0)) * 4
    d2 = ((x0[:, None, :] - x0[None, :, :]) ** 2).sum(-1)   # patches are far from the box edges
    np.fill_diagonal(d2, np.inf)
    assert np.abs(d2 - rl * rl).min() > 1e-3                 # no pair near the list radius
    counts = (d2 < rl * rl).sum(1)
    assert {cap - 1, cap, cap + 1} <= set(counts.tolist()), (cap, sorted(set(counts.tolist())))
    with m.Simulation(p, x0, np.zeros_like(x0)) as s:
        _, _, f = s.get_state(want_force=True)
        st, _, _ = s.stats()
    f_ref, scale, _, _ = oracle.lj_forces(x0, (L, L))
    assert np.all(np.abs(f - f_ref).max(axis=1) <= 1e-5 * np.maximum(scale, 1e-3))
    assert st["status"] == 0


@pytest.mark.parametrize("bad", ["nan_x", "zero_x", "outside_x", "inf_v"])
def test_invalid_initial_state_is_reported(cuda, bad):
    # the upload kernel flags the state (every index it derives is clamped) and
    # mdlg_create returns MDLG_ENONFINITE without a context
    n, L = 64, 32.0
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=9)
    if bad == "nan_x":
        x0[5, 0] = np.nan
    elif bad == "zero_x":
        x0[7, 1] = 0.0                      # the box is (0, L]
    elif bad == "outside_x":
        x0[3, 0] = L + 0.5
    else:
        v0[11, 1] = np.inf
    with pytest.raises(m.MdlgError) as e:
        m.Simulation(m.Params(n=n, box=L, dx=4.0), x0, v0)
    assert e.value.code == -5
