"""GPU parity of the Lennard-Jones velocity-Verlet MD and the fused MDLG binning
of the simulation state against the FP64 oracle.

Tolerances (FP32 pair arithmetic against FP64):
  forces      |F_gpu - F_ref| <= 1e-5 * sum_j (|F_rep,ij| + |F_att,ij|) per particle (the
              magnitudes of the repulsive and attractive terms), on positions
              exactly representable on both sides (multiples of 2^-20)
  trajectory  10 steps, every coordinate within 1e-4 sigma (minimum image)
  FP64 sums   kinetic energy rel 1e-6, potential energy and virial rel 1e-5
  counts      bit-exact on identical snapshots; ensemble f_i within 3 SE
"""
import math

import numpy as np
import pytest

import mdlg_inputs as mi
import oracle
import paper_1705_04368_gb300 as m

pytestmark = pytest.mark.gpu

# positions on multiples of 2^-20 are exact as cell origin + binary32 offset
Q = 2.0 ** -20


def _sim(n, L, x0, v0, **kw):
    p = m.Params(n=n, box=L, dx=kw.pop("dx", 4.0), **kw)
    return m.Simulation(p, x0, v0)


def _min_image(d, L):
    return d - L * np.round(d / L)


def _force_check(f_gpu, f_ref, scale, tol=1e-5, record=None):
    err = np.abs(f_gpu - f_ref).max(axis=1)
    bound = tol * np.maximum(scale, 1e-3)
    assert np.all(err <= bound), float((err / np.maximum(scale, 1e-3)).max())
    # the plain relative error |dF| / |F| per particle, beside the term-magnitude bar:
    # it is reported, and its 99th percentile must also stay within the tolerance
    # (single particles whose pair forces nearly cancel may exceed it)
    fn = np.linalg.norm(f_ref, axis=1)
    rel = np.linalg.norm(f_gpu - f_ref, axis=1)[fn > 0] / fn[fn > 0]
    stats = {"max": float(rel.max()), "p99": float(np.percentile(rel, 99)),
             "median": float(np.median(rel)), "term_bar_max": float((err / np.maximum(scale, 1e-3)).max())}
    print("force relative error |dF|/|F|:", stats)
    if record is not None:
        record("force_relative_error", stats)
    assert stats["p99"] <= tol, stats


@pytest.mark.parametrize("n,rho,seed", [(1024, 0.25, 1), (5000, 0.3, 2), (20000, 0.6, 3)])
def test_forces_match_direct_sum(cuda, n, rho, seed, record_property):
    L = mi.box_for(n, rho, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed, quantum=Q)
    with _sim(n, L, x0, v0) as s:
        x, _, f = s.get_state(want_force=True)
    assert np.array_equal(x, x0)          # identical positions on both sides
    f_ref, scale, _, _ = oracle.lj_forces(x0, (L, L))
    _force_check(f, f_ref, scale, record=record_property)


def test_forces_full_size_sampled(cuda, record_property):
    c = mi.PRODUCTION_LJ
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=1, quantum=Q)
    with _sim(c.n, c.box, x0, v0) as s:
        x, _, f = s.get_state(want_force=True)
    assert np.array_equal(x, x0)
    rng = np.random.default_rng(0)
    which = np.concatenate([rng.choice(c.n, 150, replace=False), [0, c.n - 1]])
    f_ref, scale = oracle.lj_forces_sample(x0, (c.box, c.box), which)
    _force_check(f[which], f_ref, scale, record=record_property)


def test_forces_full_size_after_resorts_bench_geometry(cuda, record_property):
    # The benchmark's configuration: N = 4 194 304, the tuned MD cells of 3.25
    # sigma (grid 0.25, skin 0.75), the device-paced re-sorts.  After 40 steps
    # (three or four re-sorts, each with a Verlet list built on cells ordered by
    # base column) the forces the engine evaluates from its current list match
    # the oracle's direct sums at the engine's own positions, on sampled particles.
    c = mi.PRODUCTION_LJ
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=3)
    p = m.Params(n=c.n, box=c.box, dx=c.dx, lag_steps=c.lags, stats_every=100, grid=0.25,
                 skin=0.75)
    with m.Simulation(p, x0, v0) as s:
        s.step(40)
        x, _, f = s.get_state(want_force=True)
        st, _, _ = s.stats()
    assert st["status"] == 0 and st["stale_steps"] == 0
    rng = np.random.default_rng(4)
    which = np.concatenate([rng.choice(c.n, 200, replace=False), [0, c.n - 1]])
    f_ref, scale = oracle.lj_forces_sample(x, (c.box, c.box), which)
    _force_check(f[which], f_ref, scale, record=record_property)


def test_tiled_system_past_2_25_slots_repeats_its_tile(cuda, record_property):
    # A periodic gas of n0 particles in a box L0 that holds a whole number of MD
    # cells (544 of 3.25 sigma) and of lattice cells (442 of 4 sigma), tiled 6 x 6:
    # 36 n0 = 33 758 892 > 2^25 particles, so the plain steps take the general
    # list-entry decode and every slot index of the sort, list and step kernels
    # runs past 2^25.  Positions on multiples of 2^-20 make every copy's cell
    # offsets identical, and particle numbers interleaved by copy (j * 36 + c)
    # order each cell's particles as in the tile, so the lists, the forces and the
    # device-paced re-sorts are the tile's: after 40 steps every copy equals the
    # tile bit for bit, the exact FP64 sums and the MDLG counts are 36 times the
    # tile's, and the forces match the oracle's direct sums on sampled particles.
    L0, T = 1768.0, 6
    n0 = int(round(0.3 * L0 * L0))
    x0, v0 = mi.lj_initial_state(n0, L0, 1.0, seed=11, quantum=Q)
    shifts = np.array([(a * L0, b * L0) for b in range(T) for a in range(T)])
    nc = len(shifts)
    X = (x0[:, None, :] + shifts[None, :, :]).reshape(-1, 2)    # particle j * 36 + c
    V = np.repeat(v0, nc, axis=0)
    assert X.shape[0] > (1 << 25)
    kw = dict(dx=4.0, lag_steps=(10, 20), stats_every=20, grid=0.25, skin=0.75)
    with m.Simulation(m.Params(n=n0, box=L0, **kw), x0, v0) as s:
        s.step(40)
        xs, vs, fs = s.get_state(want_force=True)
        sts, cs, _ = s.stats()
    with m.Simulation(m.Params(n=n0 * nc, box=L0 * T, **kw), X, V) as s:
        s.step(40)
        xb, vb, fb = s.get_state(want_force=True)
        stb, cb, _ = s.stats()
    for st in (sts, stb):
        assert st["status"] == 0 and st["stale_steps"] == 0 and st["step"] == 40
    assert stb["sort_every"] == sts["sort_every"] and stb["intervals"] == sts["intervals"]
    xb, vb, fb = (a.reshape(n0, nc, 2) for a in (xb, vb, fb))
    # positions: each copy is the tile moved by a whole number of tile widths (the
    # cell offsets are identical; the FP64 sum origin + offset that get_state forms
    # may round differently at the larger origins, by at most ~2^-40 here)
    d = xb - shifts[None, :, :] - xs[:, None, :]
    assert np.abs(d - np.round(d / L0) * L0).max() <= 1e-9
    assert np.array_equal(vb, np.broadcast_to(vs[:, None, :], vb.shape))
    assert np.array_equal(fb, np.broadcast_to(fs[:, None, :], fb.shape))
    for k in ("kinetic", "potential", "virial"):
        assert stb[k] == nc * sts[k], k
    assert np.array_equal(cb, cs * np.uint64(nc))
    rng = np.random.default_rng(12)
    which = rng.choice(n0 * nc, 200, replace=False)    # as many as the other full-size cases
    f_ref, scale = oracle.lj_forces_sample(xb.reshape(-1, 2), (L0 * T, L0 * T), which)
    _force_check(fb.reshape(-1, 2)[which], f_ref, scale, record=record_property)


@pytest.mark.parametrize("n,rho,sort_every", [(4096, 0.3, 0), (4096, 0.3, 1), (30000, 0.6, 3),
                                               (4096, 0.3, 1000)])
def test_ten_step_trajectory(cuda, n, rho, sort_every):
    # sort_every = 1000: the Verlet list goes stale mid-run and the step kernel
    # switches to the cell stencil of the current displacement bound
    L = mi.box_for(n, rho, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=n)
    ref = oracle.VV(x0, v0, (L, L), dt=0.005).run(10)
    with _sim(n, L, x0, v0, sort_every=sort_every) as s:
        s.step(10)
        x, v = s.get_state()
        st, _, _ = s.stats()
    assert np.abs(_min_image(x - ref.x, L)).max() <= 1e-4
    assert np.abs(v - ref.v).max() <= 1e-3
    assert st["status"] == 0 and st["step"] == 10


def test_late_resort_uses_wider_stencil(cuda):
    # 60 steps without a re-sort: the displacement bound grows past the skin,
    # so forces come from the cell stencil (radius 2 once 2D > skin); the
    # trajectory still follows the FP64 oracle.
    n, L = 4096, mi.box_for(4096, 0.3, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=77)
    ref = oracle.VV(x0, v0, (L, L), dt=0.005).run(60)
    with _sim(n, L, x0, v0, sort_every=100000) as s:
        s.step(60)
        x, _ = s.get_state()
        st, _, _ = s.stats()
    assert np.abs(_min_image(x - ref.x, L)).max() <= 1e-3
    assert st["status"] == 0


def test_device_paced_resort_schedule(cuda):
    # sort_every = 0 without graphs: the device paces the re-sorts.  Until 3
    # steps after the upload the interval rule of the fastest initial speed
    # (half the skin at 1.15 vmax0) applies, so no re-sort comes in the first
    # 3 steps; afterwards a step re-sorts only when the displacement bound of
    # its input would pass half the skin.  Over 400 steps: the list never goes
    # stale, the intervals are no shorter than ~0.8x the fixed rule's (the
    # fastest speed of a step stays near the initial one at T = 1), and a
    # second context on the same input re-sorts at the same steps (identical
    # positions and launch counts).
    n, L = 4096, mi.box_for(4096, 0.3, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=78)
    p = m.Params(n=n, box=L, dx=4.0, lag_steps=(5,))
    k = math.ceil((p.rcut + p.skin) / p.grid - 1e-12)
    skin_eff = k * p.grid - p.rcut
    vmax0 = math.sqrt(float((v0 * v0).sum(axis=1).max()))
    every = int(max(1.0, min(math.floor(0.5 * skin_eff / (1.15 * vmax0 * p.dt)), 1000.0)))
    assert 4 <= every <= 50
    runs = []
    for _ in range(2):
        with m.Simulation(p, x0, v0) as s:
            s.profile(True)
            s.step(3)
            assert s.profile(False)["sort"][1] == 0
            s.profile(True)
            s.step(397)
            sorts = s.profile(False)["sort"][1]
            assert sorts % 7 == 0             # 7 launches per re-sort
            x, _ = s.get_state()
            st, _, _ = s.stats()
        assert st["status"] == 0 and st["stale_steps"] == 0
        assert 1 <= sorts // 7 <= 400 / (0.8 * every) + 1, (sorts // 7, every)
        assert st["sort_every"] >= 0.8 * every
        runs.append((sorts, x))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])


def test_paced_schedule_recovers_after_a_hot_start(cuda):
    # One particle launched at 12 sigma/tau into a T = 1 gas with a small skin
    # (cells of 2.75 sigma): the first interval from the fastest uploaded speed is
    # a single step.  Once that particle has shared its energy (a few hundred
    # steps), the re-sorts must come every few steps again, predicted from the
    # device's speeds even in the first steps after each re-sort, and not stay at
    # the first interval's length.
    n, L = 4096, mi.box_for(4096, 0.3, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=79)
    v0 = v0.copy()
    v0[0] = (12.0, 0.0)
    p = m.Params(n=n, box=L, dx=4.0, lag_steps=(5,), grid=0.25, skin=0.25)
    k = math.ceil((p.rcut + p.skin) / p.grid - 1e-12)
    skin_eff = k * p.grid - p.rcut
    assert math.floor(0.5 * skin_eff / (1.15 * 12.0 * p.dt)) <= 1
    runs = []
    for _ in range(2):
        with m.Simulation(p, x0, v0) as s:
            s.step(400)
            s.profile(True)
            s.step(100)
            sorts = s.profile(False)["sort"][1] // 7
            x, _ = s.get_state()
            st, _, _ = s.stats()
        assert st["status"] == 0
        assert st["stale_steps"] <= 10, st["stale_steps"]
        assert 1 <= sorts <= 50, sorts          # intervals of two steps or more
        runs.append((sorts, x))
    assert runs[0][0] == runs[1][0] and np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("rho,T,steps,max_stale_frac", [(0.3, 1.0, 600, 0.0), (0.6, 0.8, 600, 0.01)])
def test_adaptive_resort_keeps_the_list_current(cuda, rho, T, steps, max_stale_frac):
    # A gas placed at random heats up as it relaxes (at rho = 0.6, T = 0.8 the
    # fastest speed grows by 30-50 %): a schedule fixed from the initial speeds
    # lets the Verlet list go stale (every such step takes the slower cell
    # stencil); the device-paced schedule keeps up, and the trajectory still
    # conserves momentum exactly and energy to the FP32 bound.
    n = 65536
    L = mi.box_for(n, rho, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, T, seed=91)
    with _sim(n, L, x0, v0) as s:
        st0, _, _ = s.stats()
        s.step(steps)
        st, _, _ = s.stats()
    assert st["status"] == 0
    assert st["stale_steps"] <= max_stale_frac * steps, st["stale_steps"]
    e0 = st0["kinetic"] + st0["potential"]
    e1 = st["kinetic"] + st["potential"]
    assert abs(e1 - e0) / n < 4e-3
    assert abs(st["momentum"][0]) / n < 1e-5 and abs(st["momentum"][1]) / n < 1e-5


def test_fp64_reductions_at_start(cuda):
    n, L = 8192, mi.box_for(8192, 0.3, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=11)
    with _sim(n, L, x0, v0) as s:
        st, _, _ = s.stats()
    _, _, pe, vir = oracle.lj_forces(x0, (L, L), cells=True)
    ke, px, py = oracle.VV(x0, v0, (L, L), 0.005).kinetic()
    assert st["kinetic"] == pytest.approx(ke, rel=1e-6)
    assert st["potential"] == pytest.approx(pe, rel=1e-5, abs=1e-3)
    assert st["virial"] == pytest.approx(vir, rel=1e-5, abs=1e-3)
    assert abs(st["momentum"][0] - px) < 1e-4 and abs(st["momentum"][1] - py) < 1e-4
    assert st["temperature"] == pytest.approx(1.0, rel=1e-6)


def test_conservation_long_run(cuda):
    # 1000 steps of a 65 536-particle gas: energy per particle and total momentum
    # stay put (truncated force and FP32 pair sums bound the drift).
    n, L = 65536, mi.box_for(65536, 0.3, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=12)
    with _sim(n, L, x0, v0, stats_every=100) as s:
        st0, _, _ = s.stats()
        s.step(1000)
        st1, _, _ = s.stats()
    e0 = st0["kinetic"] + st0["potential"]
    e1 = st1["kinetic"] + st1["potential"]
    assert abs(e1 - e0) / n < 2e-3
    assert abs(st1["momentum"][0]) / n < 1e-5 and abs(st1["momentum"][1]) / n < 1e-5
    assert st1["status"] == 0


def _dyadic_free_flight(n, L, seed):
    # Positions on a 2^-12 grid and velocities on a 2^-10 grid with dt = 2^-3:
    # every drift x + v dt is exact in binary32 offsets and in FP64, so the
    # library's state and the oracle's trajectory are identical snapshots.
    rng = np.random.default_rng(seed)
    x = mi.dyadic_positions(n, L, seed, bits=12, boundary_frac=0.05)
    v = np.round(rng.normal(0.0, 2.0, size=(n, 2)) * 1024) / 1024
    return x, v


@pytest.mark.parametrize("n,L,lags,sort_every,steps", [
    (5000, 64.0, (4, 7), 3, 60),
    (70000, 256.0, (1, 5, 16), 2, 48),
    # a ragged tail (n mod 4 = 3) and launches that bin 1 ... 8 lags at once
    (5003, 64.0, (1, 2, 3, 4, 6, 8, 12, 24), 5, 48),
])
def test_fused_state_binning_bit_exact(cuda, n, L, lags, sort_every, steps):
    x0, v0 = _dyadic_free_flight(n, L, seed=n)
    dt = 0.125
    vmax = 3
    with _sim(n, L, x0, v0, potential=m.POT_NONE, dt=dt, lag_steps=lags, sort_every=sort_every,
              vmax=vmax, site_mode=m.SITES_ACCUM) as s:
        s.step(steps)
        st, counts, fi = s.stats()
        sites, ncell = s.get_sites()
        x_end, _ = s.get_state()
    C = (int(L / 4.0),) * 2
    q1 = (2 * vmax + 1) ** 2 + 1
    ref = np.zeros((len(lags), q1), np.uint64)
    ref_sites = np.zeros((C[0] * C[1], q1), np.uint32)
    ref_n = np.zeros(C[0] * C[1], np.uint32)
    traj = [x0]
    xx = x0
    for _ in range(steps):
        xx = oracle.free_stream(xx, v0, (L, L), dt, 1)
        traj.append(xx)
    for li, lag in enumerate(lags):
        for t in range(lag, steps + 1, lag):
            oracle.mdlg_bin(traj[t - lag], traj[t], 4.0, C, vmax, counts=ref[li],
                            field=(li == 0), ncell=ref_n if li == 0 else None,
                            fld=ref_sites if li == 0 else None)
    assert np.array_equal(x_end, traj[-1])
    assert np.array_equal(counts, ref)
    assert np.array_equal(sites, ref_sites)
    assert np.array_equal(ncell, ref_n)
    for li, lag in enumerate(lags):
        assert st["intervals"][li] == steps // lag
        assert fi[li].sum() == pytest.approx(1.0)


def test_ensemble_fi_matches_oracle(cuda):
    # Small LJ gas (N = 1024, L = 64, dx = 4, lag 50 steps, 2000 steps): the
    # per-seed f_i of the library and of the oracle agree within 3 standard
    # errors of the difference of their seed means, bin by bin.
    c = mi.SMALL_LJ
    seeds = range(1, 17)
    g_runs, o_runs = [], []
    for seed in seeds:
        x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed)
        with _sim(c.n, c.box, x0, v0, lag_steps=c.lags) as s:
            s.step(c.steps)
            _, _, fi = s.stats()
        g_runs.append(fi[0])
        ref = oracle.VV(x0, v0, (c.box, c.box), c.dt, cells=True)
        cnt = np.zeros(50, np.uint64)
        prev = ref.x.copy()
        for _ in range(c.steps // c.lags[0]):
            ref.run(c.lags[0])
            oracle.mdlg_bin(prev, ref.x, c.dx, (16, 16), 3, counts=cnt)
            prev = ref.x.copy()
        o_runs.append(cnt / (c.n * (c.steps // c.lags[0])))
    g, o = np.array(g_runs), np.array(o_runs)
    S = len(seeds)
    se = np.sqrt(g.var(axis=0, ddof=1) / S + o.var(axis=0, ddof=1) / S)
    d = np.abs(g.mean(axis=0) - o.mean(axis=0))
    live = (g.mean(axis=0) + o.mean(axis=0)) > 1e-4
    assert np.all(d[live] <= 3 * se[live] + 1e-12), (d[live], se[live])
    assert np.all(d[~live] < 1e-4)


def test_production_run_invariants(cuda):
    # 4 194 304 particles, rho = 0.3: 200 steps with lags 10, 20, 50, 100, 200.
    c = mi.PRODUCTION_LJ
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=2)
    with _sim(c.n, c.box, x0, v0, lag_steps=c.lags, stats_every=100,
              site_mode=m.SITES_FIELD) as s:
        st0, _, _ = s.stats()
        s.step(200)
        st, counts, fi = s.stats()
        sites, ncell = s.get_sites()
    assert st["status"] == 0
    for li, lag in enumerate(c.lags):
        assert int(counts[li].sum()) == c.n * (200 // lag)
    assert np.array_equal(sites.sum(axis=1, dtype=np.int64), ncell.astype(np.int64))
    assert int(ncell.sum()) == c.n
    e0, e1 = st0["kinetic"] + st0["potential"], st["kinetic"] + st["potential"]
    assert abs(e1 - e0) / c.n < 1e-3
    assert abs(st["momentum"][0]) / c.n < 1e-5


@pytest.mark.parametrize("batched", [False, True])
def test_graph_replay_equals_direct_launches(cuda, batched):
    # use_graphs: two periods of the schedule (sort every 5, lag 50 -> 100 steps)
    # are captured once and replayed; results equal direct launches bit for bit.
    import torch
    c = mi.SMALL_LJ
    x0, v0 = mi.lj_initial_state(c.n, c.box, c.temperature, seed=5)
    out = []
    for graphs in (False, True):
        p = m.Params(n=c.n, box=c.box, dx=c.dx, lag_steps=(50,), sort_every=5, stats_every=25,
                     use_graphs=graphs)
        stream = torch.cuda.Stream()
        if batched:
            sim = m.BatchSimulation(p, [c.n, c.n], [(c.box, c.box)] * 2, np.concatenate([x0, x0]),
                                    np.concatenate([v0, v0]), stream=stream)
        else:
            sim = m.Simulation(p, x0, v0, stream=stream)
        with sim:
            sim.profile(True)
            sim.step(250)      # graph: capture steps 0-99, replay 100-199, direct 200-249
            sim.step(37)       # not aligned with the graph: direct launches
            prof = sim.profile(False)
            x, v = sim.get_state()
            st, counts, _ = sim.stats()
        out.append((x, v, counts, st, prof))
    (x1, v1, c1, s1, p1), (x2, v2, c2, s2, p2) = out
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2) and np.array_equal(c1, c2)
    assert s1["kinetic"] == s2["kinetic"] and s1["intervals"] == s2["intervals"]
    assert p1["step"][1] == p2["step"][1] and p1["sort"][1] == p2["sort"][1]


def test_tuner_times_candidates_on_gpu(cuda, tmp_path):
    from paper_1705_04368_gb300 import tune
    n, L = 4096, mi.box_for(4096, 0.3, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=41)
    p = m.Params(n=n, box=L, dx=4.0)
    best, rep = tune.tune(p, x0, v0, 1.0, candidates=((0.5, 0.5), (0.25, 0.75)), steps=20,
                          warmup=4, path=str(tmp_path / "t.json"))
    assert {r["skin"] for r in rep["candidates"]} == {0.5, 0.75}
    assert all(r["sec_per_step"] > 0 for r in rep["candidates"])
    assert best.skin in (0.5, 0.75)
