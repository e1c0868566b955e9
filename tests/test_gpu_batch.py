"""GPU parity of batched systems (mdlg_create_batch): every system of a batch
evolves and is binned exactly as a context made for it alone."""
import numpy as np
import pytest

import mdlg_inputs as mi
import paper_1705_04368_gb300 as m

pytestmark = pytest.mark.gpu

# uneven sizes (none a multiple of the 128-slot chunk) and densities
SYSTEMS = [(1000, 0.3, 31), (3000, 0.6, 32), (700, 0.1, 33), (5000, 0.45, 34)]


def _states():
    xs, vs, ns, boxes = [], [], [], []
    for n, rho, seed in SYSTEMS:
        L = mi.box_for(n, rho, 4.0)
        x, v = mi.lj_initial_state(n, L, 1.0, seed)
        xs.append(x); vs.append(v); ns.append(n); boxes.append((L, L))
    return xs, vs, ns, boxes


def _params(**kw):
    base = dict(n=0, box=64.0, dx=4.0, lag_steps=(5, 12), sort_every=3, stats_every=20)
    base.update(kw)
    return m.Params(**base)


def test_batch_equals_each_system_alone(cuda):
    xs, vs, ns, boxes = _states()
    steps = 60
    with m.BatchSimulation(_params(), ns, boxes, np.concatenate(xs), np.concatenate(vs)) as bt:
        bt.step(steps)
        xb, vb = bt.get_state()
        per = [bt.stats_system(k) for k in range(len(ns))]
        agg, agg_counts, _ = bt.stats()
    off = 0
    tot_counts = np.zeros_like(agg_counts)
    for k, (n, box) in enumerate(zip(ns, boxes)):
        p = _params(n=n, box=box[0])
        with m.Simulation(p, xs[k], vs[k]) as s:
            s.step(steps)
            x1, v1 = s.get_state()
            st1, c1, f1 = s.stats()
        assert np.array_equal(xb[off:off + n], x1), k
        assert np.array_equal(vb[off:off + n], v1), k
        stb, cb, fb = per[k]
        assert np.array_equal(cb, c1), k
        assert np.array_equal(fb, f1), k
        for key in ("kinetic", "potential", "virial"):
            assert stb[key] == st1[key], (k, key)
        assert stb["momentum"] == st1["momentum"]
        tot_counts += c1
        off += n
    assert np.array_equal(agg_counts, tot_counts)
    assert agg["kinetic"] == pytest.approx(sum(d[0]["kinetic"] for d in per), rel=1e-12)
    assert agg["status"] == 0


def test_batch_of_one_equals_single(cuda):
    n, rho, seed = 4096, 0.3, 35
    L = mi.box_for(n, rho, 4.0)
    x, v = mi.lj_initial_state(n, L, 1.0, seed)
    with m.BatchSimulation(_params(), [n], [(L, L)], x, v) as bt:
        bt.step(25)
        xb, _ = bt.get_state()
        _, cb, _ = bt.stats()
    with m.Simulation(_params(n=n, box=L), x, v) as s:
        s.step(25)
        x1, _ = s.get_state()
        _, c1, _ = s.stats()
    assert np.array_equal(xb, x1) and np.array_equal(cb, c1)


def test_batch_paced_resorts_are_deterministic(cuda):
    # sort_every = 0 without graphs: the device paces the batch's re-sorts from
    # the largest displacement bound of all systems.  The lists stay current and
    # a second batch on the same input re-sorts at the same steps.
    xs, vs, ns, boxes = _states()
    p = _params(sort_every=0)
    runs = []
    for _ in range(2):
        with m.BatchSimulation(p, ns, boxes, np.concatenate(xs), np.concatenate(vs)) as bt:
            bt.profile(True)
            bt.step(300)
            sorts = bt.profile(False)["sort"][1]
            xb, vb = bt.get_state()
            st = bt.stats()[0]
        assert st["status"] == 0 and st["stale_steps"] == 0
        assert sorts > 0
        runs.append((sorts, xb, vb))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1]) and np.array_equal(runs[0][2], runs[1][2])


def test_batch_rejects_per_site_outputs_and_bad_boxes(cuda):
    xs, vs, ns, boxes = _states()
    with pytest.raises(m.MdlgError):
        m.BatchSimulation(_params(site_mode=m.SITES_FIELD), ns, boxes, np.concatenate(xs),
                          np.concatenate(vs))
    bad = list(boxes)
    bad[1] = (bad[1][0] + 1.0, bad[1][1])       # not a multiple of dx
    with pytest.raises(m.MdlgError):
        m.BatchSimulation(_params(), ns, bad, np.concatenate(xs), np.concatenate(vs))


# ---- every system of a batch against the FP64 oracle directly ------------------

import oracle  # noqa: E402

Q = 2.0 ** -20   # positions exactly representable on both sides


def test_batch_trajectories_match_oracle(cuda):
    # 10 steps of every system of an uneven batch (rho 0.1 ... 0.6, no N a multiple
    # of the 128-slot chunk) against oracle.VV: positions within 1e-4 sigma
    xs, vs, ns, boxes = [], [], [], []
    for n, rho, seed in SYSTEMS:
        L = mi.box_for(n, rho, 4.0)
        x, v = mi.lj_initial_state(n, L, 1.0, seed, quantum=Q)
        xs.append(x); vs.append(v); ns.append(n); boxes.append((L, L))
    with m.BatchSimulation(_params(), ns, boxes, np.concatenate(xs), np.concatenate(vs)) as bt:
        bt.step(10)
        xb, _ = bt.get_state()
        assert bt.stats()[0]["status"] == 0
    off = 0
    for k, (n, box) in enumerate(zip(ns, boxes)):
        ref = oracle.VV(xs[k], vs[k], box, 0.005, cells=True).run(10)
        d = xb[off:off + n] - ref.x
        d -= box[0] * np.round(d / box[0])
        assert np.abs(d).max() <= 1e-4, (k, float(np.abs(d).max()))
        off += n


def test_batch_free_flight_counts_bit_exact(cuda):
    # non-interacting systems on dyadic grids (every drift exact in binary32 and
    # FP64): each system's MDLG totals equal the oracle's binning of its own
    # exact trajectory
    rng = np.random.default_rng(41)
    sizes = [(1337, 64.0), (4099, 128.0), (513, 32.0)]
    dt, lags, steps = 0.125, (4, 7), 42
    xs, vs = [], []
    for n, L in sizes:
        xs.append(mi.dyadic_positions(n, L, seed=n, bits=12, boundary_frac=0.05))
        vs.append(np.round(rng.normal(0.0, 2.0, size=(n, 2)) * 1024) / 1024)
    p = _params(potential=m.POT_NONE, dt=dt, lag_steps=lags, sort_every=3)
    with m.BatchSimulation(p, [n for n, _ in sizes], [(L, L) for _, L in sizes],
                           np.concatenate(xs), np.concatenate(vs)) as bt:
        bt.step(steps)
        per = [bt.stats_system(k) for k in range(len(sizes))]
    for k, (n, L) in enumerate(sizes):
        traj = [xs[k]]
        for _ in range(steps):
            traj.append(oracle.free_stream(traj[-1], vs[k], (L, L), dt, 1))
        C = (int(L / 4.0),) * 2
        ref = np.zeros((len(lags), 50), np.uint64)
        for li, lag in enumerate(lags):
            for t in range(lag, steps + 1, lag):
                oracle.mdlg_bin(traj[t - lag], traj[t], 4.0, C, 3, counts=ref[li])
        assert np.array_equal(per[k][1], ref), k


def test_batch_ensemble_fi_matches_oracle(cuda):
    # Replicas of three small systems of the replica recipe (N 1000 ... 2000, rho 0.1
    # ... 0.6, T = 1, dx = 4, lag 50), 12 seeds each, all in one batch: per replica
    # configuration the seed-mean f_i of the batch and of the oracle agree within
    # 3 standard errors of their difference, bin by bin.
    configs = [(1000, 0.1), (1500, 0.35), (2000, 0.6)]
    seeds = range(12)
    steps, lag = 1000, 50
    xs, vs, ns, boxes, tags = [], [], [], [], []
    for ci, (n, rho) in enumerate(configs):
        L = mi.box_for(n, rho, 4.0)
        for sd in seeds:
            x, v = mi.lj_initial_state(n, L, 1.0, 5000 + 100 * ci + sd)
            xs.append(x); vs.append(v); ns.append(n); boxes.append((L, L)); tags.append(ci)
    p = _params(lag_steps=(lag,), sort_every=0, stats_every=0)
    with m.BatchSimulation(p, ns, boxes, np.concatenate(xs), np.concatenate(vs)) as bt:
        bt.step(steps)
        g_fi = [bt.stats_system(k)[2][0] for k in range(len(ns))]
    o_fi = []
    for k in range(len(ns)):
        L = boxes[k][0]
        ref = oracle.VV(xs[k], vs[k], (L, L), 0.005, cells=True)
        cnt = np.zeros(50, np.uint64)
        prev = ref.x.copy()
        for _ in range(steps // lag):
            ref.run(lag)
            oracle.mdlg_bin(prev, ref.x, 4.0, (int(L / 4.0),) * 2, 3, counts=cnt)
            prev = ref.x.copy()
        o_fi.append(cnt / (ns[k] * (steps // lag)))
    tags = np.array(tags)
    for ci in range(len(configs)):
        g = np.array([g_fi[k] for k in np.where(tags == ci)[0]])
        o = np.array([o_fi[k] for k in np.where(tags == ci)[0]])
        S = len(g)
        se = np.sqrt(g.var(axis=0, ddof=1) / S + o.var(axis=0, ddof=1) / S)
        d = np.abs(g.mean(axis=0) - o.mean(axis=0))
        live = (g.mean(axis=0) + o.mean(axis=0)) > 1e-4
        assert np.all(d[live] <= 3 * se[live] + 1e-12), (ci, d[live], se[live])
        assert np.all(d[~live] < 1e-4), ci
