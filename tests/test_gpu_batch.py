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


def test_batch_rejects_per_site_outputs_and_bad_boxes(cuda):
    xs, vs, ns, boxes = _states()
    with pytest.raises(m.MdlgError):
        m.BatchSimulation(_params(site_mode=m.SITES_FIELD), ns, boxes, np.concatenate(xs),
                          np.concatenate(vs))
    bad = list(boxes)
    bad[1] = (bad[1][0] + 1.0, bad[1][1])       # not a multiple of dx
    with pytest.raises(m.MdlgError):
        m.BatchSimulation(_params(), ns, bad, np.concatenate(xs), np.concatenate(vs))
