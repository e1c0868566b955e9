"""Checkpoint / resume: 1000 steps, save, 1000 more steps is bit-identical to
2000 steps, also when the checkpoint is loaded into another context created
with the same parameters (and a different initial state), for a single system
with every optional output on and for a batch."""
import numpy as np
import pytest

import mdlg_inputs as mi
import paper_1705_04368_gb300 as m

pytestmark = pytest.mark.gpu


def _record(s, xi=False):
    x, v = s.get_state()
    st, counts, fi = s.stats()
    out = {"x": x, "v": v, "counts": counts, "ke": st["kinetic"], "pe": st["potential"],
           "step": st["step"], "intervals": st["intervals"], "msd": np.array(st["msd"]),
           "vacf": np.array(st["vacf"])}
    if xi:
        out["xi"] = s.get_collision()[0]
        out["sites"] = s.get_sites()[0]
    return out


def _same(a, b, msd_exact=True):
    for k in a:
        if k in ("msd", "vacf") and not msd_exact:
            assert np.allclose(a[k], b[k], rtol=1e-12), k      # FP64 atomic sums
        elif isinstance(a[k], np.ndarray):
            assert np.array_equal(a[k], b[k]), k
        else:
            assert a[k] == b[k], k


def test_resume_single_system_bit_identical(cuda):
    n, L = 20000, mi.box_for(20000, 0.3, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=31)
    x1, v1 = mi.lj_initial_state(n, L, 1.0, seed=32)
    p = m.Params(n=n, box=L, dx=4.0, lag_steps=(3, 7, 50), sort_every=5, stats_every=10, msd=True,
                 vacf=True,
                 site_mode=m.SITES_FIELD | m.SITES_XI, lattice_u=(0.2, -0.1))
    with m.Simulation(p, x0, v0) as ref:
        ref.step(2000)
        want = _record(ref, xi=True)
    with m.Simulation(p, x0, v0) as a:
        a.step(1000)
        ck = a.save()
        a.step(1000)
        got_a = _record(a, xi=True)
    with m.Simulation(m.Params(**{**p.__dict__, "use_graphs": True}), x1, v1) as b:
        b.step(17)                       # some other history, then replaced
        b.load(ck)
        b.step(1000)
        got_b = _record(b, xi=True)
    _same(want, got_a, msd_exact=False)
    _same(want, got_b, msd_exact=False)


def test_resume_paced_schedule_bit_identical(cuda):
    # sort_every = 0: the device paces the re-sorts from the values of earlier
    # steps.  A checkpoint taken between re-sorts carries those values, so the
    # resumed run, in the same or in a fresh context, re-sorts at the same steps
    # and ends bit-identical to the uninterrupted one.
    n, L = 20000, mi.box_for(20000, 0.3, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=33)
    x1, v1 = mi.lj_initial_state(n, L, 1.0, seed=34)
    p = m.Params(n=n, box=L, dx=4.0, lag_steps=(10, 50), stats_every=100)
    with m.Simulation(p, x0, v0) as ref:
        ref.step(1000)
        want = _record(ref)
    with m.Simulation(p, x0, v0) as a:
        a.step(503)
        ck = a.save()
        a.step(497)
        got_a = _record(a)
    with m.Simulation(p, x1, v1) as b:
        b.step(11)                       # some other history, then replaced
        b.load(ck)
        b.step(497)
        got_b = _record(b)
    _same(want, got_a)
    _same(want, got_b)


def test_resume_batch_and_rejects_other_shapes(cuda):
    ns = [3000, 5000, 1200]
    boxes = [(mi.box_for(k, 0.3, 4.0),) * 2 for k in ns]
    xs, vs = zip(*[mi.lj_initial_state(k, b[0], 1.0, seed=40 + i) for i, (k, b) in enumerate(zip(ns, boxes))])
    x0, v0 = np.concatenate(xs), np.concatenate(vs)
    p = m.Params(n=0, box=64.0, dx=4.0, lag_steps=(10,), sort_every=7)
    with m.BatchSimulation(p, ns, boxes, x0, v0) as ref:
        ref.step(400)
        want = _record(ref)
    with m.BatchSimulation(p, ns, boxes, x0, v0) as a:
        a.step(150)
        ck = a.save()
    with m.BatchSimulation(p, ns, boxes, x0, v0) as b:
        b.load(ck)
        b.step(250)
        got = _record(b)
    _same(want, got)
    # a context of another shape refuses the checkpoint
    with m.BatchSimulation(p, ns[:2], boxes[:2], x0[:8000], v0[:8000]) as c:
        with pytest.raises(m.MdlgError):
            c.load(ck)
    with pytest.raises(m.MdlgError):
        with m.BatchSimulation(p, ns, boxes, x0, v0) as d:
            d.load(ck[:-8])


def test_resume_into_context_with_captured_graph(cuda):
    # the loading context has replayed graphs of its own schedule (sort every 5,
    # lag 10, statistics every 10: 20-step graphs); the load drops them, the
    # next steps capture new ones, and the result equals an uninterrupted run
    n, L = 8000, mi.box_for(8000, 0.3, 4.0)
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=51)
    p = m.Params(n=n, box=L, dx=4.0, lag_steps=(10,), sort_every=5, stats_every=10,
                 use_graphs=True)
    with m.Simulation(p, x0, v0) as ref:
        ref.step(333)
        want = _record(ref)
    with m.Simulation(p, x0, v0) as a:
        a.step(133)
        ck = a.save()
    with m.Simulation(p, x0, v0) as b:
        b.step(60)                      # captures and replays a graph
        b.load(ck)
        b.step(200)
        got = _record(b)
    _same(want, got)
