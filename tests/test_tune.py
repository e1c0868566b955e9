"""Autotuner host logic (no GPU): candidate filtering, choice, cache round trip."""
import json

import numpy as np

import paper_1705_04368_gb300 as m
from paper_1705_04368_gb300 import tune


def test_tuner_picks_fastest_and_caches(tmp_path):
    p = m.Params(n=4096, box=120.0, dx=4.0)
    calls = []

    def fake_timer(cand, x0, v0, steps, warmup):
        calls.append((cand.grid, cand.skin))
        if cand.skin == 1.0:
            raise RuntimeError("cannot build")
        return 1e-3 * (1.0 + abs(cand.skin - 0.75)) * (1.1 if cand.grid == 0.25 else 1.0)

    path = str(tmp_path / "tune.json")
    cands = ((0.5, 0.5), (0.5, 0.75), (0.5, 1.0), (0.25, 0.75))
    best, rep = tune.tune(p, None, None, 1.0, candidates=cands, timer=fake_timer, path=path)
    assert (best.grid, best.skin) == (0.5, 0.75) and not rep["cached"]
    assert any("error" in r for r in rep["candidates"])
    data = json.load(open(path))
    assert rep["key"] in data
    # second call: cached, no timing
    n_calls = len(calls)
    best2, rep2 = tune.tune(p, None, None, 1.0, candidates=cands, timer=fake_timer, path=path)
    assert rep2["cached"] and len(calls) == n_calls and best2.skin == 0.75


def test_tuner_skips_grids_that_do_not_divide(tmp_path):
    p = m.Params(n=100, box=10.0, dx=2.5)      # 0.5 divides 2.5 and 10; 0.3 does not
    seen = []

    def timer(cand, *a):
        seen.append(cand.grid)
        return 1.0

    best, rep = tune.tune(p, None, None, 1.0, candidates=((0.5, 0.5), (0.3, 0.5)), timer=timer,
                          path=str(tmp_path / "t.json"))
    assert seen == [0.5] and best.grid == 0.5
    assert "rho=1" in rep["key"] and "n=1e+02" in rep["key"]


def test_batch_tuning_keeps_sort_interval_and_checks_every_box(tmp_path):
    # the batch variant: candidates must divide every system's box, the caller's
    # re-sort interval is kept, and the cache key describes the ensemble
    ns = np.array([1000, 3000])
    boxes = np.array([[60.0, 60.0], [100.0, 100.0]])
    p = m.Params(n=0, box=64.0, dx=4.0, sort_every=7)
    seen = []

    def fake(cand, ns_, boxes_, x0, v0, steps, warmup):
        seen.append((cand.grid, cand.skin, cand.sort_every))
        return 1.0 + cand.skin

    orig = tune.time_batch_candidate
    tune.time_batch_candidate = fake
    try:
        best, rep = tune.tune_batch(p, ns, boxes, None, None, 1.0,
                                    candidates=((0.5, 0.5), (0.3, 0.25), (0.25, 0.75)),
                                    path=str(tmp_path / "b.json"))
    finally:
        tune.time_batch_candidate = orig
    assert [s[0] for s in seen] == [0.5, 0.25] and all(s[2] == 7 for s in seen)
    assert (best.grid, best.skin, best.sort_every) == (0.5, 0.5, 7)
    assert rep["key"].startswith("batch nsys=2 n=4e+03")


def test_default_candidates_are_valid_geometries_for_the_benchmark_boxes():
    # every default (grid, skin) gives an MD cell width (grid * ceil((rc + skin) /
    # grid), the list radius) from 2.75 to 4.0 sigma, on a power-of-two grid that
    # divides the lattice spacing dx = 4; the production boxes (L = 3740 at
    # rho = 0.3, 2644 at rho = 0.6) stay within 65535 base cells per axis on every
    # grid, so the library accepts each candidate there
    import math
    import mdlg_inputs as mi
    widths = []
    for g, sk in tune.DEFAULT_CANDIDATES:
        assert g > 0 and math.log2(g) == int(math.log2(g))
        assert (4.0 / g) == int(4.0 / g)
        w = g * math.ceil((2.5 + sk) / g - 1e-12)
        assert 2.75 - 1e-12 <= w <= 4.0 + 1e-12, (g, sk, w)
        widths.append(w)
        for c in (mi.PRODUCTION_LJ, mi.PRODUCTION_LJ_DENSE):
            assert c.box / g <= 65535 and (c.box / g) == int(c.box / g), (g, c.box)
    assert len(set(widths)) == len(widths)            # no two candidates alike
    assert {3.125, 3.25, 3.375} <= set(widths)        # the fine steps around the usual optimum
