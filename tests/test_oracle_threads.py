"""The threaded build of the oracle (the benchmark's all-core CPU baseline) gives
the serial build's results: the same force on every particle (each particle's
sum keeps its order), the same integer histograms, and energies equal to
rounding.  The threaded build runs in a child process, because one process
loads one build."""
import json
import os
import subprocess
import sys

import numpy as np

import mdlg_inputs as mi
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import mdlg_inputs as mi, oracle
t = oracle.use_threads(4)
x, v = mi.lj_initial_state(3000, 100.0, 1.0, seed=3)
f, fs, pe, vir = oracle.lj_forces(x, (100.0, 100.0), cells=True)
ref = oracle.VV(x, v, (100.0, 100.0), 0.005, cells=True).run(5)
cnt, _, _, vs = oracle.mdlg_bin(x, ref.x, 4.0, (25, 25), 3)
pos, vel = mi.idealgas_state(20001, 64.0, 1.0, seed=4)
ig = oracle.stream_bin_f32(pos, vel, [1.0, 2.0], [0.5, 2.0], 3)
np.save(sys.argv[2], np.concatenate([f.ravel(), ref.x.ravel(), ref.v.ravel()]))
print(json.dumps({"threads": t, "pe": pe, "vir": vir, "cnt": cnt.tolist(), "vs": vs.tolist(),
                  "ig": ig.ravel().tolist(), "pe_end": ref.pe}))
"""


def test_threaded_build_matches_serial(tmp_path):
    out = tmp_path / "f.npy"
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT, str(out)], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    got = json.loads(r.stdout.strip().splitlines()[-1])
    assert got["threads"] == 4
    x, v = mi.lj_initial_state(3000, 100.0, 1.0, seed=3)
    f, fs, pe, vir = oracle.lj_forces(x, (100.0, 100.0), cells=True)
    ref = oracle.VV(x, v, (100.0, 100.0), 0.005, cells=True).run(5)
    cnt, _, _, vs = oracle.mdlg_bin(x, ref.x, 4.0, (25, 25), 3)
    pos, vel = mi.idealgas_state(20001, 64.0, 1.0, seed=4)
    ig = oracle.stream_bin_f32(pos, vel, [1.0, 2.0], [0.5, 2.0], 3)
    arr = np.load(out)
    assert np.array_equal(arr, np.concatenate([f.ravel(), ref.x.ravel(), ref.v.ravel()]))
    assert got["cnt"] == cnt.tolist() and got["vs"] == vs.tolist()
    assert got["ig"] == ig.ravel().tolist()
    assert abs(got["pe"] - pe) <= 1e-12 * abs(pe) and abs(got["vir"] - vir) <= 1e-12 * abs(vir)
    assert abs(got["pe_end"] - ref.pe) <= 1e-12 * abs(ref.pe)
