"""The oracle's C code under the undefined-behaviour and address sanitizers:
a build with -fsanitize=undefined,address (UBSan linked statically, aborting on
the first report; ASan through its preloaded runtime) runs every entry point on
small inputs in a subprocess, including boundary points, overflow moves and
periodic wrapping."""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mdlg_oracle.c")

DRIVER = textwrap.dedent("""
    import numpy as np, sys
    sys.path.insert(0, %r)
    import mdlg_inputs as mi, oracle
    from oracle import closed_form as cf
    L = 24.0
    x0, v0 = mi.lj_initial_state(60, L, 1.0, seed=3)
    f, s, pe, vir = oracle.lj_forces(x0, (L, L))
    f2, s2, _, _ = oracle.lj_forces(x0, (L, L), cells=True)
    oracle.lj_forces_sample(x0, (L, L), np.array([0, 59]))
    for sf in (False, True):
        oracle.VV(x0, v0, (L, L), 0.005, cells=True, shifted_force=sf).run(5)
    oracle.free_stream(x0, v0, (L, L), 0.5, 3)
    xp = mi.dyadic_positions(200, L, seed=1, bits=4, boundary_frac=0.3)
    xc = mi.displaced(xp, L, seed=2, scale=9.0, bits=4, boundary_frac=0.3)
    c, n, fld, vs = oracle.mdlg_bin(xp, xc, 2.0, (12, 12), 2, field=True,
                                    shift_prev=(-30.5, 7.25), shift_cur=(1e3, -2e3))
    oracle.collision((12, 12), 2, fld, fld)
    oracle.collision((1, 1), 3, np.ones((1, 50), np.uint32), np.zeros((1, 50), np.uint32))
    oracle.msd(xp, xc, (L, L))
    pos, vel = mi.idealgas_state(500, 16.0, 1.0, seed=4)
    oracle.stream_bin_f32(pos, vel, [1.0, 3.0], [0.5, 2.0], 3, us=[[0.1, 0.0], [0.0, -0.2]])
    print("ok")
""") % ROOT


def _runtime(name):
    out = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True)
    path = out.stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_oracle_under_sanitizers(tmp_path):
    lib = str(tmp_path / "liboracle_san.so")
    asan = _runtime("libasan.so")
    flags = ["-fsanitize=undefined", "-fno-sanitize-recover=all", "-static-libubsan"]
    if asan:
        flags = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-static-libubsan"]
    r = subprocess.run(["gcc", "-O1", "-g", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                        *flags, SRC, "-o", lib, "-lm"], capture_output=True, text=True)
    if r.returncode != 0 and asan:        # toolchain without a usable ASan: UBSan alone
        asan = None
        flags = ["-fsanitize=undefined", "-fno-sanitize-recover=all", "-static-libubsan"]
        r = subprocess.run(["gcc", "-O1", "-g", "-std=c11", "-ffp-contract=off", "-fPIC",
                            "-shared", *flags, SRC, "-o", lib, "-lm"], capture_output=True,
                           text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ORACLE_LIB=lib, UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    if asan:
        env["LD_PRELOAD"] = asan
        env["ASAN_OPTIONS"] = "detect_leaks=0:halt_on_error=1"
    p = subprocess.run([sys.executable, "-c", DRIVER], env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0 and p.stdout.strip().endswith("ok"), p.stderr[-3000:]
