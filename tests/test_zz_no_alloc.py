"""mdlg_forces_static: the entry point for callers that cannot allocate device
memory (inside a CUDA graph being captured, under a framework's own memory
pool, in loops that must not block in the allocator).  Its scratch lives in a
static device array of the library.  This test calls it through the C ABI twice
in a row on different systems (the truncated-shifted and the shifted-force
potential) and checks each result against the FP64 oracle (forces particle by
particle, kinetic and potential energy, virial, momentum) and against the
context path (mdlg_create + mdlg_get_state + mdlg_stats), within the force and
reduction tolerances of the other GPU tests.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import mdlg_inputs as mi
import oracle
import paper_1705_04368_gb300 as m
from paper_1705_04368_gb300 import binding as b

pytestmark = pytest.mark.gpu

Q = 2.0 ** -20   # positions exactly representable on both sides


def _context_result(params, x0, v0):
    with m.Simulation(params, x0, v0) as s:
        st0, _, _ = s.stats()
        _, _, f = s.get_state(want_force=True)
    return f, st0


def _static_result(cuda, params, x0, v0):
    import torch
    x = torch.from_numpy(x0).to(cuda)
    v = torch.from_numpy(v0).to(cuda)
    f = torch.full_like(x, float("nan"))
    obs = torch.full((5,), float("nan"), dtype=torch.float64, device=cuda)
    status = torch.full((1,), -99, dtype=torch.int32, device=cuda)
    cp = params.to_c()
    rc = m.lib().mdlg_forces_static(ctypes.byref(cp), x.data_ptr(), v.data_ptr(), f.data_ptr(),
                                    obs.data_ptr(), status.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    return f.cpu().numpy(), obs.cpu().numpy(), int(status.item())


@pytest.mark.parametrize("repeat", [0, 1])
def test_static_forces_match_oracle_and_context_two_calls(cuda, repeat):
    cases = [(5000, 0.3, 21, m.POT_LJ_TS), (3000, 0.6, 22, m.POT_LJ_SF)]
    for n, rho, seed, pot in cases:          # two calls in a row, different systems
        L = mi.box_for(n, rho, 4.0)
        x0, v0 = mi.lj_initial_state(n, L, 1.0, seed, quantum=Q)
        params = m.Params(n=n, box=L, dx=4.0, potential=pot)
        sf = pot == m.POT_LJ_SF
        f_st, obs, status = _static_result(cuda, params, x0, v0)
        assert status == 0
        # the FP64 oracle (direct O(N^2) sum): forces particle by particle
        f_ref, scale, pe, vir = oracle.lj_forces(x0, (L, L), shifted_force=sf)
        err = np.abs(f_st - f_ref).max(axis=1)
        assert np.all(err <= 1e-5 * np.maximum(scale, 1e-3)), float(err.max())
        ke = 0.5 * float((v0 * v0).sum())
        assert obs[0] == pytest.approx(ke, rel=1e-6)
        assert obs[1] == pytest.approx(pe, rel=1e-5, abs=1e-3)
        assert obs[2] == pytest.approx(vir, rel=1e-5, abs=1e-3)
        mom = v0.sum(axis=0)
        assert abs(obs[3] - mom[0]) < 1e-4 and abs(obs[4] - mom[1]) < 1e-4
        # and the context path on the same input
        f_ctx, st = _context_result(params, x0, v0)
        assert np.all(np.abs(f_st - f_ctx).max(axis=1) <= 1e-5 * np.maximum(scale, 1e-3))
        assert obs[0] == pytest.approx(st["kinetic"], rel=1e-6)
        assert obs[1] == pytest.approx(st["potential"], rel=1e-5, abs=1e-3)


def test_static_rejects_sizes_beyond_the_maximum(cuda):
    n = b.STATIC_MAX_N + 1
    params = m.Params(n=n, box=mi.box_for(n, 0.3, 4.0), dx=4.0).to_c()
    dummy = ctypes.c_void_p(1)
    rc = m.lib().mdlg_forces_static(ctypes.byref(params), dummy, dummy, dummy, dummy, None, None)
    assert rc == -4   # MDLG_EOVERFLOW, before any GPU work


def test_static_rejects_other_potentials(cuda):
    n = 1000
    params = m.Params(n=n, box=mi.box_for(n, 0.3, 4.0), dx=4.0, potential=m.POT_NONE).to_c()
    dummy = ctypes.c_void_p(1)
    rc = m.lib().mdlg_forces_static(ctypes.byref(params), dummy, dummy, dummy, dummy, None, None)
    assert rc == -1   # MDLG_EINVAL, before any GPU work
