"""GPU adjoint (mdlg_adjoint) of soft-binned MDLG occupations, checked against
the FP64 oracle: exact in free flight, central finite differences of the FP64
trajectory for the Lennard-Jones gas, and the torch.autograd wrapper."""
import math

import numpy as np
import pytest

import mdlg_inputs as mi
import oracle
from oracle import closed_form as cf
import paper_1705_04368_gb300 as m

pytestmark = pytest.mark.gpu

V = 3
W = 2 * V + 1
VEL = oracle.velocity_table(V)
M2 = (VEL ** 2).sum(axis=1).astype(np.float64)      # weights of the second moment


def _free_flight_case(n=3000, L=64.0, seed=7):
    rng = np.random.default_rng(seed)
    x = mi.dyadic_positions(n, L, seed, bits=12, boundary_frac=0.0)
    v = np.round(rng.normal(0.0, 2.0, size=(n, 2)) * 1024) / 1024
    return x, v


def test_free_flight_soft_values_and_gradients_exact(cuda):
    # No forces: x_K = x_0 + K dt v_0 exactly on both sides, so ftilde matches the
    # oracle to rounding and the gradients follow from the loss alone.
    n, L, dx, dt, K, width = 3000, 64.0, 4.0, 0.125, 8, 2.0
    x0, v0 = _free_flight_case(n, L)
    p = m.Params(n=n, box=L, dx=dx, dt=dt, potential=m.POT_NONE, sort_every=4, vmax=V)
    with m.Simulation(p, x0, v0) as s:
        out = s.adjoint(K, 4, width, dloss=M2)
    xK = oracle.free_stream(x0, v0, (L, L), dt, K)
    ref = cf.soft_fi(xK, x0, (L, L), dx, width, V)
    assert np.allclose(out["ftilde"], ref, atol=1e-12, rtol=1e-10)
    assert out["loss"] == pytest.approx(float(M2 @ ref), rel=1e-10)
    assert out["grad_eps"] == 0.0 and out["grad_sigma"] == 0.0

    def loss(xs, vs):
        return float(M2 @ cf.soft_fi(oracle.free_stream(xs, vs, (L, L), dt, K), xs, (L, L), dx,
                                     width, V))

    rng = np.random.default_rng(1)
    for which in ("x", "v"):
        u = rng.normal(size=(n, 2))
        u /= np.linalg.norm(u)
        h = 1e-4
        if which == "x":
            fd = (loss(x0 + h * u, v0) - loss(x0 - h * u, v0)) / (2 * h)
            got = float((out["grad_x0"] * u).sum())
        else:
            fd = (loss(x0, v0 + h * u) - loss(x0, v0 - h * u)) / (2 * h)
            got = float((out["grad_v0"] * u).sum())
        assert got == pytest.approx(fd, rel=2e-4, abs=1e-9), which


def _lj_loss(x0, v0, L, eps, sigma, K, dx, width, sf=False):
    s = oracle.VV(x0, v0, (L, L), dt=0.005, eps=eps, sigma=sigma, cells=True, shifted_force=sf)
    s.run(K)
    return float(M2 @ cf.soft_fi(s.x, x0, (L, L), dx, width, V))


# (n, rho, K, checkpoint interval, shifted force, check eps/sigma)
LJ_CASES = [
    (2048, 0.3, 40, 20, False, True),
    (2048, 0.3, 100, 20, True, True),
    (16384, 0.3, 200, 20, True, True),      # the adjoint workload, continuous forces
    (16384, 0.3, 200, 20, False, False),    # the same with the force truncated at rc
]


@pytest.mark.parametrize("n,rho,K,ckpt,sf,params", LJ_CASES,
                         ids=[f"n{c[0]}_K{c[2]}_{'sf' if c[4] else 'ts'}" for c in LJ_CASES])
def test_lj_gradients_match_fp64_finite_differences(cuda, n, rho, K, ckpt, sf, params):
    # Central differences of the FP64 oracle trajectory, steps of 1e-6.  With the
    # force truncated at rc (ts) the discrete trajectory jumps wherever a pair
    # crosses rc at a step; perturbing eps or sigma moves every pair, and the
    # jumps then enter any difference quotient however small the step, so the
    # eps/sigma check for ts uses a short horizon; the continuous shifted force
    # (sf) is checked at the full 200 steps.
    L = mi.box_for(n, rho, 4.0)
    dx, width = 4.0, 2.0
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=n + 3)
    p = m.Params(n=n, box=L, dx=dx, sort_every=ckpt, vmax=V,
                 potential=m.POT_LJ_SF if sf else m.POT_LJ_TS)
    with m.Simulation(p, x0, v0) as s:
        out = s.adjoint(K, ckpt, width, dloss=M2)
    L0 = _lj_loss(x0, v0, L, 1.0, 1.0, K, dx, width, sf)
    assert out["loss"] == pytest.approx(L0, rel=2e-4)
    h = 1e-6
    if params:
        fd_eps = (_lj_loss(x0, v0, L, 1 + h, 1.0, K, dx, width, sf)
                  - _lj_loss(x0, v0, L, 1 - h, 1.0, K, dx, width, sf)) / (2 * h)
        fd_sig = (_lj_loss(x0, v0, L, 1.0, 1 + h, K, dx, width, sf)
                  - _lj_loss(x0, v0, L, 1.0, 1 - h, K, dx, width, sf)) / (2 * h)
        assert out["grad_eps"] == pytest.approx(fd_eps, rel=2e-3, abs=1e-8)
        assert out["grad_sigma"] == pytest.approx(fd_sig, rel=2e-3, abs=1e-8)
    rng = np.random.default_rng(2)
    for which in ("x", "v"):
        u = rng.normal(size=(n, 2))
        u /= np.linalg.norm(u)
        if which == "x":
            lp = _lj_loss(x0 + h * u, v0, L, 1.0, 1.0, K, dx, width, sf)
            lm = _lj_loss(x0 - h * u, v0, L, 1.0, 1.0, K, dx, width, sf)
            got = float((out["grad_x0"] * u).sum())
        else:
            lp = _lj_loss(x0, v0 + h * u, L, 1.0, 1.0, K, dx, width, sf)
            lm = _lj_loss(x0, v0 - h * u, L, 1.0, 1.0, K, dx, width, sf)
            got = float((out["grad_v0"] * u).sum())
        fd = (lp - lm) / (2 * h)
        assert got == pytest.approx(fd, rel=2e-3, abs=1e-9), which


def test_autograd_wrapper_matches_entry_point(cuda):
    import torch
    from paper_1705_04368_gb300.autograd import soft_mdlg
    n, rho = 1024, 0.25
    L = 64.0
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=99)
    p = m.Params(n=n, box=L, dx=4.0, vmax=V)
    xt = torch.tensor(x0, requires_grad=True)
    vt = torch.tensor(v0, requires_grad=True)
    et = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    st = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    ft = soft_mdlg(xt, vt, et, st, p, 60, 20, 2.0)
    loss = (torch.from_numpy(M2) * ft).sum()
    loss.backward()
    with m.Simulation(m.Params(n=n, box=L, dx=4.0, vmax=V, sort_every=20), x0, v0) as s:
        ref = s.adjoint(60, 20, 2.0, dloss=M2)
    # soft values and parameter adjoints are FP64 atomic sums (last-bit order
    # effects); the per-particle gradients are deterministic
    assert np.allclose(ft.detach().numpy(), ref["ftilde"], rtol=1e-12, atol=0)
    assert np.array_equal(xt.grad.numpy(), ref["grad_x0"])
    assert np.array_equal(vt.grad.numpy(), ref["grad_v0"])
    assert et.grad.item() == pytest.approx(ref["grad_eps"], rel=1e-12)
    assert st.grad.item() == pytest.approx(ref["grad_sigma"], rel=1e-12)


def test_adjoint_preconditions(cuda):
    n, L = 1024, 64.0
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=98)
    with m.Simulation(m.Params(n=n, box=L, dx=4.0, sort_every=10), x0, v0) as s:
        with pytest.raises(m.MdlgError):
            s.adjoint(30, 20, 2.0)          # checkpoint interval != sort interval
        with pytest.raises(m.MdlgError):
            s.adjoint(25, 10, 2.0)          # not a whole number of segments
        with pytest.raises(m.MdlgError):
            s.adjoint(20, 10, 5.0)          # width above 0.875 dx
        s.adjoint(20, 10, 2.0)              # fine: forward only
        s.step(3)
        with pytest.raises(m.MdlgError):
            s.adjoint(20, 10, 2.0)          # not at a re-sort


def test_lj_gradients_elementwise_for_single_particles(cuda):
    # Individual gradient entries: for 8 particles, each coordinate of x0 and v0
    # perturbed alone by +-1e-6 (FP64 oracle trajectory, shifted-force LJ, 100
    # steps, checkpoints every 20), the central difference against the adjoint's
    # entry for that particle and coordinate.
    n, rho, K, ckpt = 2048, 0.3, 100, 20
    L = mi.box_for(n, rho, 4.0)
    dx, width, h = 4.0, 2.0, 1e-6
    x0, v0 = mi.lj_initial_state(n, L, 1.0, seed=n + 5)
    p = m.Params(n=n, box=L, dx=dx, sort_every=ckpt, vmax=V, potential=m.POT_LJ_SF)
    with m.Simulation(p, x0, v0) as s:
        out = s.adjoint(K, ckpt, width, dloss=M2)
    picks = np.random.default_rng(11).choice(n, size=8, replace=False)
    got, fd = [], []
    for i in picks:
        for a in (0, 1):
            for which in ("x", "v"):
                e = np.zeros((n, 2))
                e[i, a] = h
                if which == "x":
                    lp = _lj_loss(x0 + e, v0, L, 1.0, 1.0, K, dx, width, True)
                    lm = _lj_loss(x0 - e, v0, L, 1.0, 1.0, K, dx, width, True)
                    got.append(out["grad_x0"][i, a])
                else:
                    lp = _lj_loss(x0, v0 + e, L, 1.0, 1.0, K, dx, width, True)
                    lm = _lj_loss(x0, v0 - e, L, 1.0, 1.0, K, dx, width, True)
                    got.append(out["grad_v0"][i, a])
                fd.append((lp - lm) / (2 * h))
    got, fd = np.array(got), np.array(fd)
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.all(np.abs(got - fd) <= 5e-3 * np.abs(fd) + 1e-3 * scale), \
        (got.tolist(), fd.tolist())
