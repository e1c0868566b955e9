"""Host-side analyses of the MDLG equilibrium f_i (Secs. IV-A, V, VI of
arXiv:1705.04368): velocity moments Psi, Phi and the two temperatures theta_2,
theta_3 (Eqs. Psi, Phi, tet2, tet3), the closed-form equilibrium of Eq.
feqfull with the exponential velocity-correlation model of Eq. vca, and the
(dx, dt) pairs whose equilibrium matches the D2Q9 weights (Eq. wif0eqn,
Fig. dtdx).

These operate on the (2V+1)^2 (+1 overflow) vector of f_i / rho that
Simulation.stats() returns (or on the closed form); they are a few hundred
floating-point operations each and run on the host in FP64.  Velocity index
i = (v_y + V)(2V+1) + (v_x + V), as everywhere in the library.
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import numpy as np

# D2Q9 lattice Boltzmann weights (Sec. V): rest, axis, diagonal
D2Q9 = {(0, 0): 4.0 / 9.0, (1, 0): 1.0 / 9.0, (1, 1): 1.0 / 36.0}


def lb_equilibrium(u: Sequence[float], vmax: int = 1, theta: float = 1.0 / 3.0,
                   rho: float = 1.0) -> np.ndarray:
    """Second-order lattice Boltzmann equilibrium of Sec. V (Eq. f0lb) for the
    D2Q9 weights, f_i^0 = rho w_i (1 + v.u/theta + (v.u)^2/(2 theta^2) - u.u/(2 theta)),
    laid out on the (2V+1)^2 window (zero outside the first shell) plus an
    empty overflow entry."""
    vel = velocity_table(vmax).astype(np.float64)
    w = np.zeros(len(vel))
    for k, (vx, vy) in enumerate(vel.astype(int)):
        if max(abs(vx), abs(vy)) <= 1:
            w[k] = D2Q9[(max(abs(vx), abs(vy)), min(abs(vx), abs(vy)))]
    uu = np.asarray(u, dtype=np.float64)
    vu = vel @ uu
    f = rho * w * (1.0 + vu / theta + 0.5 * vu * vu / (theta * theta) - 0.5 * (uu @ uu) / theta)
    return np.concatenate([f, [0.0]])


def velocity_table(vmax: int) -> np.ndarray:
    """(Q, 2) integer lattice velocities in index order."""
    w = 2 * vmax + 1
    i = np.arange(w * w)
    return np.stack([i % w - vmax, i // w - vmax], axis=1)


def _window(f, vmax: int) -> np.ndarray:
    q = (2 * vmax + 1) ** 2
    f = np.asarray(f, dtype=np.float64).reshape(-1)
    if f.size not in (q, q + 1):
        raise ValueError(f"expected {q} or {q + 1} entries for V = {vmax}, got {f.size}")
    return f[:q]


def moments(f, vmax: int, u: Sequence[float] = (0.0, 0.0), a: Optional[float] = None,
            shells: Optional[int] = None) -> dict:
    """Velocity moments of a discrete distribution f_i (overflow entry ignored).

    rho = sum_i f_i, mean = sum_i f_i v_i / rho and the central moments about
    u (lattice units) M2[a][b] = sum_i f_i c_ia c_ib / rho, M3[a][b][c] likewise
    with c_i = v_i - u.  With the displacement width a (Eq. eqn:a) also
    Psi = M2 / a^2 (Eq. Psi) and Phi = M3 / a^3 (Eq. Phi).  shells = s keeps
    only the velocities with |v_x|, |v_y| <= s (s = 1: the nine velocities of a
    single shell).
    """
    fw = _window(f, vmax).copy()
    vel = velocity_table(vmax).astype(np.float64)
    if shells is not None:
        fw[np.abs(vel).max(axis=1) > shells] = 0.0
    rho = fw.sum()
    c = vel - np.asarray(u, dtype=np.float64)
    m2 = np.einsum("i,ia,ib->ab", fw, c, c) / rho
    m3 = np.einsum("i,ia,ib,ic->abc", fw, c, c, c) / rho
    out = {"rho": rho, "mean": (fw @ vel) / rho, "M2": m2, "M3": m3}
    if a is not None:
        out["Psi"] = m2 / (a * a)
        out["Phi"] = m3 / (a ** 3)
    return out


def theta2(f, vmax: int, u: Sequence[float] = (0.0, 0.0), shells: Optional[int] = None) -> float:
    """theta_2 = a^2 Psi_xx, the second central moment along x (Eq. tet2)."""
    return float(moments(f, vmax, u, shells=shells)["M2"][0, 0])


def theta3(f_plus, f_minus, du: float, vmax: int, shells: Optional[int] = None) -> float:
    """theta_3 = (1 / 3 rho) d/du_x sum_i f_i(u) v_ix^3 (Eq. tet3), as the central
    difference of two distributions taken at u_x = +du and -du."""
    vx3 = velocity_table(vmax)[:, 0].astype(np.float64) ** 3
    out = []
    for f in (f_plus, f_minus):
        fw = _window(f, vmax).copy()
        if shells is not None:
            fw[np.abs(velocity_table(vmax)).max(axis=1) > shells] = 0.0
        out.append((fw @ vx3) / fw.sum())
    return (out[0] - out[1]) / (2.0 * du) / 3.0


# ---- closed-form equilibrium (Eqs. fgen, feqfull, fialpha) ------------------------

def _axis_factor(c: float, a: float) -> float:
    """One-axis factor of Eq. fialpha: the wedge (1 - |s|)_+ averaged over a
    Gaussian of width a centred at c = v - u (lattice units)."""
    if a == 0.0:
        return max(0.0, 1.0 - abs(c))
    s2a = math.sqrt(2.0) * a
    norm = a / math.sqrt(2.0 * math.pi)
    gauss = [math.exp(-(c + d) ** 2 / (2.0 * a * a)) for d in (-1.0, 0.0, 1.0)]
    erfs = [math.erf((c + d) / s2a) for d in (-1.0, 0.0, 1.0)]
    return (norm * (gauss[0] - 2.0 * gauss[1] + gauss[2])
            + 0.5 * (c - 1.0) * (erfs[0] - erfs[1])
            + 0.5 * (c + 1.0) * (erfs[2] - erfs[1]))


def feq(vmax: int, a: float, u: Sequence[float] = (0.0, 0.0)) -> np.ndarray:
    """f_i^eq / rho^eq of Eq. feqfull on the window, plus the overflow mass."""
    ks = range(-vmax, vmax + 1)
    fx = np.array([_axis_factor(k - u[0], a) for k in ks])
    fy = np.array([_axis_factor(k - u[1], a) for k in ks])
    win = np.outer(fy, fx).ravel()
    return np.concatenate([win, [1.0 - win.sum()]])


def msd_exponential(temperature: float, tau: float, t: float, mass: float = 1.0) -> float:
    """<dx_a^2>(t) = 2 (k_B T / m) tau^2 (exp(-t / tau) + t / tau - 1) (Eq. vca)."""
    x = t / tau
    # expm1 keeps the ballistic limit T t^2 accurate for t << tau
    return 2.0 * temperature / mass * tau * tau * (math.expm1(-x) + x)


def _bisect(fn, lo: float, hi: float, tol: float = 1e-14, it: int = 200) -> float:
    flo = fn(lo)
    for _ in range(it):
        mid = 0.5 * (lo + hi)
        fm = fn(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
        if hi - lo <= tol * max(1.0, abs(mid)):
            break
    return 0.5 * (lo + hi)


def a2_matching_weight(v: Sequence[int], weight: float) -> float:
    """a^2 at which f_i^eq(a) / rho = weight for lattice velocity v at u = 0
    (one equation of the over-determined Eq. wif0eqn).  f_i^eq is monotone in
    a on the bracket used: decreasing for the rest velocity, increasing for the
    first shell below its maximum."""
    def g(a2):
        a = math.sqrt(a2)
        return _axis_factor(float(v[0]), a) * _axis_factor(float(v[1]), a) - weight
    return _bisect(g, 1e-4, 0.3)


def consistent_dt(dx: float, temperature: float, tau: float, mass: float = 1.0,
                  weights: Optional[dict] = None) -> dict:
    """Time steps dt that make the equilibrium at lattice spacing dx equal the
    lattice Boltzmann weights (Sec. V, Fig. dtdx): for every weight w_i, a^2
    from Eq. wif0eqn, then dt from a^2 dx^2 = <dx_a^2>(dt) of Eq. vca.
    Returns {velocity: (a^2, dt)}."""
    weights = D2Q9 if weights is None else weights
    out = {}
    for v, w in weights.items():
        a2 = a2_matching_weight(v, w)
        target = a2 * dx * dx
        hi = 1.0
        while msd_exponential(temperature, tau, hi, mass) < target:
            hi *= 2.0
        dt = _bisect(lambda t: msd_exponential(temperature, tau, t, mass) - target, 0.0, hi)
        out[v] = (a2, dt)
    return out
