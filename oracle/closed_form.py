"""Closed-form MDLG equilibrium of Sec. IV-A (Eqs. fieqW, fgen, feqfull, fialpha).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product library.

For uniformly placed particles whose displacements over the coarse time step
are Gaussian with per-axis variance <dx_a^2> and mean u_a dt, the expected
occupation of lattice velocity v_i divided by the particles per cell is the
product over axes of

    f_{i,a} = N [ g(u-1) - 2 g(u) + g(u+1) ]
              + (u-1)/2 [ erf((u-1)/(sqrt2 a)) - erf(u/(sqrt2 a)) ]
              + (u+1)/2 [ erf((u+1)/(sqrt2 a)) - erf(u/(sqrt2 a)) ]

with g(z) = exp(-z^2 / (2 a^2)), N = a / sqrt(2 pi), a^2 = <dx_a^2> / dx^2 and
u = u_{i,a} = v_{i,a} - u_a (lattice units).  This is the Gaussian convolution
of the one-dimensional wedge W(s) = (1 - |s|)_+ evaluated at u (Eq. fieqW).

For the ballistic (collisionless) gas at temperature T with unit mass,
<dx_a^2> = T dt^2 (Sec. IV-A), so a = sqrt(T) dt / dx.
"""
from __future__ import annotations

import math

import numpy as np

# D2Q9 lattice Boltzmann weights of Sec. V (rest, axis, diagonal).
D2Q9_WEIGHTS = (4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0)


def f_axis(u: float, a: float) -> float:
    """One-axis factor f_{i,a} of Eq. fialpha at shifted velocity u, width a."""
    if a == 0.0:
        # Degenerate limit: no displacement spread, the wedge itself.
        return max(0.0, 1.0 - abs(u))
    n = a / math.sqrt(2.0 * math.pi)

    def g(z: float) -> float:
        return math.exp(-z * z / (2.0 * a * a))

    def e(z: float) -> float:
        return math.erf(z / (math.sqrt(2.0) * a))

    return (n * (g(u - 1.0) - 2.0 * g(u) + g(u + 1.0))
            + 0.5 * (u - 1.0) * (e(u - 1.0) - e(u))
            + 0.5 * (u + 1.0) * (e(u + 1.0) - e(u)))


def feq_over_rho(v: tuple[int, int], a: float, u: tuple[float, float] = (0.0, 0.0)) -> float:
    """f_i^eq / rho^eq for lattice velocity v = (v_x, v_y) (Eq. feqfull)."""
    return f_axis(v[0] - u[0], a) * f_axis(v[1] - u[1], a)


def feq_window(vmax: int, a: float, u: tuple[float, float] = (0.0, 0.0)) -> np.ndarray:
    """f_i^eq / rho^eq on the (2V+1)^2 window plus the overflow entry.

    Index i = (v_y + V)(2V+1) + (v_x + V); entry (2V+1)^2 holds the mass of all
    displacements outside the window, 1 - sum of the window (the axis factors
    each sum to one over all integers).
    """
    w = 2 * vmax + 1
    fx = np.array([f_axis(k - u[0], a) for k in range(-vmax, vmax + 1)])
    fy = np.array([f_axis(k - u[1], a) for k in range(-vmax, vmax + 1)])
    out = np.empty(w * w + 1)
    out[: w * w] = np.outer(fy, fx).ravel()
    out[w * w] = 1.0 - out[: w * w].sum()
    return out


def a_ballistic(temperature: float, dt: float, dx: float, mass: float = 1.0) -> float:
    """a for free flight: <dx_a^2> = (T/m) dt^2 (Sec. IV-A), a^2 = <dx_a^2>/dx^2."""
    return math.sqrt(temperature / mass) * dt / dx


def msd_exponential_vacf(temperature: float, tau: float, t: float) -> float:
    """<dx_a^2> for an exponentially decaying velocity autocorrelation (Eq. vca)."""
    return 2.0 * temperature * tau * tau * (math.exp(-t / tau) + t / tau - 1.0)


# ---------------------------------------------------------------------------
# Soft-binned MDLG occupations (the differentiable loss of the adjoint)
# ---------------------------------------------------------------------------
# The cell indicator of Sec. III, 1 on (c dx, (c+1) dx], is replaced by the same
# box smoothed with a Gaussian of standard deviation s:
#     u_c(x) = Phi((x - c dx) / s) - Phi((x - (c+1) dx) / s),
# so that sum_c u_c(x) = 1 and u_c -> indicator as s -> 0.  The soft occupation
# of Eq. MDni over one interval, averaged over particles, is
#     ft_i = (1/N) sum_j prod_a sum_c u_c(x_ja(t)) u_{c - v_ia}(x_ja(t - dt)).


def _phi_cdf(z):
    from scipy.special import ndtr
    return ndtr(z)


def soft_fi(x_end, x_start, box, dx, width, vmax):
    """Soft f_i on the (2V+1)^2 window, index i = (v_y+V)(2V+1) + (v_x+V).

    x_end, x_start: (n, 2) positions in (0, L]; the displacement is taken by
    minimum image.  width: the smoothing s in length units.
    """
    x_end = np.asarray(x_end, dtype=np.float64)
    x_start = np.asarray(x_start, dtype=np.float64)
    L = np.asarray(box, dtype=np.float64).reshape(2)
    w = 2 * vmax + 1
    M = int(math.ceil(8.0 * width / dx)) + 1
    k_axis = []
    for a in range(2):
        d = x_end[:, a] - x_start[:, a]
        d -= L[a] * np.round(d / L[a])
        ta = x_end[:, a] / dx                  # lattice units
        tb = (x_end[:, a] - d) / dx            # start, unwrapped next to the end
        sw = width / dx
        base = np.floor(ta).astype(np.int64)
        kv = np.zeros((x_end.shape[0], w))
        for dc in range(-M, M + 1):
            c = base + dc
            ua = _phi_cdf((ta - c) / sw) - _phi_cdf((ta - c - 1) / sw)
            for vi, v in enumerate(range(-vmax, vmax + 1)):
                ub = _phi_cdf((tb - (c - v)) / sw) - _phi_cdf((tb - (c - v) - 1) / sw)
                kv[:, vi] += ua * ub
        k_axis.append(kv)
    kx, ky = k_axis
    return np.einsum("ny,nx->yx", ky, kx).ravel() / x_end.shape[0]
