"""Host-side closed forms used to pin the oracle (test infrastructure only).

- Maxwell equal-area construction, Eq. Maxwell_equal_area (Sec. 3.1):
  P(rho_v) = P(rho_l) = P_sat and int_{rho_v}^{rho_l} (P_sat - P)/rho^2 = 0.
- Second-gradient flat-interface profile (Sec. 2.1): with the grand-potential
  excess omega(rho) = rho int_{rho_v}^{rho} (P(r) - P_sat)/r^2 dr, the
  equilibrium profile obeys kappa/2 (drho/dx)^2 = omega(rho), so the width of
  Eq. interface_W is W = (rho_l - rho_v) / sqrt(2 max omega / kappa) and the
  surface tension sigma = int sqrt(2 kappa omega) drho.
- Equimolar radius, Eq. equmol2Ddrop (and its 3D analogue), Laplace law
  Eq. Laplace_equimolar.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

from .lbm import EOS


def _dP(eos: EOS, rho: float) -> float:
    h = 1e-6 * max(rho, 1e-3)
    return (eos(rho + h) - eos(rho - h)) / (2 * h)


def spinodals(eos: EOS):
    """Local max and min of P(rho) on (0, 1/b) (the two spinodal densities)."""
    hi = (1.0 / eos.b) * (0.999 if eos.eos != 3 else 3.99)
    grid = np.concatenate([np.geomspace(1e-9, 1e-2, 400), np.linspace(1e-2, hi, 20000)])
    d = np.array([_dP(eos, r) for r in grid])
    idx = np.nonzero(np.sign(d[:-1]) != np.sign(d[1:]))[0]
    if len(idx) < 2:
        raise ValueError("no spinodal pair: T/Tc >= 1?")
    roots = [optimize.brentq(lambda r: _dP(eos, r), grid[k], grid[k + 1], xtol=1e-15)
             for k in idx[:2]]
    return roots[0], roots[1]


def _outer_roots(eos: EOS, p: float, s1: float, s2: float):
    hi = (1.0 / eos.b) * (0.999999 if eos.eos != 3 else 3.999)
    rv = optimize.brentq(lambda r: eos(r) - p, 1e-300, s1, xtol=1e-300, rtol=1e-15,
                         maxiter=500)
    rl = optimize.brentq(lambda r: eos(r) - p, s2, hi, xtol=1e-300, rtol=1e-15,
                         maxiter=500)
    return rv, rl


def _area(eos: EOS, p: float, rv: float, rl: float) -> float:
    val, _ = integrate.quad(lambda r: (p - eos(r)) / r ** 2, rv, rl, epsabs=1e-15,
                            epsrel=1e-13, limit=400, points=None)
    return val


def maxwell(eos: EOS):
    """Coexistence (rho_v, rho_l, P_sat) by the equal-area rule."""
    s1, s2 = spinodals(eos)
    pmax, pmin = eos(s1), eos(s2)
    lo = max(pmin, 0.0) + 1e-14 * abs(pmax)
    hi = pmax - 1e-14 * abs(pmax)

    def g(p):
        rv, rl = _outer_roots(eos, p, s1, s2)
        # scale the area by 1/rho_v so both ends of the bracket stay O(1)
        return _area(eos, p, rv, rl) * rv

    p = optimize.brentq(g, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
    rv, rl = _outer_roots(eos, p, s1, s2)
    return rv, rl, p


def omega_excess(eos: EOS, rho, rho_v: float, p_sat: float):
    """Grand-potential excess rho * int_{rho_v}^{rho} (P - P_sat)/r^2 dr."""
    def one(r):
        val, _ = integrate.quad(lambda s: (eos(s) - p_sat) / s ** 2, rho_v, r,
                                epsabs=1e-15, epsrel=1e-13, limit=400)
        return r * val
    if np.ndim(rho):
        return np.array([one(r) for r in rho])
    return one(rho)


def max_omega(eos: EOS, rho_v: float, rho_l: float, p_sat: float) -> float:
    grid = np.linspace(rho_v, rho_l, 401)[1:-1]
    vals = omega_excess(eos, grid, rho_v, p_sat)
    k = int(np.argmax(vals))
    lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, len(grid) - 1)]
    res = optimize.minimize_scalar(lambda r: -omega_excess(eos, r, rho_v, p_sat),
                                   bounds=(lo, hi), method="bounded",
                                   options={"xatol": 1e-12})
    return -res.fun


def interface_width(eos: EOS, kappa: float, coex=None) -> float:
    rv, rl, p = coex if coex is not None else maxwell(eos)
    return (rl - rv) / math.sqrt(2.0 * max_omega(eos, rv, rl, p) / kappa)


def kappa_for_width(eos: EOS, width: float, coex=None) -> float:
    rv, rl, p = coex if coex is not None else maxwell(eos)
    return width ** 2 * 2.0 * max_omega(eos, rv, rl, p) / (rl - rv) ** 2


def surface_tension(eos: EOS, kappa: float, coex=None) -> float:
    rv, rl, p = coex if coex is not None else maxwell(eos)
    val, _ = integrate.quad(lambda r: math.sqrt(max(2.0 * kappa *
                                                    omega_excess(eos, r, rv, p), 0.0)),
                            rv, rl, epsabs=1e-13, epsrel=1e-10, limit=200)
    return val


def vdw_sigma_near_critical(a: float, b: float, kappa: float, t_over_tc: float) -> float:
    """Eq. vdw_surface_tension: 16a/(27b^2) sqrt(kappa/a) (1 - Tr)^(3/2)."""
    return 16.0 * a / (27.0 * b * b) * math.sqrt(kappa / a) * (1.0 - t_over_tc) ** 1.5


def equimolar_radius(rho: np.ndarray, rho_v: float, rho_l: float, dim: int) -> float:
    """Radius of the sphere (dim 3) or circle (dim 2) holding the excess mass."""
    excess = float(np.sum(rho - rho_v)) / (rho_l - rho_v)
    if dim == 2:
        return math.sqrt(excess / math.pi)
    return (3.0 * excess / (4.0 * math.pi)) ** (1.0 / 3.0)


def layered_poiseuille(layers, g: float, top: str = "wall"):
    """Steady body-force-driven flow through flat layers (Sec. 4.1, Eqs.
    poiseuille_odes and poiseuille_odes_BD): in each layer
    d/dy(mu du/dy) + rho g = 0, u = 0 at y = 0, u and mu du/dy continuous at
    each interface, and at the top y = H either u = 0 (top="wall") or
    du/dy = 0 (top="symmetry", the mid-plane of a channel mirrored about it).
    layers: [(thickness, rho, mu), ...] from y = 0 upward. Returns u(y).
    Each layer's u is a parabola a y^2 + B y + C with a = -rho g / (2 mu);
    the 2K unknowns (B, C) solve the 2K conditions above."""
    K = len(layers)
    edges = np.concatenate([[0.0], np.cumsum([t for t, _, _ in layers])])
    a = [-r * g / (2.0 * m) for _, r, m in layers]
    A = np.zeros((2 * K, 2 * K))
    rhs = np.zeros(2 * K)
    A[0, 1] = 1.0                                        # u(0) = 0
    row = 1
    for k in range(K - 1):
        y = edges[k + 1]
        mk, mn = layers[k][2], layers[k + 1][2]
        A[row, 2 * k], A[row, 2 * k + 1] = y, 1.0        # u continuous
        A[row, 2 * k + 2], A[row, 2 * k + 3] = -y, -1.0
        rhs[row] = (a[k + 1] - a[k]) * y * y
        row += 1
        A[row, 2 * k], A[row, 2 * k + 2] = mk, -mn       # mu du/dy continuous
        rhs[row] = 2.0 * y * (mn * a[k + 1] - mk * a[k])
        row += 1
    H = edges[-1]
    if top == "wall":
        A[row, 2 * K - 2], A[row, 2 * K - 1] = H, 1.0
        rhs[row] = -a[-1] * H * H
    else:
        A[row, 2 * K - 2] = 1.0
        rhs[row] = -2.0 * a[-1] * H
    BC = np.linalg.solve(A, rhs)

    def u(y):
        y = np.asarray(y, dtype=float)
        k = np.clip(np.searchsorted(edges, y, side="right") - 1, 0, K - 1)
        return np.asarray(a)[k] * y * y + BC[2 * k] * y + BC[2 * k + 1]
    return u


def channel_flow_from_profile(rho_rows, g: float, nu):
    """Steady U(y) of body-force-driven flow along a channel mirrored about
    its mid-plane, for a density profile across it (rho at the fluid rows,
    halfway walls half a row beyond the first and last): the momentum
    balance d/dy(rho nu dU/dy) + rho g = 0 of a parallel flow, integrated
    row by row. A flat interface adds no shear stress (the Korteweg tensor
    has no xy part when rho varies along y only), so this is the diffuse-
    interface counterpart of layered_poiseuille. nu: a number, or the
    kinematic viscosity of each row. Even row count assumed."""
    r = np.asarray(rho_rows, dtype=float)
    mu = r * np.broadcast_to(np.asarray(nu, dtype=float), r.shape)
    m = len(r) // 2
    U = np.zeros(len(r))
    U[0] = 0.5 * g * np.sum(r[:m]) / mu[0]                # wall to the first row
    for j in range(1, m):
        U[j] = U[j - 1] + g * np.sum(r[j:m]) / (0.5 * (mu[j - 1] + mu[j]))
    U[m:] = U[:m][::-1]
    return U
