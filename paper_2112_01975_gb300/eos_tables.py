"""Host-side set-up values for synthetic workloads: coexistence densities by
the Maxwell equal-area rule (Sec. 3.1, Eq. Maxwell_equal_area) and the
capillary coefficient giving a chosen second-gradient interface width
(Eq. interface_W), for the van der Waals and Peng-Robinson EOS.

These prepare initial conditions only (the drop profile between the two
densities); nothing here is part of a time step. Written independently of
the test oracle and cross-checked against it by a CPU test.
"""
from __future__ import annotations

import functools
import math

import numpy as np
from scipy import integrate, optimize

B_DEFAULT = 2.0 / 21.0


def _rtc(eos: int, a: float, b: float) -> float:
    return 8.0 * a / (27.0 * b) if eos == 0 else (0.0778 / 0.45724) * a / b


def _alpha(eos: int, tr: float, acentric: float = 0.344) -> float:
    if eos != 1:
        return 1.0
    m = 0.37464 + 1.54226 * acentric - 0.26992 * acentric ** 2
    return (1.0 + m * (1.0 - math.sqrt(tr))) ** 2


def pressure(eos: int, tr: float, a: float, b: float = B_DEFAULT):
    rt = tr * _rtc(eos, a, b)
    al = _alpha(eos, tr)

    def P(r):
        r = np.asarray(r, dtype=float)
        base = r * rt / (1.0 - b * r)
        if eos == 0:
            return base - a * r * r
        return base - a * al * r * r / (1.0 + 2.0 * b * r - b * b * r * r)
    return P


def _dP(P, r):
    h = 1e-7 * max(r, 1e-6)
    return float((P(r + h) - P(r - h)) / (2 * h))


@functools.lru_cache(maxsize=256)
def coexistence(eos: int, tr: float, a: float, b: float = B_DEFAULT):
    """(rho_v, rho_l, P_sat) of the equal-area rule."""
    P = pressure(eos, tr, a, b)
    grid = np.concatenate([np.geomspace(1e-9, 0.05, 300), np.linspace(0.05, 0.999 / b, 6000)])
    d = np.array([_dP(P, r) for r in grid])
    k = np.nonzero(np.sign(d[:-1]) != np.sign(d[1:]))[0]
    s1 = optimize.brentq(lambda r: _dP(P, r), grid[k[0]], grid[k[0] + 1])
    s2 = optimize.brentq(lambda r: _dP(P, r), grid[k[1]], grid[k[1] + 1])
    hi = 0.9999999 / b

    def roots(p):
        return (optimize.brentq(lambda r: float(P(r)) - p, 1e-300, s1, xtol=1e-300, rtol=1e-15),
                optimize.brentq(lambda r: float(P(r)) - p, s2, hi, xtol=1e-300, rtol=1e-15))

    def area(p):
        rv, rl = roots(p)
        v, _ = integrate.quad(lambda r: (p - float(P(r))) / r ** 2, rv, rl, epsabs=1e-14,
                              epsrel=1e-12, limit=300)
        return v * rv

    pmax, pmin = float(P(s1)), float(P(s2))
    lo = max(pmin, 0.0) + 1e-13 * abs(pmax)
    p = optimize.brentq(area, lo, pmax * (1 - 1e-13), xtol=1e-300, rtol=1e-14)
    rv, rl = roots(p)
    return rv, rl, p


def kappa_for_width(eos: int, tr: float, a: float, width: float = 5.0, b: float = B_DEFAULT):
    """kappa with second-gradient width W = (rho_l - rho_v) / max|rho'| = width,
    from kappa/2 rho'^2 = rho int_{rho_v}^{rho} (P - P_sat)/r^2 dr."""
    rv, rl, ps = coexistence(eos, tr, a, b)
    P = pressure(eos, tr, a, b)

    def omega(r):
        v, _ = integrate.quad(lambda s: (float(P(s)) - ps) / s ** 2, rv, r, epsabs=1e-14,
                              epsrel=1e-12, limit=300)
        return r * v
    res = optimize.minimize_scalar(lambda r: -omega(r), bounds=(rv, rl), method="bounded",
                                   options={"xatol": 1e-10})
    return width ** 2 * 2.0 * (-res.fun) / (rl - rv) ** 2


def stable_a(eos: int, tr: float, cs2_max: float = 0.1, b: float = B_DEFAULT) -> float:
    """Attraction a (lattice units) scaled so that the liquid's isothermal
    dP/drho is cs2_max; coexistence densities do not depend on a."""
    a0 = 9.0 / 49.0 if eos == 0 else 2.0 / 49.0
    _, rl, _ = coexistence(eos, tr, a0, b)
    cs2 = _dP(pressure(eos, tr, a0, b), rl)
    return a0 * min(1.0, cs2_max / cs2)


class SetupTable:
    """The set-up values of a sweep's requests, (a, rho_v, rho_l, kappa) as
    functions of T/Tc on [lo, hi], for one EOS and interface width: each
    evaluated at the deg + 1 Chebyshev points of the interval (a, rho_l and
    kappa directly, rho_v through its logarithm) and interpolated by the
    Chebyshev series through them. Degree 32 reproduces the direct values
    to about 1e-8 relative on the van der Waals sweep range [0.5, 0.95]
    (tested); building it costs deg + 1 direct evaluations once, a lookup
    microseconds, so a server pays the Maxwell construction at start-up
    and not per request."""

    def __init__(self, eos: int = 0, lo: float = 0.5, hi: float = 0.95, deg: int = 32,
                 width: float = 5.0):
        from numpy.polynomial import chebyshev
        self.eos, self.lo, self.hi, self.width = eos, lo, hi, width
        x = np.cos(np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1))
        vals = np.array([self._direct(lo + (hi - lo) * (xx + 1.0) / 2.0) for xx in x])
        vals[:, 1] = np.log(vals[:, 1])
        self._coef = [chebyshev.chebfit(x, vals[:, j], deg) for j in range(4)]
        self._val = chebyshev.chebval

    def _direct(self, tr: float):
        a = stable_a(self.eos, tr)
        rv, rl, _ = coexistence(self.eos, tr, a)
        return np.array([a, rv, rl, kappa_for_width(self.eos, tr, a, width=self.width)])

    def __call__(self, tr: float):
        """(a, rho_v, rho_l, kappa) at T/Tc = tr (computed directly outside [lo, hi])."""
        if not (self.lo <= tr <= self.hi):
            return tuple(float(v) for v in self._direct(tr))
        x = 2.0 * (tr - self.lo) / (self.hi - self.lo) - 1.0
        a, lrv, rl, k = (float(self._val(x, c)) for c in self._coef)
        return a, math.exp(lrv), rl, k
