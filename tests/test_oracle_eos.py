"""Pins of the oracle's equations of state and of the host-side closed forms.

Critical points and critical compressibilities are textbook values of each
EOS (Sec. 3.1), and for the Shan-Chen forms the values Appendix G prints; the van der Waals Maxwell construction is checked with the
closed-form antiderivative of P/rho^2, not with the quadrature the tool uses.
"""
import math

import numpy as np
import pytest

from conftest import printed
from oracle import physics as ph
from oracle.lbm import EOS
from paper_2112_01975_gb300 import inputs


def _d(e, r, h=1e-4):
    return (e(r + h) - e(r - h)) / (2 * h), (e(r + h) - 2 * e(r) + e(r - h)) / h ** 2


def test_vdw_critical_point_closed_form():
    """a = 27/64 R2Tc2/Pc, b = RTc/(8Pc): rho_c = 1/(3b), Pc = a/(27b^2) = 3/4 for
    (9/49, 2/21), and both derivatives vanish there at T = Tc."""
    e = EOS(0, 1.0)
    rc = 1.0 / (3.0 * e.b)
    assert e(rc) == pytest.approx(e.a / (27 * e.b ** 2), rel=1e-14)
    assert e(rc) == pytest.approx(0.75, rel=1e-14)
    d1, d2 = _d(e, rc)
    assert abs(d1) < 1e-7 and abs(d2) < 1e-5
    assert e(rc) / (rc * e.RTc) == pytest.approx(3.0 / 8.0, rel=1e-13)


@pytest.mark.parametrize("eos,zc", [(1, 0.3074), (2, 1.0 / 3.0), (3, 0.3590)])
def test_critical_compressibility(eos, zc):
    """At T = Tc the inflection of P(rho) has P' = P'' = 0 (to the rounding of the
    printed constants) and Zc = Pc/(rho_c R Tc) is the textbook value of the EOS."""
    e = EOS(eos, 1.0)
    grid = np.linspace(0.05, 0.99 / e.b if eos != 3 else 3.5 / e.b, 20001)
    d1 = np.gradient(e(grid), grid)
    k = int(np.argmin(np.abs(d1)))
    from scipy import optimize
    rc = optimize.minimize_scalar(lambda r: abs(_d(e, r)[1]), bounds=(grid[k] * 0.8, grid[k] * 1.2),
                                  method="bounded", options={"xatol": 1e-10}).x
    d1, d2 = _d(e, rc)
    scale = e(rc) / rc
    assert abs(d1) < 2e-3 * scale
    assert e(rc) / (rc * e.RTc) == pytest.approx(zc, rel=2e-3)


@pytest.mark.parametrize("eos,gc,rc", [(4, -4.0, math.log(2.0)), (5, -math.exp(2.0), 1.0)])
def test_shan_chen_critical_points(eos, gc, rc):
    """The critical couplings and densities the paper prints for the two
    Shan-Chen pseudo-potentials (Appendix G: G_c = -4, rho_c = 0.6931 and
    G_c = -7.389, rho_c = 1): at T/Tc = 1 the coupling is G_c and P' = P'' = 0
    at rho_c, and nowhere else does P' vanish."""
    e = EOS(eos, 1.0)
    assert e.RT == pytest.approx(gc, rel=1e-15)
    pv = printed({4: "shan_chen_1_critical", 5: "shan_chen_2_critical"}[eos])
    assert round(rc, 4) == pytest.approx(pv["rho_c"], abs=1e-12)        # as printed
    assert round(gc, 3) == pytest.approx(pv["G_c"], abs=1e-12)
    d1, d2 = _d(e, rc)
    assert abs(d1) < 1e-7 and abs(d2) < 1e-5
    grid = np.linspace(0.05, 5.0, 4001)
    assert np.all(np.gradient(e(grid), grid) > -1e-6)          # no loop at T = Tc
    below = EOS(eos, 0.9)
    assert np.min(np.gradient(below(grid), grid)) < 0.0          # a van der Waals loop below


@pytest.mark.parametrize("eos", [4, 5])
def test_shan_chen_sound_faster_in_vapour(eos):
    """The paper's remark on the Shan-Chen forms (Appendix G): at coexistence
    the isothermal sound speed dP/drho is larger in the vapour than in the
    liquid, the reverse of the cubic equations of state."""
    e = EOS(eos, 0.8)
    rv, rl, _ = ph.maxwell(e)
    assert _d(e, rv)[0] > _d(e, rl)[0] > 0.0
    v = EOS(0, 0.8)
    vv, vl, _ = ph.maxwell(v)
    assert _d(v, vv)[0] < _d(v, vl)[0]


def test_maxwell_vdw_closed_form_area():
    """int P/rho^2 = RT ln(rho/(1 - b rho)) - a rho for vdW; the tool's
    (rho_v, rho_l, P_sat) must zero both the pressure jump and the area."""
    e = EOS(0, 0.8, a=9 / 490)
    rv, rl, ps = ph.maxwell(e)

    def anti(r):
        return e.RT * math.log(r / (1 - e.b * r)) - e.a * r
    area = ps * (1 / rv - 1 / rl) - (anti(rl) - anti(rv))
    assert abs(e(rv) - ps) < 1e-12 * ps and abs(e(rl) - ps) < 1e-12 * ps
    assert abs(area) < 1e-11 * ps / rv


def test_corresponding_states():
    """Coexistence densities in units of rho_c = 1/(3b) depend on T/Tc alone."""
    a1 = ph.maxwell(EOS(0, 0.7, a=9 / 49, b=2 / 21))
    a2 = ph.maxwell(EOS(0, 0.7, a=0.0011, b=0.05))
    assert a1[0] * 2 / 21 == pytest.approx(a2[0] * 0.05, rel=1e-9)
    assert a1[1] * 2 / 21 == pytest.approx(a2[1] * 0.05, rel=1e-9)
    p1 = ph.maxwell(EOS(1, 0.7, a=2 / 49))
    p2 = ph.maxwell(EOS(1, 0.7, a=2 / 245))
    assert p1[0] == pytest.approx(p2[0], rel=1e-9) and p1[1] == pytest.approx(p2[1], rel=1e-9)


def test_printed_density_ratio_tr077():
    """Sec. 4.1 quotes rho_l/rho_v = 10.1 at T_r = 0.77 for vdW (simulated);
    the equal-area ratio is within the paper's quoted deviations of it."""
    pv = printed("layered_poiseuille_a")
    rv, rl, _ = ph.maxwell(EOS(0, pv["T_r"]))
    assert rl / rv == pytest.approx(pv["density_ratio"], rel=0.02)


def test_surface_tension_near_critical_asymptote():
    """Eq. vdw_surface_tension is the T_r -> 1 limit of the second-gradient sigma."""
    a, b, kap = 9 / 49, 2 / 21, 0.02
    errs = []
    for tr in (0.99, 0.995):
        e = EOS(0, tr, a=a, b=b)
        s = ph.surface_tension(e, kap)
        errs.append(abs(s / ph.vdw_sigma_near_critical(a, b, kap, tr) - 1))
    assert errs[1] < 0.01
    assert errs[1] < 0.7 * errs[0]     # converges as T_r -> 1


def test_width_scales_as_sqrt_kappa_over_a():
    """W = (rho_l - rho_v)/max|grad rho| grows as sqrt(kappa) and as 1/sqrt(a)."""
    e1 = EOS(0, 0.8, a=9 / 49)
    e2 = EOS(0, 0.8, a=9 / 490)
    w1 = ph.interface_width(e1, 0.1)
    assert ph.interface_width(e1, 0.4) == pytest.approx(2 * w1, rel=1e-9)
    assert ph.interface_width(e2, 0.1) == pytest.approx(math.sqrt(10) * w1, rel=1e-9)


@pytest.mark.parametrize("w", [inputs.DROP_D2Q9_64, inputs.DROP_D3Q27_128,
                               inputs.COALESCENCE_D3Q27_256, inputs.IMPACT_D3Q27_384])
def test_workload_constants_match_maxwell(w):
    """The stored init densities and kappa of each workload come from the EOS."""
    e = EOS(w.eos, w.t_over_tc, a=w.a, b=w.b)
    rv, rl, ps = ph.maxwell(e)
    assert w.rho_v == pytest.approx(rv, rel=1e-8)
    assert w.rho_l == pytest.approx(rl, rel=1e-8)
    assert w.kappa == pytest.approx(ph.kappa_for_width(e, 5.0, (rv, rl, ps)), rel=1e-5)
