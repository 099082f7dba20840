"""Density-dependent relaxation time (the vapour/liquid viscosity ratio of
the paper's Sec. 5.2 and of Sec. 4.1 configuration (b)) on the GPU.

- Parity with the oracle, FP64 to 1e-10 and FP32 at its storage tolerance,
  on a D2Q9 and a D3Q27 drop with tau_v != tau.
- Layered Poiseuille flow, configuration (b) (vdW T/Tc 0.36, density ratio
  1.2e3, mu_l / mu_v = 11.3, so nu_v = 109 nu_l: tau 0.52 and 2.68) on the
  paper's 200-row channel, mirrored with liquid films on both walls: the
  steady velocity (FP64) follows the momentum balance of the simulated
  density and viscosity profile within 1 % (measured 0.08 %) and the
  sharp-interface layer solution within 5 % (measured 2.1 %). FP32 storage
  is not asserted here: with the liquid at tau 0.52 (omega 1.92, rounding
  noise barely damped) and a drive of 1e-7, it runs 14 % off FP64.
"""
import numpy as np
import pytest

from conftest import printed
from oracle import physics as ph
from oracle.lbm import EOS, OracleLBM
from paper_2112_01975_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_01975_gb300 import build
    build.build()
    from paper_2112_01975_gb300 import lbm as L
    return L


def _errs(g, o):
    rg, ug, Ug = g.moments()
    ro, uo, Uo, _ = o.moments()
    er = float(np.max(np.abs(rg - ro) / ro))
    scale = max(float(np.max(np.abs(uo))), float(np.max(np.abs(Uo))))
    return er, float(np.max(np.abs(Ug - Uo))) / scale


@pytest.mark.parametrize("lattice", [0, 1])
@pytest.mark.parametrize("storage,rtol,utol", [(0, 1e-10, 1e-10), (1, 5e-3, 5e-3)])
def test_variable_viscosity_parity(lbm, lattice, storage, rtol, utol):
    if lattice == 0:
        w = inputs.DROP_D2Q9_64
        shape = (64, 64, 1)
        rho = inputs.add_noise(inputs.drop(64, 64, 1, 14.0, w.rho_v, w.rho_l), 1e-4, 71)
    else:
        w = inputs.DROP_D3Q27_128
        shape = (32, 30, 28)
        rho = inputs.add_noise(inputs.drop(*shape, 8.0, w.rho_v, w.rho_l), 1e-4, 72)
    kw = dict(a=w.a, b=w.b, tau_v=1.3, visc_rho=(w.rho_v, w.rho_l))
    g = lbm.LBM(lattice, *shape, w.eos, w.t_over_tc, w.kappa, 0.7, storage=storage, **kw)
    o = OracleLBM(lattice, *shape, w.eos, w.t_over_tc, w.kappa, 0.7, **kw)
    g.init(rho)
    o.init(rho)
    g.step(300)
    o.step(300)
    er, eU = _errs(g, o)
    assert er < rtol and eU < utol, (er, eU)


def test_layered_poiseuille_viscosity_ratio_200_rows(lbm):
    tr, H, tau_l, grav = 0.36, 200, 0.52, 1e-7
    a0 = 9 / 49
    e0 = EOS(0, tr, a=a0)
    _, rl0, _ = ph.maxwell(e0)
    h = 1e-6 * rl0
    a = a0 * min(1.0, 0.1 / ((e0(rl0 + h) - e0(rl0 - h)) / (2 * h)))
    e = EOS(0, tr, a=a)
    rv, rl, ps = ph.maxwell(e)
    kap = ph.kappa_for_width(e, 5.0, (rv, rl, ps))
    nu_l = (tau_l - 0.5) / 3.0
    nu_v = nu_l * (rl / rv) / printed("layered_poiseuille_b")["viscosity_ratio"]   # mu_l / mu_v
    nx, ny, hl = 5, H + 2, H // 4
    mask = np.zeros((ny, nx), np.uint8)
    mask[0] = mask[-1] = 1
    yp = np.arange(ny) - 0.5
    rho = np.repeat(inputs.tanh_interface(np.minimum(yp, H - yp) - hl, rl, rv, 5.0), nx)
    rho[mask.ravel() == 1] = rl
    g = lbm.LBM(0, nx, ny, 1, 0, tr, kap, tau_l, a=a, mask=mask.ravel(), rho_w=rl,
                g=(grav, 0.0), tau_v=0.5 + 3 * nu_v, visc_rho=(rv, rl))
    g.init(rho)
    g.step(int(3 * hl * hl / nu_l))
    r, _, U = g.moments()
    rr, U64 = r.reshape(ny, nx)[1:-1, 2], U[: g.N].reshape(ny, nx)[1:-1, 2]
    nu = nu_l + (nu_v - nu_l) * np.clip((rl - rr) / (rl - rv), 0.0, 1.0)
    Ud = ph.channel_flow_from_profile(rr, grav, nu)
    ys = np.arange(1, H + 1) - 0.5
    us = ph.layered_poiseuille([(hl, rl, rl * nu_l), (H / 2 - hl, rv, rv * nu_v)], grav,
                               top="symmetry")(np.minimum(ys, H - ys))
    e_d = np.max(np.abs(U64 - Ud)) / Ud.max()
    e_s = np.max(np.abs(U64 - us)) / us.max()
    assert e_d < 0.01 and e_s < 0.05, (e_d, e_s)
