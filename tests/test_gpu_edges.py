"""Degenerate and boundary cases of the GPU path: zero steps, a lattice with
no fluid node, the smallest lattices the 2-ring stencils allow (5 nodes a
side) against the oracle, and a uniform state at rest, which the method
leaves unchanged."""
import numpy as np
import pytest

from oracle.lbm import OracleLBM
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


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_zero_steps_change_nothing(lbm, storage):
    w = inputs.DROP_D3Q27_128
    g = lbm.LBM(1, 20, 18, 16, w.eos, w.t_over_tc, w.kappa, 1.0, a=w.a, b=w.b, storage=storage)
    g.init(inputs.drop(20, 18, 16, 5.0, w.rho_v, w.rho_l))
    f0 = g.get_populations()
    g.step(0)
    g.sync()
    assert np.array_equal(g.get_populations(), f0)


@pytest.mark.parametrize("storage", [0, 1])
def test_all_solid_lattice(lbm, storage):
    w = inputs.DROP_D2Q9_64
    mask = np.ones(8 * 6, np.uint8)
    g = lbm.LBM(0, 8, 6, 1, w.eos, w.t_over_tc, w.kappa, 1.0, a=w.a, b=w.b, mask=mask,
                rho_w=w.rho_v, storage=storage)
    g.init(np.full(48, w.rho_v))
    g.step(10)
    m, j = g.reduce()
    assert m == 0.0 and np.all(j == 0.0)
    rho, u, U = g.moments()
    assert np.all(rho == w.rho_v) and np.all(u == 0.0) and np.all(U == 0.0)


@pytest.mark.parametrize("lattice", [0, 1])
def test_smallest_lattice_parity(lbm, lattice):
    w = inputs.DROP_D3Q27_128 if lattice == 1 else inputs.DROP_D2Q9_64
    nz = 5 if lattice == 1 else 1
    rho = inputs.add_noise(inputs.drop(5, 5, nz, 1.5, w.rho_v, w.rho_l), 1e-3, 101)
    g = lbm.LBM(lattice, 5, 5, nz, w.eos, w.t_over_tc, w.kappa, 1.0, a=w.a, b=w.b)
    o = OracleLBM(lattice, 5, 5, nz, w.eos, w.t_over_tc, w.kappa, 1.0, a=w.a, b=w.b)
    g.init(rho)
    o.init(rho)
    g.step(100)
    o.step(100)
    rg, ro = g.moments()[0], o.moments()[0]
    assert np.max(np.abs(rg - ro) / ro) < 1e-10
    g32 = lbm.LBM(lattice, 5, 5, nz, w.eos, w.t_over_tc, w.kappa, 1.0, a=w.a, b=w.b, storage=lbm.F32)
    g32.init(rho)
    g32.step(100)
    assert np.max(np.abs(g32.moments()[0] - ro) / ro) < 5e-3


@pytest.mark.parametrize("storage,tol", [(0, 1e-13), (1, 1e-5), (2, 1e-3), (3, 1e-2)])
def test_uniform_state_at_rest_stays(lbm, storage, tol):
    """A uniform state at rest has no force and no correction: over 50 steps
    it changes only by rounding (each step recomputes f_eq(rho, 0) from the
    rounded sum rho of its populations, a few units in the last place)."""
    w = inputs.DROP_D3Q27_128
    g = lbm.LBM(1, 33, 12, 10, w.eos, w.t_over_tc, w.kappa, 0.8, a=w.a, b=w.b, storage=storage)
    g.init(np.full(33 * 12 * 10, w.rho_l))
    f0 = g.get_populations()
    g.step(50)
    f1 = g.get_populations()
    assert np.max(np.abs(f1 - f0)) <= tol * np.max(np.abs(f0))
    m, j = g.reduce()
    assert np.all(np.abs(j) < 1e-9 * m)


def test_fp64_probe_measures_a_plausible_rate(lbm):
    """The FP64 FMA-chain probe (the FP64 roofline's denominator) reports a
    rate between a tenth and three times GB300's nominal 1.25 TFLOP/s, and
    two runs agree within 10 %."""
    a = lbm.probe_fp64_tflops()
    b = lbm.probe_fp64_tflops()
    assert 0.125 < a < 3.75, a
    assert abs(a - b) < 0.1 * max(a, b), (a, b)


def test_bounded_wait_runs_out_and_returns(lbm):
    """The fused kernels' bounded wait, made to run out on a barrier phase
    that nothing completes (2e6 cycles, about a millisecond): every waiting
    warp records the timeout in the status word and the kernel returns; the
    context stays usable (a step on a fresh lattice afterwards is fine)."""
    st, ms = lbm.selftest_wait_timeout(2_000_000)
    assert st == 2, st
    assert 0.0 < ms < 200.0, ms
    w = inputs.DROP_D3Q27_128
    g = lbm.LBM(1, 24, 20, 16, w.eos, w.t_over_tc, w.kappa, 1.0, a=w.a, b=w.b, storage=1)
    g.init(inputs.drop(24, 20, 16, 5.0, w.rho_v, w.rho_l))
    g.step(4)
    g.sync()
