"""GPU (CUDA, through the C ABI) against the FP64 CPU oracle on the same
seeded inputs. Tolerance: max relative density error <= 1e-10 and max
velocity error <= 1e-10 of the field's max |u| (both FP64, differences come
only from summation order and fused multiply-adds)."""
import numpy as np
import pytest

from oracle.lbm import OracleLBM
from paper_2112_01975_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_01975_gb300 import build
    build.build()
    from paper_2112_01975_gb300 import lbm as L
    return L


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def vel_err(a, b):
    scale = max(float(np.max(np.abs(b))), 1e-300)
    return float(np.max(np.abs(a - b))) / scale


def pair(L, lattice, nx, ny, nz, eos, tr, kappa, tau, a, b, mask=None, rho_w=1.0, flags=0):
    g = L.LBM(lattice, nx, ny, nz, eos, tr, kappa, tau, mask=mask, a=a, b=b, rho_w=rho_w,
              flags=flags)
    o = OracleLBM(lattice, nx, ny, nz, eos, tr, kappa, tau, mask=mask, a=a, b=b, rho_w=rho_w,
                  flags=flags)
    return g, o


def compare(g, o, mask=None):
    rg, ug, Ug = g.moments()
    ro, uo, Uo, _ = o.moments()
    fl = np.ones(g.N, bool) if mask is None else (mask == 0)
    fl2 = np.tile(fl, g.D)
    assert np.isfinite(rg).all()
    er = rel_err(rg[fl], ro[fl])
    eu = vel_err(ug[fl2], uo[fl2])
    eU = vel_err(Ug[fl2], Uo[fl2])
    return er, eu, eU


def test_d2q9_drop_64x64_1000_steps(lbm):
    w = inputs.DROP_D2Q9_64
    g, o = pair(lbm, 0, 64, 64, 1, w.eos, w.t_over_tc, w.kappa, w.tau, w.a, w.b)
    rho0 = w.rho0()
    g.init(rho0)
    o.init(rho0)
    rg, ug, _ = g.moments()
    ro, uo, _, _ = o.moments()
    assert rel_err(rg, ro) < 1e-14 and np.abs(ug - uo).max() < 1e-14   # u = 0 up to roundoff
    g.step(w.steps)
    o.step(w.steps)
    er, eu, eU = compare(g, o)
    assert er < TOL and eu < TOL and eU < TOL, (er, eu, eU)
    mg, jg = g.reduce()
    mo, jo = o.reduce()
    assert abs(mg - mo) / mo < 1e-13
    assert np.allclose(jg, jo, atol=1e-9 * mo)


def test_d3q27_pr_mask_ragged_1000_steps(lbm):
    """150 x 7 x 6: two 128-wide x tiles with a ragged tail, Peng-Robinson
    liquid slab, a solid block in the vapour with virtual wall density rho_v.
    (A block inside the liquid with rho_w = rho_v diverges in the oracle too.)"""
    w = inputs.DROP_D3Q27_128
    nx, ny, nz = 150, 7, 6
    mask = inputs.block_mask(nx, ny, nz, (125, 0, 0), (135, 3, 6))
    rho = inputs.add_noise(inputs.slab(nx, ny, nz, 30, 110, w.rho_v, w.rho_l), 1e-3, 21)
    rho = np.where(mask == 1, 1.0, rho)
    g, o = pair(lbm, 1, nx, ny, nz, w.eos, w.t_over_tc, w.kappa, 0.8, w.a, w.b, mask=mask,
                rho_w=w.rho_v)
    g.init(rho)
    o.init(rho)
    g.step(1000)
    o.step(1000)
    er, eu, eU = compare(g, o, mask)
    assert er < TOL and eu < TOL and eU < TOL, (er, eu, eU)


def _pillar_case():
    """D3Q27 32^3, Peng-Robinson T/Tc 0.7: a wall at z = 0 with 4x4x6
    pillars at pitch 8 (seeded offset), solid density rho_v, and a drop of
    radius 7 resting 3 nodes above the pillar tops (seeded noise)."""
    w = inputs.DROP_D3Q27_128
    n = 32
    mask = inputs.pillar_mask(n, n, n, side=4, height=6, pitch=8, seed=4)
    rho = inputs.add_noise(inputs.drop(n, n, n, 7.0, w.rho_v, w.rho_l, center=(16, 16, 16)), 1e-4, 23)
    return w, n, mask, np.where(mask == 1, w.rho_v, rho)


def test_d3q27_pr_pillars_32cubed_1000_steps(lbm):
    """The 32^3 pillar case in FP64 against the oracle after 1000 steps at
    1e-10, with mass conserved to 1e-13."""
    w, n, mask, rho = _pillar_case()
    g = lbm.LBM(1, n, n, n, w.eos, w.t_over_tc, w.kappa, 0.8, mask=mask, a=w.a, b=w.b, rho_w=w.rho_v)
    try:   # the -fopenmp build: bitwise the plain oracle, on all host cores
        o = OracleLBM(1, n, n, n, w.eos, w.t_over_tc, w.kappa, 0.8, mask=mask, a=w.a, b=w.b,
                      rho_w=w.rho_v, openmp=True)
    except Exception:
        o = OracleLBM(1, n, n, n, w.eos, w.t_over_tc, w.kappa, 0.8, mask=mask, a=w.a, b=w.b,
                      rho_w=w.rho_v)
    g.init(rho)
    o.init(rho)
    m0, _ = g.reduce()
    g.step(1000)
    o.step(1000)
    er, eu, eU = compare(g, o, mask)
    assert er < TOL and eu < TOL and eU < TOL, (er, eu, eU)
    m1, _ = g.reduce()
    assert abs(m1 / m0 - 1) < 1e-13


def test_d3q27_vdw_drop_odd_sizes_1000_steps(lbm):
    w = inputs.DROP_D2Q9_64
    nx, ny, nz = 21, 19, 17
    rho = inputs.add_noise(inputs.drop(nx, ny, nz, 5.0, w.rho_v, w.rho_l), 1e-4, 7)
    u0 = 0.01 * inputs.uniform_pm1(8, 3 * nx * ny * nz)
    g, o = pair(lbm, 1, nx, ny, nz, w.eos, w.t_over_tc, w.kappa, 0.7, w.a, w.b)
    g.init(rho, u0)
    o.init(rho, u0)
    g.step(1000)
    o.step(1000)
    er, eu, eU = compare(g, o)
    assert er < TOL and eu < TOL and eU < TOL, (er, eu, eU)


def test_minimum_size_5x5x5_with_flow(lbm):
    w = inputs.DROP_D2Q9_64
    rho = inputs.add_noise(np.full(125, 2.0), 1e-2, 9)
    u0 = 0.05 * inputs.uniform_pm1(10, 375)
    g, o = pair(lbm, 1, 5, 5, 5, w.eos, w.t_over_tc, w.kappa, 0.9, w.a, w.b)
    g.init(rho, u0)
    o.init(rho, u0)
    g.step(200)
    o.step(200)
    er, eu, eU = compare(g, o)
    assert er < TOL and eu < TOL and eU < TOL, (er, eu, eU)


def test_full_size_single_step_against_oracle(lbm):
    """128^3 Peng-Robinson drop (the benchmark workload): after 20 GPU steps,
    one more step from the GPU's own state is compared with one oracle step
    from that same state, on every node."""
    w = inputs.DROP_D3Q27_128
    g, o = pair(lbm, 1, w.nx, w.ny, w.nz, w.eos, w.t_over_tc, w.kappa, w.tau, w.a, w.b)
    g.init(w.rho0())
    g.step(20)
    f = g.get_populations()
    o.set_populations(f)
    g.step(1)
    o.step(1)
    fg = g.get_populations()
    fo = o.get_populations()
    assert float(np.max(np.abs(fg - fo) / np.abs(fo))) < 1e-12
    er, eu, eU = compare(g, o)
    assert er < 1e-13 and eu < 1e-11 and eU < 1e-11


def test_full_size_mass_conservation(lbm):
    w = inputs.DROP_D3Q27_128
    g = lbm.LBM(1, w.nx, w.ny, w.nz, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b)
    g.init(w.rho0())
    m0, _ = g.reduce()
    g.step(200)
    m1, _ = g.reduce()
    assert abs(m1 - m0) / m0 < 1e-12


def test_uniform_state_and_zero_steps(lbm):
    g = lbm.LBM(0, 16, 9, 1, 0, 0.8, 0.02, 1.0, a=9 / 490)
    g.init(np.full(144, 2.5))
    f0 = g.get_populations()
    g.step(0)
    assert np.array_equal(g.get_populations(), f0)
    g.step(25)
    assert np.abs(g.get_populations() - f0).max() < 1e-14


def test_graph_replay_equals_plain_steps_bitwise(lbm):
    w = inputs.DROP_D2Q9_64
    a = lbm.LBM(0, 64, 64, 1, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b)
    b = lbm.LBM(0, 64, 64, 1, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b)
    r = w.rho0()
    a.init(r)
    b.init(r)
    a.step(37)            # one plain + graph replays + one plain
    for _ in range(37):
        b.step(1)         # plain launches only
    assert np.array_equal(a.get_populations(), b.get_populations())


def test_runs_are_bitwise_reproducible(lbm):
    w = inputs.DROP_D3Q27_128
    out = []
    for _ in range(2):
        g = lbm.LBM(1, 40, 36, 33, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b)
        g.init(inputs.add_noise(inputs.drop(40, 36, 33, 10.0, w.rho_v, w.rho_l), 1e-4, 5))
        g.step(50)
        out.append((g.get_populations(), g.reduce()))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1][0] == out[1][1][0] and np.array_equal(out[0][1][1], out[1][1][1])


def test_device_and_host_io_agree(lbm):
    import torch
    w = inputs.DROP_D2Q9_64
    g = lbm.LBM(0, 64, 64, 1, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b)
    r = w.rho0()
    g.init(torch.from_numpy(r).cuda())
    g.step(10)
    rh, uh, Uh = g.moments()
    dev = tuple(torch.empty(n, dtype=torch.float64, device="cuda") for n in (g.N, 2 * g.N, 2 * g.N))
    g.moments(out=dev)
    assert np.array_equal(dev[0].cpu().numpy(), rh)
    assert np.array_equal(dev[1].cpu().numpy(), uh)
    assert np.array_equal(dev[2].cpu().numpy(), Uh)
    fd = torch.empty(9 * g.N, dtype=torch.float64, device="cuda")
    g.get_populations(fd)
    assert np.array_equal(fd.cpu().numpy(), g.get_populations())


def test_nonfinite_density_is_reported_and_blocks_steps(lbm):
    g = lbm.LBM(0, 16, 16, 1, 0, 0.8, 0.02, 1.0, a=9 / 490)
    r = np.full(256, 2.0)
    r[37] = np.nan
    g.init(r)
    g.step(1)
    with pytest.raises(lbm.LBMError) as e:
        g.sync(5000)
    assert e.value.code == 4
    with pytest.raises(lbm.LBMError) as e:
        g.step(1)
    assert e.value.code == 6
    g.init(np.full(256, 2.0))      # re-initialising clears the state
    g.step(3)
    g.sync(5000)


@pytest.mark.parametrize("storage", [0, 1])
def test_long_step_call_stops_at_a_nonfinite_density(lbm, storage):
    """lbm_step polls the status word every 64 steps: a NaN planted in the
    initial density (from the host) stops a 4000-step call within two
    polling intervals with LBM_ENONFINITE from lbm_step itself, and the
    launches after it are not issued."""
    g = lbm.LBM(0, 16, 16, 1, 0, 0.8, 0.02, 1.0, a=9 / 490, storage=storage)
    r = np.full(256, 2.0)
    r[37] = np.nan
    g.init(r)
    l0 = g.launches
    with pytest.raises(lbm.LBMError) as e:
        g.step(4000)
    assert e.value.code == 4
    per_step = 2 if storage == 0 else 1
    assert g.launches - l0 <= per_step * (3 * 64 + 2)
    with pytest.raises(lbm.LBMError) as e:
        g.step(1)
    assert e.value.code == 6
    g.init(np.full(256, 2.0))
    g.step(4000)                   # a healthy state runs through the polls
    g.sync(5000)
    assert g.launches - l0 >= per_step * 4000


def test_long_step_call_stops_in_the_tma_staged_form(lbm):
    """The same status polling with the TMA-staged FP32 step (D3Q27, the
    warp-specialised kernel whose waits are bounded): a NaN stops a
    4000-step call with LBM_ENONFINITE within two polling intervals."""
    g = lbm.LBM(1, 64, 16, 12, 0, 0.8, 0.02, 1.0, a=9 / 490, storage=lbm.F32)
    g.set_fused_variant(lbm.FUSED_WS_TMA)
    r = np.full(64 * 16 * 12, 2.0)
    r[5000] = np.nan
    g.init(r)
    assert g.fused_variant == lbm.FUSED_WS_TMA
    l0 = g.launches
    with pytest.raises(lbm.LBMError) as e:
        g.step(4000)
    assert e.value.code == 4
    assert g.launches - l0 <= 3 * 64 + 2
    g.init(np.full(64 * 16 * 12, 2.0))
    g.step(500)
    g.sync(5000)


def test_phi_off_flag_matches_oracle(lbm):
    from oracle.lbm import PHI_OFF
    nx = 64
    rho = (3.0 * (1 + 1e-3 * np.sin(2 * np.pi * np.arange(nx) / nx)))[None, :] * np.ones((5, 1))
    u = np.zeros((2, 5, nx))
    u[0] = 0.2
    g = lbm.LBM(0, nx, 5, 1, 0, 0.8, 0.02, 0.6, a=9 / 490, flags=lbm.FLAG_PHI_OFF)
    o = OracleLBM(0, nx, 5, 1, 0, 0.8, 0.02, 0.6, a=9 / 490, flags=PHI_OFF)
    g.init(rho.ravel(), u.ravel())
    o.init(rho.ravel(), u.ravel())
    g.step(300)
    o.step(300)
    er, eu, eU = compare(g, o)
    assert er < TOL and eu < TOL
