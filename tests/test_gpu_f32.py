"""FP32 storage with the fused FP32 step, against the FP64 CPU oracle.

Tolerances: the stated accuracy of FP32 storage is coexistence densities
within 0.5 % of FP64, so densities are compared node by node at 5e-3 of
rho. FP32 rounds at 6e-8; one node update chains a few hundred operations
and the force, a sum of differences of O(1) numbers, loses about three
digits to cancellation, so a relaxing drop stays near 5e-5 (D2Q9, 1000
steps) while a vapour slab at 1/145 of the liquid density with a wall and
noise reaches 2.6e-3 in the vapour. Velocities are compared at 5e-3 of the
field's max |u|; the physical U = u + F/(2 rho) (Sec. 2.3.5), a sum whose two
terms nearly cancel in a resting state, at 5e-3 of the larger of max |u| and
max |U|. One step from an identical state is compared at 2e-6 of
max f.
"""
import numpy as np
import pytest

from oracle.lbm import OracleLBM
from paper_2112_01975_gb300 import inputs

pytestmark = pytest.mark.gpu

RHO_TOL = 5e-3
U_TOL = 5e-3


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_01975_gb300 import build
    build.build()
    from paper_2112_01975_gb300 import lbm as L
    return L


def errs(g, o, mask=None):
    rg, ug, Ug = g.moments()
    ro, uo, Uo, _ = o.moments()
    fl = np.ones(g.N, bool) if mask is None else (mask == 0)
    fl2 = np.tile(fl, g.D)
    er = float(np.max(np.abs(rg[fl] - ro[fl]) / ro[fl]))
    eu = float(np.max(np.abs(ug[fl2] - uo[fl2]))) / max(float(np.max(np.abs(uo[fl2]))), 1e-12)
    # U = u + F/(2 rho) cancels near rest: its rounding scales with its terms
    scale = max(float(np.max(np.abs(Uo[fl2]))), float(np.max(np.abs(uo[fl2]))), 1e-12)
    eU = float(np.max(np.abs(Ug[fl2] - Uo[fl2]))) / scale
    return er, eu, eU


def pair(L, lattice, nx, ny, nz, w, tau, mask=None, rho_w=1.0):
    g = L.LBM(lattice, nx, ny, nz, w.eos, w.t_over_tc, w.kappa, tau, mask=mask, a=w.a, b=w.b,
              rho_w=rho_w, storage=L.F32)
    o = OracleLBM(lattice, nx, ny, nz, w.eos, w.t_over_tc, w.kappa, tau, mask=mask, a=w.a,
                  b=w.b, rho_w=rho_w)
    return g, o


def test_f32_d2q9_drop_1000_steps(lbm):
    w = inputs.DROP_D2Q9_64
    g, o = pair(lbm, 0, 64, 64, 1, w, w.tau)
    r = w.rho0()
    g.init(r)
    o.init(r)
    g.step(1000)
    o.step(1000)
    er, eu, eU = errs(g, o)
    assert er < RHO_TOL and eu < U_TOL and eU < U_TOL, (er, eu, eU)


def test_f32_d3q27_mask_ragged_1000_steps(lbm):
    """nx = 150: four 32-wide tiles and a ragged one; solid block in the vapour."""
    w = inputs.DROP_D3Q27_128
    nx, ny, nz = 150, 7, 6
    mask = inputs.block_mask(nx, ny, nz, (125, 0, 0), (135, 3, 6))
    rho = inputs.add_noise(inputs.slab(nx, ny, nz, 30, 110, w.rho_v, w.rho_l), 1e-4, 21)
    g, o = pair(lbm, 1, nx, ny, nz, w, 0.8, mask=mask, rho_w=w.rho_v)
    g.init(rho)
    o.init(rho)
    g.step(1000)
    o.step(1000)
    er, eu, eU = errs(g, o, mask)
    assert er < RHO_TOL and eu < U_TOL and eU < U_TOL, (er, eu, eU)


@pytest.mark.parametrize("shape,tau", [((21, 19, 17), 0.7), ((37, 13, 9), 1.0)])
def test_f32_d3q27_small_odd_sizes(lbm, shape, tau):
    """Tiles wider than the lattice (x halo wraps several times) and odd sizes."""
    w = inputs.DROP_D3Q27_128
    nx, ny, nz = shape
    rho = inputs.add_noise(inputs.drop(nx, ny, nz, min(shape) / 3, w.rho_v, w.rho_l), 1e-4, 7)
    u0 = 0.01 * inputs.uniform_pm1(8, 3 * nx * ny * nz)
    g, o = pair(lbm, 1, nx, ny, nz, w, tau)
    g.init(rho, u0)
    o.init(rho, u0)
    g.step(500)
    o.step(500)
    er, eu, eU = errs(g, o)
    assert er < RHO_TOL and eu < U_TOL and eU < U_TOL, (er, eu, eU)


def test_f32_minimum_size(lbm):
    w = inputs.DROP_D3Q27_128
    rho = inputs.add_noise(np.full(125, 2.0), 1e-2, 9)
    u0 = 0.05 * inputs.uniform_pm1(10, 375)
    g, o = pair(lbm, 1, 5, 5, 5, w, 0.9)
    g.init(rho, u0)
    o.init(rho, u0)
    g.step(100)
    o.step(100)
    rg, ug, _ = g.moments()
    ro, uo, _, _ = o.moments()
    assert np.max(np.abs(rg - ro) / ro) < RHO_TOL
    assert np.max(np.abs(ug - uo)) < 1e-5        # the flow has decayed: absolute


def test_f32_full_size_single_step(lbm):
    """128^3 benchmark workload: one FP32 step from the GPU's own state against
    one FP64 oracle step from the same (widened) state."""
    w = inputs.DROP_D3Q27_128
    g, o = pair(lbm, 1, w.nx, w.ny, w.nz, w, w.tau)
    g.init(w.rho0())
    g.step(20)
    o.set_populations(g.get_populations())
    g.step(1)
    o.step(1)
    fg = g.get_populations()
    fo = o.get_populations()
    assert float(np.max(np.abs(fg - fo))) < 2e-6 * float(np.max(np.abs(fo)))


def test_f32_mass_drift(lbm):
    w = inputs.DROP_D3Q27_128
    g = lbm.LBM(1, w.nx, w.ny, w.nz, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b,
                storage=lbm.F32)
    g.init(w.rho0())
    m0, _ = g.reduce()
    g.step(500)
    m1, _ = g.reduce()
    assert abs(m1 - m0) / m0 < 1e-5


def test_f32_chunking_and_graph_do_not_change_results(lbm):
    w = inputs.DROP_D3Q27_128
    g = lbm.LBM(1, 64, 40, 48, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b,
                storage=lbm.F32)
    g.init(inputs.add_noise(inputs.drop(64, 40, 48, 12.0, w.rho_v, w.rho_l), 1e-4, 4))
    g.step(3)
    f0 = g.get_populations()
    outs = []
    for chunk in (1, 5, 16, 48):
        g.set_populations(f0)
        g.set_chunk(chunk)
        g.step(9)                  # graph replays plus a plain step
        outs.append(g.get_populations())
    g.set_populations(f0)
    for _ in range(9):
        g.step(1)                  # plain launches only
    outs.append(g.get_populations())
    for x in outs[1:]:
        assert np.array_equal(outs[0], x)


@pytest.mark.parametrize("shape,chunk,solid", [((64, 40, 48), 16, False), ((45, 37, 29), 7, True),
                                              ((128, 128, 128), 32, False)])
def test_f32_seven_row_tiles_do_not_change_results(lbm, shape, chunk, solid):
    """32 x 7 tiles (ragged in y, with and without solids, and the 128^3
    bench lattice at its one-wave chunk) give bitwise the populations of the
    default 32 x 8 tiles, through graph replays and plain launches."""
    w = inputs.DROP_D3Q27_128
    nx, ny, nz = shape
    mask = None
    if solid:
        mask = np.zeros(nx * ny * nz, dtype=np.uint8)
        z = np.arange(nx * ny * nz) // (nx * ny)
        mask[z == 0] = 1
    g = lbm.LBM(1, nx, ny, nz, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b,
                storage=lbm.F32, mask=mask, rho_w=w.rho_v)
    g.init(inputs.add_noise(inputs.drop(nx, ny, nz, nx / 5.0, w.rho_v, w.rho_l), 1e-4, 5))
    g.set_chunk(chunk)
    g.step(3)
    f0 = g.get_populations()
    assert g.tile() == (32, 8)
    g.step(9)
    f8 = g.get_populations()
    g.set_populations(f0)
    g.set_tile(7)
    assert g.tile() == (32, 7)
    g.step(8)                      # graph replays
    g.step(1)                      # and a plain launch
    assert np.array_equal(g.get_populations(), f8)


@pytest.mark.parametrize("shape,chunk,solid", [((128, 40, 48), 16, True), ((36, 20, 24), 5, True),
                                              ((96, 64, 33), 1, False)])
def test_f32_tma_staged_form_is_bitwise_the_plain_form(lbm, shape, chunk, solid):
    """The TMA-staged form (each entering plane's halo box copied into shared
    memory two planes ahead; nodes whose halo coordinates wrap read from
    global memory) gives bitwise the populations of the plain form: tiles
    whose box lies inside the lattice (128 x 40), ragged tiles that all
    touch the lattice's edges (36 x 20), chunks of one plane, a solid
    bottom plane with pillars, graph replays and a plain launch."""
    w = inputs.DROP_D3Q27_128
    nx, ny, nz = shape
    mask = None
    if solid:
        mask = inputs.pillar_mask(nx, ny, nz, 2, 4, 6)
    g = lbm.LBM(1, nx, ny, nz, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b,
                storage=lbm.F32, mask=mask, rho_w=w.rho_v)
    g.init(inputs.add_noise(inputs.drop(nx, ny, nz, min(nx, ny, nz) / 4.0, w.rho_v, w.rho_l), 1e-4, 7))
    g.set_chunk(chunk)
    g.step(3)
    f0 = g.get_populations()
    g.step(9)
    ref = g.get_populations()
    g.set_populations(f0)
    g.set_fused_variant(lbm.FUSED_WS_TMA)
    assert g.fused_variant == lbm.FUSED_WS_TMA
    g.step(8)                      # graph replays
    g.step(1)                      # and a plain launch
    assert np.array_equal(g.get_populations(), ref)


def test_f32_tma_staged_form_rejects_other_cases(lbm):
    """Rows not 16-byte aligned (nx not a multiple of 4 for FP32, of 8 for
    16-bit shifted storage), D2Q9, FP64 storage and 7-row tiles have no
    TMA-staged form."""
    w = inputs.DROP_D3Q27_128
    for nx, lattice, storage in ((37, 1, lbm.F32), (64, 0, lbm.F32), (60, 1, lbm.F16S), (64, 1, lbm.F64)):
        g = lbm.LBM(lattice, nx, 16 if lattice else 64, 12 if lattice else 1, w.eos, w.t_over_tc,
                    w.kappa, w.tau, a=w.a, b=w.b, storage=storage)
        with pytest.raises(lbm.LBMError):
            g.set_fused_variant(lbm.FUSED_WS_TMA)
    g = lbm.LBM(1, 64, 16, 12, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b, storage=lbm.F32)
    with pytest.raises(lbm.LBMError):   # the one-group TMA-staged form is one of shifted storage
        g.set_fused_variant(lbm.FUSED_TM_TMA)
    g.set_tile(7)
    with pytest.raises(lbm.LBMError):
        g.set_fused_variant(lbm.FUSED_WS_TMA)
    g.set_tile(8)
    g.set_fused_variant(lbm.FUSED_WS_TMA)
    with pytest.raises(lbm.LBMError):
        g.set_tile(7)


def test_f32_tile_setter_rejects_other_cases(lbm):
    w = inputs.DROP_D3Q27_128
    g = lbm.LBM(1, 32, 16, 12, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b, storage=lbm.F32)
    for bad in (6, 9, 0):
        with pytest.raises(lbm.LBMError):
            g.set_tile(bad)
    h = lbm.LBM(1, 32, 16, 12, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b, storage=lbm.F16S)
    with pytest.raises(lbm.LBMError):
        h.set_tile(7)
    assert h.tile() == (32, 8)
    d = lbm.LBM(0, 64, 64, 1, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b, storage=lbm.F32)
    assert d.tile() == (128, 1)
    with pytest.raises(lbm.LBMError):
        d.set_tile(7)


def test_f32_population_io_roundtrip(lbm):
    import torch
    w = inputs.DROP_D2Q9_64
    g = lbm.LBM(0, 64, 64, 1, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b,
                storage=lbm.F32)
    g.init(w.rho0())
    g.step(5)
    f = g.get_populations()
    assert np.array_equal(f.astype(np.float32).astype(np.float64), f)
    fd = torch.empty(9 * g.N, dtype=torch.float64, device="cuda")
    g.get_populations(fd)
    assert np.array_equal(fd.cpu().numpy(), f)
    g.set_populations(fd)
    assert np.array_equal(g.get_populations(), f)


def test_f32_coexistence_within_half_percent_of_fp64(lbm):
    """Flat interface (Sec. 3.1 setup, scaled down): FP32 coexistence densities
    within 0.5 % of the FP64 oracle's."""
    from oracle import physics as ph
    from oracle.lbm import EOS
    a = 9 / 490
    e = EOS(0, 0.8, a=a)
    rv, rl, ps = ph.maxwell(e)
    kap = ph.kappa_for_width(e, 5.0, (rv, rl, ps))
    nx = 128
    rho = inputs.slab(nx, 5, 1, 32, 96, rv, rl, 5.0)
    g = lbm.LBM(0, nx, 5, 1, 0, 0.8, kap, 1.0, a=a, storage=lbm.F32)
    o = OracleLBM(0, nx, 5, 1, 0, 0.8, kap, 1.0, a=a)
    g.init(rho)
    o.init(rho)
    g.step(4500)
    o.step(4500)
    r32 = g.moments()[0].reshape(5, nx)[2]
    r64 = o.moments()[0].reshape(5, nx)[2]
    assert abs(r32[0] / r64[0] - 1) < 5e-3
    assert abs(r32[64] / r64[64] - 1) < 5e-3



def test_f32_autotune_keeps_the_state(lbm):
    w = inputs.DROP_D3Q27_128
    g = lbm.LBM(1, 64, 48, 40, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b,
                storage=lbm.F32)
    g.init(inputs.add_noise(inputs.drop(64, 48, 40, 10.0, w.rho_v, w.rho_l), 1e-4, 6))
    g.step(4)
    f0 = g.get_populations()
    chunk = g.autotune()
    assert 1 <= chunk <= 128
    assert np.array_equal(g.get_populations(), f0)
    g.step(6)
    g.sync()


@pytest.fixture(scope="module")
def pillar_oracle():
    """The 32^3 pillar case on the oracle, 1000 steps (once for the module)."""
    from test_gpu_parity import _pillar_case
    w, n, mask, rho = _pillar_case()
    kw = dict(mask=mask, a=w.a, b=w.b, rho_w=w.rho_v)
    try:   # the -fopenmp build: bitwise the plain oracle, on all host cores
        o = OracleLBM(1, n, n, n, w.eos, w.t_over_tc, w.kappa, 0.8, openmp=True, **kw)
    except Exception:
        o = OracleLBM(1, n, n, n, w.eos, w.t_over_tc, w.kappa, 0.8, **kw)
    o.init(rho)
    o.step(1000)
    return w, n, mask, rho, o


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_f32_pr_pillars_32cubed_1000_steps(lbm, pillar_oracle, variant):
    """The 32^3 pillar case of the FP64 parity tests (a wall with 4x4x6
    pillars, a Peng-Robinson drop above them) in FP32 storage, with each form
    of the fused step (plain, warp-specialised, Tensor Memory, both, and
    both with TMA-staged planes), against the FP64 oracle after 1000 steps
    at the FP32 tolerances; the five forms agree bitwise."""
    w, n, mask, rho, o = pillar_oracle

    def run(var):
        g = lbm.LBM(1, n, n, n, w.eos, w.t_over_tc, w.kappa, 0.8, mask=mask, a=w.a, b=w.b,
                    rho_w=w.rho_v, storage=lbm.F32)
        g.set_fused_variant(var)
        g.init(rho)
        g.step(1000)
        return g

    g = run(variant)
    er, eu, eU = errs(g, o, mask)
    assert er < RHO_TOL and eu < U_TOL and eU < U_TOL, (er, eu, eU)
    if variant:
        assert np.array_equal(run(0).get_populations(), g.get_populations())
