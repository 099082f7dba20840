"""The two largest workloads at full size, compared with the oracle at
sampled nodes (the full CPU oracle cannot step lattices of 16.8 M and
37.7 M nodes in test time).

For each sampled node, the oracle computes its post-collision populations
from its 5x5x5 neighbourhood in the GPU's state (oracle_post_local, pinned
to the full oracle step on CPU); the GPU's next state must hold them where
the push step puts them (the neighbour in direction c_i, or the node itself
after a bounce-back). Samples: seeded random nodes, nodes inside the
interface, fluid nodes next to a solid and contact-line nodes (interface
nodes next to a solid).

Workloads: two touching drops of radius 40 in a periodic 256^3 box at
Peng-Robinson T/Tc = 0.45 (coalescence, density ratio 6.6e4); a drop of
radius 60 moving down at U = 0.115 (We = rho_l U^2 D / sigma = 100) onto a
two-plane wall with 8x8x16 pillars at pitch 16 in a 384x384x256 box at
T/Tc = 0.5 (impact, density ratio 1.1e4). Both at nu = 0.075 (tau = 0.725),
interface width 5, started at rest in the physical velocity.
"""
import numpy as np
import pytest

from oracle import sample
from oracle.lbm import OracleLBM
from paper_2112_01975_gb300 import eos_tables, inputs

pytestmark = pytest.mark.gpu

# one step from an identical state, of max |f|: FP64, FP32, FP16-, BF16-shifted
STEP_TOL = {0: 1e-12, 1: 2e-6, 2: 2e-4, 3: 2e-3}
MASS_TOL = {0: 1e-12, 1: 1e-5, 2: 1e-4, 3: 1e-3}
W, TAU = 5.0, 0.725


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_01975_gb300 import build
    build.build()
    from paper_2112_01975_gb300 import lbm as L
    return torch, L


def pr_state(t_over_tc):
    a = eos_tables.stable_a(1, t_over_tc)
    rv, rl, _ = eos_tables.coexistence(1, t_over_tc, a)
    return a, rv, rl, eos_tables.kappa_for_width(1, t_over_tc, a, width=W)


def _pick(rng, idx, count, shape):
    nz, ny, nx = shape
    return [(int(n % nx), int((n // nx) % ny), int(n // (nx * ny)))
            for n in rng.choice(idx, size=min(count, idx.size), replace=False)]


def samples(shape, rho, mask, seed, count=24):
    """Node coordinates: random, in the interface, next to solids, on the
    contact line. Solid nodes are left out (they are never collided)."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    fluid = np.ones(rho.size, bool) if mask is None else mask == 0
    pts = _pick(rng, np.flatnonzero(fluid), count, shape)
    band = (rho > 0.1) & (rho < 5.0) & fluid
    pts += _pick(rng, np.flatnonzero(band), count, shape)
    if mask is not None:
        m3 = mask.reshape(nz, ny, nx).astype(bool)
        near = np.zeros_like(m3)
        for ax in range(3):
            near |= np.roll(m3, 1, axis=ax) | np.roll(m3, -1, axis=ax)
        near = near.ravel() & fluid
        pts += _pick(rng, np.flatnonzero(near), count, shape)
        pts += _pick(rng, np.flatnonzero(near & band), count, shape)
    return pts


def check_sampled_step(torch, g, o, shape, mask, pts, tol):
    """One GPU step against the oracle's node-local update at pts."""
    N, Q = g.N, g.Q
    f0 = torch.empty(Q * N, dtype=torch.float64, device="cuda")
    g.get_populations(f0)
    f0 = f0.view(Q, N)
    _, c = o.weights()
    blocks = [sample.block_indices(shape, x, y, z, 3) for (x, y, z) in pts]
    bidx = torch.from_numpy(np.stack(blocks)).cuda()
    bvals = f0[:, bidx].permute(1, 2, 0).cpu().numpy()        # [sample][125][Q]
    fmax = float(f0.abs().max())
    del f0
    g.step(1)
    f1 = torch.empty(Q * N, dtype=torch.float64, device="cuda")
    g.get_populations(f1)
    f1 = f1.view(Q, N)
    pushed = [sample.pushed_indices(shape, x, y, z, c, mask) for (x, y, z) in pts]
    pj = torch.tensor([[j for j, _ in p] for p in pushed], device="cuda")
    pd = torch.tensor([[d for _, d in p] for p in pushed], device="cuda")
    got = f1[pj, pd].cpu().numpy()                             # [sample][Q]
    del f1
    mask_np = mask if mask is not None else np.zeros(N, np.uint8)
    worst = 0.0
    for s, blk in enumerate(blocks):
        want = o.post_local(bvals[s], mask_np[blk])
        worst = max(worst, float(np.max(np.abs(got[s] - want))))
    assert worst < tol * fmax, (worst, fmax)


@pytest.mark.parametrize("storage", [0, 1, 2, 3])
def test_coalescence_256cubed(env, storage):
    torch, L = env
    n, R, tr = 256, 40.0, 0.45
    a, rv, rl, kap = pr_state(tr)
    assert 6e4 < rl / rv < 7e4
    shape = (n, n, n)
    centres = [(n // 2 - R, n // 2, n // 2), (n // 2 + R, n // 2, n // 2)]
    rho = inputs.add_noise(inputs.drops(n, n, n, centres, R, rv, rl, width=W), 1e-4, 3)
    g = L.LBM(1, n, n, n, 1, tr, kap, TAU, a=a, storage=storage)
    g.init(rho)
    m0, _ = g.reduce()
    g.step(300)
    m1, _ = g.reduce()
    assert abs(m1 / m0 - 1) < MASS_TOL[storage]
    rho_now = g.moments()[0]
    assert rho_now.min() > 0.5 * rv and rho_now.max() < 1.1 * rl
    # the neck has grown: liquid on the line between the centres at the contact point
    assert rho_now[n // 2 + n * (n // 2 + n * (n // 2))] > 0.5 * rl
    o = OracleLBM(1, 5, 5, 5, 1, tr, kap, TAU, a=a)
    check_sampled_step(torch, g, o, shape, None, samples(shape, rho_now, None, 3),
                       STEP_TOL[storage])
    g.sync()
    g.close()


def test_impact_on_pillars_384x384x256(env):
    """The impact workload (inputs.IMPACT_D3Q27_384: a two-plane wall with
    8x8x16 pillars, a drop of radius 60 at We = 100) in FP32 for 300 steps:
    mass, bounds, contact with the pillar tops, sampled nodes against the
    oracle's node-local update."""
    torch, L = env
    w = inputs.IMPACT_D3Q27_384
    nx, ny, nz = w.nx, w.ny, w.nz
    shape = (nz, ny, nx)
    rho, u0, mask = w.fields()
    rv, rl = w.rho_v, w.rho_l
    g = L.LBM(1, nx, ny, nz, w.eos, w.t_over_tc, w.kappa, w.tau, mask=mask, a=w.a, b=w.b,
              rho_w=w.rho_w, storage=L.F32)
    g.init(rho, u0)
    m0, _ = g.reduce()
    g.step(300)      # the drop's front reaches the pillar tops after ~70 steps
    m1, _ = g.reduce()
    assert abs(m1 / m0 - 1) < MASS_TOL[1]
    rho_now = g.moments()[0]
    assert rho_now[mask == 0].min() > 0.02 * rv and rho_now.max() < 1.1 * rl
    # liquid on the plane just above the pillar tops, under the drop: contact
    zt = w.wall + w.pillar[1]
    top = rho_now.reshape(nz, ny, nx)[zt, ny // 2 - 16:ny // 2 + 16, nx // 2 - 16:nx // 2 + 16]
    assert top.max() > 0.5 * rl
    o = OracleLBM(1, 5, 5, 5, w.eos, w.t_over_tc, w.kappa, w.tau, a=w.a, b=w.b, rho_w=w.rho_w)
    check_sampled_step(torch, g, o, shape, mask, samples(shape, rho_now, mask, 4), STEP_TOL[1])
    g.sync()
    g.close()
