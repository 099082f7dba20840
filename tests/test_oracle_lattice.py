"""Pins of the oracle's lattice, product form, stencils and exact invariants.

Each check compares the oracle against something the paper or the
mathematics fixes independently of the oracle's own formulas: exact
rationals, moment identities of the product form (Appendix D), Taylor
exactness of the stencils on polynomials (Eqs. PPcond1-2, Ccond1-2), exact
conservation and symmetry of the update.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

from oracle.lbm import OracleLBM, ZETA_LITERAL
from paper_2112_01975_gb300 import inputs

RNG = np.random.default_rng(12345)


def small(lattice, n=8, **kw):
    nz = 1 if lattice == 0 else n
    kw.setdefault("kappa", 0.02)
    return OracleLBM(lattice, n, n, nz, 0, 0.8, kw.pop("kappa"), 1.0, a=9 / 490, **kw)


@pytest.mark.parametrize("lattice", [0, 1])
def test_weights_exact_rationals(lattice):
    """Eq. wi: products of 2/3 (c = 0) and 1/6 (c = +-1)."""
    o = small(lattice)
    w, c = o.weights()
    D = 2 if lattice == 0 else 3
    for wi, ci in zip(w, c):
        nz = int(np.count_nonzero(ci[:D]))
        exact = Fraction(2, 3) ** (D - nz) * Fraction(1, 6) ** nz
        assert wi == pytest.approx(float(exact), rel=4e-16, abs=0)
    if lattice == 0:
        assert sorted(set(np.round(w * 36).astype(int))) == [1, 4, 16]   # 1/36, 1/9, 4/9
    else:
        assert sorted(set(np.round(w * 216).astype(int))) == [1, 4, 16, 64]  # 1/216 .. 8/27


@pytest.mark.parametrize("lattice", [0, 1])
def test_weights_isotropy(lattice):
    """Lattice moments up to fourth order equal the isotropic Maxwellian ones at cs2 = 1/3."""
    o = small(lattice)
    w, c = o.weights()
    D = 2 if lattice == 0 else 3
    c = c[:, :D].astype(float)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(D) / 3, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(D)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(m4, iso, atol=1e-16)


@pytest.mark.parametrize("lattice", [0, 1])
def test_equilibrium_moments(lattice):
    """Eq. LBMeq with P0 = rho/3: sum f = rho, sum c f = rho u, sum c c f = P0 I + rho u u,
    and the D3Q27/D2Q9 bias sum c_a^3 f = sum c_a f (remark after Eq. LBMstar)."""
    o = small(lattice)
    _, c = o.weights()
    D = 2 if lattice == 0 else 3
    c = c[:, :D].astype(float)
    for _ in range(5):
        rho = RNG.uniform(0.1, 8.0)
        u = RNG.uniform(-0.3, 0.3, D)
        f = o.feq(rho, u)
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(c.T @ f, rho * u, rtol=1e-13, atol=1e-14)
        assert np.allclose(np.einsum("i,ia,ib->ab", f, c, c),
                           rho / 3 * np.eye(D) + rho * np.outer(u, u), rtol=1e-13, atol=1e-14)
        assert np.allclose(np.einsum("i,ia->a", f, c ** 3), rho * u, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("lattice", [0, 1])
def test_extended_equilibrium_moments_appendix_d(lattice):
    """Appendix D (moments of f*): sum (f* - feq) = 0, sum c (f* - feq) = F,
    sum c c (f* - feq) = u F + F u + Phi + F F / rho, diagonals included."""
    o = small(lattice)
    _, c = o.weights()
    D = 2 if lattice == 0 else 3
    c = c[:, :D].astype(float)
    for _ in range(5):
        rho = RNG.uniform(0.1, 8.0)
        u = RNG.uniform(-0.2, 0.2, D)
        F = RNG.uniform(-0.05, 0.05, D)
        Phi = RNG.uniform(-0.01, 0.01, D)
        d = o.fstar(rho, u, F, Phi) - o.feq(rho, u)
        assert abs(d.sum()) < 1e-14 * rho
        assert np.allclose(c.T @ d, F, atol=1e-14)
        want = np.outer(u, F) + np.outer(F, u) + np.diag(Phi) + np.outer(F, F) / rho
        assert np.allclose(np.einsum("i,ia,ib->ab", d, c, c), want, atol=1e-14)


def test_literal_zeta_star_breaks_appendix_d():
    """The printed zeta* (u_a^2, not (u_a + F_a/rho)^2) misses the diagonal of
    sum c c f* = rho xi* xi* + ..., which is why the shifted reading is taken."""
    o = OracleLBM(1, 8, 8, 8, 0, 0.8, 0.02, 1.0, a=9 / 490, flags=ZETA_LITERAL)
    _, c = o.weights()
    c = c.astype(float)
    rho, u, F, Phi = 2.0, np.array([0.1, -0.05, 0.02]), np.array([0.03, 0.02, -0.04]), np.zeros(3)
    d = o.fstar(rho, u, F, Phi) - o.feq(rho, u)
    want = np.outer(u, F) + np.outer(F, u) + np.outer(F, F) / rho
    got = np.einsum("i,ia,ib->ab", d, c, c)
    assert not np.allclose(np.diag(got), np.diag(want), atol=1e-6)


@pytest.mark.parametrize("lattice", [0, 1])
def test_stencils_exact_on_quartics(lattice):
    """Eqs. PP_discrete + PPcond1-2: with G1 = 4/3, G2 = -1/6 the stencil returns
    grad g exactly for polynomials of degree <= 4; Eqs. capillary_discrete +
    Ccond1-2 with (G3, G4) = (2, -1) return -grad lap g exactly."""
    import sympy as sp
    n = 14 if lattice == 0 else 12
    o = OracleLBM(lattice, n, n, 1 if lattice == 0 else n, 0, 0.8, 0.02, 1.0, a=9 / 490)
    D = o.D
    X = sp.symbols("x y z")[:D]
    rs = np.random.default_rng(7)
    terms = [m for m in itertools.product(range(5), repeat=D) if sum(m) <= 4]
    poly = sum(sp.Rational(int(rs.integers(-9, 10)), 10) * sp.Mul(*[v ** e for v, e in zip(X, m)])
               for m in terms)
    grid = np.meshgrid(*[np.arange(s) for s in ((o.nz, o.ny, o.nx) if D == 3 else (o.ny, o.nx))],
                       indexing="ij")
    coords = grid[::-1]  # x, y[, z]
    f = sp.lambdify(X, poly, "numpy")
    g = np.asarray(f(*coords), dtype=float).ravel()
    grad = [sp.lambdify(X, sp.diff(poly, v), "numpy") for v in X]
    lap = sum(sp.diff(poly, v, 2) for v in X)
    glap = [sp.lambdify(X, sp.diff(lap, v), "numpy") for v in X]
    s1 = o.stencil(g, 4 / 3, -1 / 6).reshape(D, -1)
    s2 = o.stencil(g, 2.0, -1.0).reshape(D, -1)
    inner = np.ones(coords[0].shape, bool)
    for cc, s in zip(coords, coords[0].shape[::-1]):
        inner &= (cc >= 2) & (cc < s - 2)
    inner = inner.ravel()
    scale = np.abs(g).max()
    for a in range(D):
        ga = np.broadcast_to(np.asarray(grad[a](*coords), dtype=float), coords[0].shape).ravel()
        la = np.broadcast_to(np.asarray(glap[a](*coords), dtype=float), coords[0].shape).ravel()
        assert np.allclose(s1[a][inner], ga[inner], atol=1e-11 * scale)
        assert np.allclose(s2[a][inner], -la[inner], atol=1e-11 * scale)
    # a degree-5 term leaves the predicted O(grad^5) residual: not exact any more
    g5 = g + (coords[0].astype(float) ** 5).ravel() / 1000.0
    s5 = o.stencil(g5, 4 / 3, -1 / 6).reshape(D, -1)
    ga = np.broadcast_to(np.asarray(grad[0](*coords), dtype=float), coords[0].shape).ravel()
    ga = ga + 5 * (coords[0].astype(float) ** 4).ravel() / 1000.0
    assert np.abs(s5[0][inner] - ga[inner]).max() > 1e-4


@pytest.mark.parametrize("lattice", [0, 1])
def test_uniform_state_is_fixed_point(lattice):
    o = small(lattice, n=6)
    o.init(np.full(o.N, 2.5))
    f0 = o.get_populations()
    o.step(20)
    assert np.abs(o.get_populations() - f0).max() < 1e-14


def _two_phase(lattice, n, mask=None, seed=11):
    from paper_2112_01975_gb300.inputs import add_noise, drop
    nz = 1 if lattice == 0 else n
    o = OracleLBM(lattice, n, n, nz, 0, 0.8, 0.0255116, 1.0, a=9 / 490, mask=mask,
                  rho_w=0.84)
    rho = add_noise(drop(n, n, nz, n / 4, 0.8388, 6.7645), 1e-3, seed)
    return o, rho


@pytest.mark.parametrize("lattice", [0, 1])
def test_mass_exactly_conserved_periodic(lattice):
    """Collision keeps sum f (sum Psi = 1) and streaming permutes: mass is kept to roundoff."""
    o, rho = _two_phase(lattice, 16 if lattice == 0 else 10)
    o.init(rho)
    m0, _ = o.reduce()
    o.step(60)
    m1, _ = o.reduce()
    assert abs(m1 - m0) / m0 < 1e-13


def test_mass_conserved_with_bounce_back():
    from paper_2112_01975_gb300.inputs import block_mask
    n = 10
    mask = block_mask(n, n, n, (3, 3, 0), (6, 7, 4))
    o, rho = _two_phase(1, n, mask=mask)
    o.init(np.where(mask == 1, 0.0, rho))
    m0, _ = o.reduce()
    o.step(40)
    m1, _ = o.reduce()
    assert abs(m1 - m0) / m0 < 1e-13


@pytest.mark.parametrize("lattice", [0, 1])
def test_momentum_balance(lattice):
    """sum_i c_i f* - sum_i c_i feq = F at every node, so on a periodic box
    J(t+1) = J(t) + sum_x F(x, t) to roundoff."""
    o, rho = _two_phase(lattice, 16 if lattice == 0 else 10)
    o.init(rho)
    o.step(5)
    for _ in range(3):
        _, j0 = o.reduce()
        _, _, _, F = o.moments()
        o.step(1)
        _, j1 = o.reduce()
        Fs = F.reshape(o.D, -1).sum(axis=1)
        assert np.allclose(j1 - j0, Fs, atol=1e-12)


def test_d3q27_z_invariant_reduces_to_d2q9():
    """Product form marginalises (sum over c_z of Psi_z = 1): z-invariant D3Q27
    data evolve as the D2Q9 run."""
    from paper_2112_01975_gb300.inputs import add_noise, drop
    n, nz = 16, 5
    rho2 = add_noise(drop(n, n, 1, 5.0, 0.8388, 6.7645), 1e-3, 3)
    o2 = OracleLBM(0, n, n, 1, 0, 0.8, 0.0255116, 1.0, a=9 / 490)
    o3 = OracleLBM(1, n, n, nz, 0, 0.8, 0.0255116, 1.0, a=9 / 490)
    o2.init(rho2)
    o3.init(np.tile(rho2, nz))
    o2.step(30)
    o3.step(30)
    r2, u2, _, _ = o2.moments()
    r3, u3, _, _ = o3.moments()
    r3 = r3.reshape(nz, -1)
    u3 = u3.reshape(3, nz, -1)
    for z in range(nz):
        assert np.allclose(r3[z], r2, rtol=1e-12)
        assert np.allclose(u3[0, z], u2[: n * n], atol=1e-13)
        assert np.allclose(u3[1, z], u2[n * n:], atol=1e-13)
        assert np.abs(u3[2, z]).max() < 1e-14


def test_mirror_symmetry():
    """Mirroring the initial state in x mirrors the result (u_x flips sign)."""
    from paper_2112_01975_gb300.inputs import add_noise, drop
    n = 16
    rho = add_noise(drop(n, n, 1, 5.0, 0.8388, 6.7645, center=(6, 8, 0)), 1e-3, 5)
    rm = rho.reshape(n, n)[:, ::-1]
    # mirror about x -> (n-1) - x keeps the node set
    a = OracleLBM(0, n, n, 1, 0, 0.8, 0.0255116, 1.0, a=9 / 490)
    b = OracleLBM(0, n, n, 1, 0, 0.8, 0.0255116, 1.0, a=9 / 490)
    a.init(rho)
    b.init(np.ascontiguousarray(rm).ravel())
    a.step(25)
    b.step(25)
    ra, ua, _, _ = a.moments()
    rb, ub, _, _ = b.moments()
    assert np.allclose(rb.reshape(n, n)[:, ::-1], ra.reshape(n, n), rtol=1e-12)
    assert np.allclose(-ub[: n * n].reshape(n, n)[:, ::-1], ua[: n * n].reshape(n, n), atol=1e-13)


@pytest.mark.parametrize("lattice", [0, 1])
def test_node_local_post_matches_full_step(lattice):
    """oracle_post_local on a node's neighbourhood gives exactly the values the
    full oracle step pushes from that node (bounce-back included)."""
    from oracle import sample
    from paper_2112_01975_gb300.inputs import add_noise, block_mask, drop
    n = 12
    nz = 1 if lattice == 0 else 10
    mask = block_mask(n, n, nz, (0, 0, 0), (n, 2, nz))          # a wall at y = 0, 1
    o = OracleLBM(lattice, n, n, nz, 0, 0.8, 0.0255116, 0.9, a=9 / 490, mask=mask, rho_w=0.84)
    rho = add_noise(drop(n, n, nz, 3.5, 0.8388, 6.7645), 1e-3, 13)
    u0 = 0.02 * np.random.default_rng(3).uniform(-1, 1, o.D * o.N)
    o.init(np.where(mask == 1, 1.0, rho), u0)
    o.step(3)
    f = o.get_populations().reshape(o.Q, -1)
    o.step(1)
    f1 = o.get_populations().reshape(o.Q, -1)
    _, c = o.weights()
    shape = (nz, n, n)
    for (x, y, z) in [(5, 5, 0), (0, 2, nz - 1), (11, 3, nz // 2), (6, 11, min(1, nz - 1))]:
        idx = sample.block_indices(shape, x, y, z, o.D)
        block = f[:, idx].T
        post = o.post_local(block, mask[idx])
        for i, (j, d) in enumerate(sample.pushed_indices(shape, x, y, z, c, mask)):
            assert post[i] == pytest.approx(f1[j, d], rel=1e-14, abs=1e-16)


def test_openmp_build_is_bitwise_the_plain_oracle():
    """The -fopenmp build of the oracle (the all-cores CPU baseline) runs the
    same node loops on several threads; every iteration writes its own
    entries, so populations, moments and the pressure tensor are bitwise
    those of the plain build (masked D3Q27 drop with a body force)."""
    from oracle import build as obuild
    try:
        obuild.build(openmp=True)
    except Exception as exc:   # no OpenMP in this compiler
        pytest.skip(f"no -fopenmp build: {exc}")
    w = inputs.DROP_D3Q27_128
    nx, ny, nz = 20, 18, 16
    mask = inputs.block_mask(nx, ny, nz, (0, 0, 0), (nx, ny, 1))
    rho = inputs.add_noise(inputs.drop(nx, ny, nz, 5.0, w.rho_v, w.rho_l, center=(10, 9, 8)), 1e-4, 61)
    rho = np.where(mask == 1, w.rho_v, rho)
    out = []
    for omp in (False, True):
        o = OracleLBM(1, nx, ny, nz, w.eos, w.t_over_tc, w.kappa, 0.8, mask=mask, a=w.a, b=w.b,
                      rho_w=w.rho_v, g=(1e-6, 0.0, -1e-5), openmp=omp)
        o.init(rho)
        o.step(30)
        out.append((o.get_populations(), o.moments(), o.pressure_tensor()))
    assert np.array_equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][2], out[1][2])
