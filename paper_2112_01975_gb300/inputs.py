"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds no arithmetic of the lattice Boltzmann method itself: it
only draws seeded numbers and lays out initial density/velocity fields and
solid masks on the lattice. Every field is returned as float64 numpy arrays in
the library's layout: scalar fields ``[z][y][x]`` flattened with x fastest,
vector fields as ``D`` consecutive planes of that shape.

Noise: ``xi = U[-1, 1)`` from splitmix64(seed XOR linear index), the published
counter-based generator of Steele, Lea and Flood (2014), written out here.

Initial drop profile: a tanh between the two coexistence densities whose
maximum slope equals the interface-width definition W = (rho_l - rho_v) /
max|grad rho| of Sec. 3.5 (Eq. interface_W).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied to each uint64 of ``x``."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """n draws of U[-1, 1): top 53 bits of splitmix64(seed ^ i), i = 0..n-1."""
    idx = np.arange(n, dtype=np.uint64) ^ np.uint64(seed & _M64)
    bits = splitmix64(idx) >> np.uint64(11)
    return bits.astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def _coords(nx: int, ny: int, nz: int):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def tanh_interface(dist: np.ndarray, rho_in: float, rho_out: float,
                   width: float) -> np.ndarray:
    """rho_in where dist << 0, rho_out where dist >> 0, max slope
    (rho_in - rho_out) / width at dist = 0."""
    return 0.5 * (rho_in + rho_out) - 0.5 * (rho_in - rho_out) * np.tanh(2.0 * dist / width)


def drop(nx: int, ny: int, nz: int, radius: float, rho_v: float, rho_l: float,
         width: float = 5.0, center=None) -> np.ndarray:
    """Liquid drop of the given radius centred at (nx/2, ny/2[, nz/2])."""
    x, y, z = _coords(nx, ny, nz)
    cx, cy, cz = center if center is not None else (nx // 2, ny // 2, nz // 2 if nz > 1 else 0)
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + ((z - cz) ** 2 if nz > 1 else 0.0))
    return tanh_interface(r - radius, rho_l, rho_v, width).ravel()


def drops(nx: int, ny: int, nz: int, centers, radius: float, rho_v: float,
          rho_l: float, width: float = 5.0) -> np.ndarray:
    """Several drops: pointwise maximum of single-drop profiles."""
    out = None
    for c in centers:
        d = drop(nx, ny, nz, radius, rho_v, rho_l, width, center=c)
        out = d if out is None else np.maximum(out, d)
    return out


def slab(nx: int, ny: int, nz: int, x0: float, x1: float, rho_v: float,
         rho_l: float, width: float = 5.0) -> np.ndarray:
    """Liquid for x0 <= x < x1 (flat interfaces normal to x), vapour elsewhere."""
    x, _, _ = _coords(nx, ny, nz)
    mid = 0.5 * (x0 + x1)
    half = 0.5 * (x1 - x0)
    return tanh_interface(np.abs(x - mid) - half, rho_l, rho_v, width).ravel()


def add_noise(rho: np.ndarray, rel: float, seed: int) -> np.ndarray:
    """rho * (1 + rel * xi), xi = U[-1, 1) from splitmix64(seed ^ index)."""
    return rho * (1.0 + rel * uniform_pm1(seed, rho.size))


def pillar_mask(nx: int, ny: int, nz: int, side: int = 8, height: int = 16,
                pitch: int = 16, seed: int = 4, wall: int = 1) -> np.ndarray:
    """uint8 solid mask: a wall of `wall` planes (z < wall) plus square
    pillars (side x side x height) on a square lattice of the given pitch, on
    z = wall .. wall + height - 1. The pillar lattice offset in x and y comes
    from the seed."""
    off = splitmix64(np.array([seed], dtype=np.uint64))[0]
    ox = int(off % np.uint64(pitch))
    oy = int((off >> np.uint64(32)) % np.uint64(pitch))
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[:wall] = 1
    xs = ((np.arange(nx) - ox) % pitch) < side
    ys = ((np.arange(ny) - oy) % pitch) < side
    col = np.logical_and(ys[:, None], xs[None, :])
    m[wall:wall + height][:, col] = 1
    return m.ravel()


def block_mask(nx: int, ny: int, nz: int, lo, hi) -> np.ndarray:
    """uint8 mask with one solid box lo <= (x, y, z) < hi."""
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = 1
    return m.ravel()


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: lattice, sizes, fluid parameters, init recipe.

    ``rho_v``/``rho_l`` are the Maxwell equal-area coexistence densities of
    the EOS at ``t_over_tc`` (eq. Maxwell_equal_area) and ``kappa`` the
    capillary coefficient that gives a second-gradient interface width of 5
    lattice units; both are recomputed from the EOS by a CPU test.
    """
    name: str
    lattice: int          # 0 = D2Q9, 1 = D3Q27
    nx: int
    ny: int
    nz: int
    eos: int              # 0 vdW, 1 PR, 2 RKS, 3 CS
    t_over_tc: float
    kappa: float
    tau: float
    rho_v: float
    rho_l: float
    radius: float
    seed: int
    a: float
    b: float
    noise: float = 1e-4
    steps: int = 1000
    centres: tuple = ()   # several drops of the same radius; empty: one drop at the centre
    # impact on a textured wall: pillar mask of this seed (None: no solid),
    # the drop's lowest point `gap` nodes above the pillar tops, moving down
    # at u_down in the liquid (scaled by the liquid fraction in the interface)
    mask_seed: int | None = None
    gap: float = 8.0
    u_down: float = 0.0
    pillar: tuple = (8, 16, 16)   # side, height, pitch
    wall: int = 1                 # planes of the wall under the pillars

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def rho_w(self) -> float | None:
        """Virtual density of solid nodes: the vapour's (non-wetting)."""
        return self.rho_v if self.mask_seed is not None else None

    def fields(self, shape=None):
        """(rho0, u0, mask) on the workload's lattice, or on ``shape`` = (nx,
        ny, nz) with the drop radius and centres scaled by nx' / nx (pillars
        and the gap above them keep their size); the same noise amplitude and
        seed. u0 is None for a start at rest, mask None without solids."""
        nx, ny, nz = shape if shape is not None else (self.nx, self.ny, self.nz)
        s = nx / self.nx
        R = self.radius * s
        mask = None
        if self.mask_seed is not None:
            side, height, pitch = self.pillar
            mask = pillar_mask(nx, ny, nz, side=side, height=height, pitch=pitch,
                               seed=self.mask_seed, wall=self.wall)
            c = (nx // 2, ny // 2, self.wall + height - 1 + R + self.gap)
            r = drop(nx, ny, nz, R, self.rho_v, self.rho_l, center=c)
        elif self.centres:
            r = drops(nx, ny, nz, [tuple(v * s for v in cc) for cc in self.centres], R,
                      self.rho_v, self.rho_l)
        else:
            r = drop(nx, ny, nz, R, self.rho_v, self.rho_l)
        if self.noise:
            r = add_noise(r, self.noise, self.seed)
        u0 = None
        if self.u_down:
            u0 = np.zeros(3 * r.size)
            frac = (r - self.rho_v) / (self.rho_l - self.rho_v)
            u0[2 * r.size:] = -self.u_down * frac
        if mask is not None:
            r = np.where(mask == 1, self.rho_v, r)
            if u0 is not None:
                u0[2 * r.size:][mask == 1] = 0.0
        return r, u0, mask

    def rho0(self) -> np.ndarray:
        return self.fields()[0]

    def rho0_scaled(self, n: int) -> np.ndarray:
        """The same layout on an n^3 (3D) or n^2 (2D) lattice: radius and
        drop centres scaled by n / nx; the same noise amplitude and seed."""
        return self.fields((n, n, n if self.lattice == 1 else 1))[0]

    def u0(self) -> np.ndarray:
        d = 2 if self.lattice == 0 else 3
        u = self.fields()[1]
        return np.zeros(d * self.nodes) if u is None else u


# The EOS attraction parameter a is the named one scaled down by corresponding
# states (coexistence densities depend on T/Tc and b only): with a = 9/49 the
# liquid's isothermal sound speed squared dP/drho is 1.13 in lattice units and
# the explicit update diverges within ten steps; a/10 gives 0.113. kappa is
# scaled with a so that the interface width stays 5.

# D2Q9 static drop, 64x64 periodic, van der Waals (a = 9/490, b = 2/21) at
# T/Tc = 0.8, drop radius 16, tau = 1.
DROP_D2Q9_64 = Workload("d2q9_drop_64x64_vdw_tr0.8", 0, 64, 64, 1, 0, 0.8,
                        kappa=0.0255116006, tau=1.0, rho_v=0.838834226444,
                        rho_l=6.76447040010, radius=16.0, seed=1,
                        a=9.0 / 490.0, b=2.0 / 21.0, steps=1000)

# D3Q27 static drop, 128^3 periodic, Peng-Robinson (a = 2/245, b = 2/21,
# acentric factor 0.344) at T/Tc = 0.7, drop radius 24, tau = 1.
DROP_D3Q27_128 = Workload("d3q27_drop_128^3_pr_tr0.7", 1, 128, 128, 128, 1, 0.7,
                          kappa=0.0223020350, tau=1.0, rho_v=0.0556350874516,
                          rho_l=8.08032155174, radius=24.0, seed=2,
                          a=2.0 / 245.0, b=2.0 / 21.0, steps=20000)

# The same drop at 96^3 (radius 18): a smaller case for profiler captures,
# still larger than L2 (2 x 191 MB of populations).
DROP_D3Q27_96 = dataclasses.replace(DROP_D3Q27_128, name="d3q27_drop_96^3_pr_tr0.7", nx=96,
                                    ny=96, nz=96, radius=18.0)

# D3Q27 coalescence, 256^3 periodic, Peng-Robinson (b = 2/21, a scaled for a
# liquid dP/drho of 0.1) at T/Tc = 0.45 (Maxwell density ratio 6.6e4): two
# drops of radius 40 touching at the centre, tau = 0.725.
COALESCENCE_D3Q27_256 = Workload("d3q27_coalescence_256^3_pr_tr0.45", 1, 256, 256, 256, 1, 0.45,
                                 kappa=0.0100296894491, tau=0.725,
                                 rho_v=0.000142187914218311, rho_l=9.42493892983339,
                                 radius=40.0, seed=3, a=0.00162040657246882, b=2.0 / 21.0,
                                 steps=10000, centres=((88.0, 128.0, 128.0), (168.0, 128.0, 128.0)))

# D3Q27 drop impact on a textured wall, 384x384x256: a wall two planes thick
# (z = 0, 1: the force stencils reach two nodes, so a thinner wall would
# couple the fluid above it to the fluid below its periodic image) plus
# 8x8x16 square pillars at pitch 16 (lattice offset from seed 4), solid
# density rho_w = rho_v (non-wetting); Peng-Robinson (b = 2/21, a scaled for
# a liquid dP/drho of 0.1) at T/Tc = 0.5 (Maxwell density ratio 1.1e4); a
# drop of radius 60 whose lowest point is 8 nodes above the pillar tops,
# moving down at U = 0.115 in the liquid (We = rho_l U^2 2R / sigma = 100,
# sigma = 0.146), tau = 0.725 (Re = U 2R / nu = 184), no noise. The largest
# single-GPU workload; FP32 storage.
IMPACT_D3Q27_384 = Workload("d3q27_impact_384x384x256_pr_tr0.5", 1, 384, 384, 256, 1, 0.5,
                            kappa=0.011670519231996029, tau=0.725,
                            rho_v=0.000832893711960915, rho_l=9.219284708837831,
                            radius=60.0, seed=4, a=0.00216512412385399, b=2.0 / 21.0,
                            noise=0.0, steps=20000, mask_seed=4, u_down=0.115, wall=2)

WORKLOADS = {w.name: w for w in (DROP_D2Q9_64, DROP_D3Q27_128, DROP_D3Q27_96,
                                 COALESCENCE_D3Q27_256, IMPACT_D3Q27_384)}
