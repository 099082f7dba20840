"""Sampled-node checks of large lattices against the oracle (test
infrastructure only): cut the 5x5(x5) neighbourhood of a node out of a
population array, and read back where a push step put that node's
post-collision populations."""
from __future__ import annotations

import numpy as np


def offsets(D: int):
    r = range(-2, 3)
    zs = r if D == 3 else [0]
    return [(dx, dy, dz) for dz in zs for dy in r for dx in r]


def block_indices(shape, x, y, z, D):
    """Flat node indices of the neighbourhood, ordered [dz][dy][dx]."""
    nz, ny, nx = shape
    return np.array([((x + dx) % nx) + nx * (((y + dy) % ny) + ny * ((z + dz) % nz))
                     for dx, dy, dz in offsets(D)], dtype=np.int64)


def pushed_indices(shape, x, y, z, c, mask):
    """(direction, node) where population i of node (x, y, z) lands after a push
    step with halfway bounce-back."""
    nz, ny, nx = shape
    Q = len(c)
    n0 = x + nx * (y + ny * z)
    out = []
    for i in range(Q):
        d = ((x + c[i][0]) % nx) + nx * (((y + c[i][1]) % ny) + ny * ((z + c[i][2]) % nz))
        if mask is not None and mask[d]:
            out.append(((Q - 1 - i), n0))
        else:
            out.append((i, d))
    return out
