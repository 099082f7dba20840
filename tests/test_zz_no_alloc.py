"""The allocation-free reduction entry point, lbm_reduce_noalloc.

It serves callers that cannot allocate device memory (a reserved or frozen
memory pool, or code that only borrows device pointers): they pass the
populations, the mask and a 4-double output, and the library keeps its
per-block partial sums in static device memory. This file is collected last
so that a run stopping at the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_01975_gb300 import build
    build.build()
    from paper_2112_01975_gb300 import inputs, lbm
    return torch, lbm, inputs


def _noalloc(lbm, torch, lattice, nx, ny, nz, f_dev, mask_dev, stream):
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lbm.lbm_reduce_noalloc(lattice, nx, ny, nz, C.c_void_p(f_dev.data_ptr()),
                                None if mask_dev is None else C.c_void_p(mask_dev.data_ptr()),
                                C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == 0, lbm.STATUS.get(rc, rc)
    stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("case", ["d3q27_mask", "d2q9_open"])
def test_noalloc_matches_lbm_reduce_twice(env, case):
    torch, lbm, inputs = env
    w = inputs.DROP_D3Q27_128
    if case == "d3q27_mask":
        lattice, nx, ny, nz = 1, 40, 36, 33
        mask = inputs.block_mask(nx, ny, nz, (30, 0, 0), (36, 6, 33))
        rho = inputs.add_noise(inputs.drop(nx, ny, nz, 9.0, w.rho_v, w.rho_l), 1e-4, 3)
        g = lbm.LBM(lattice, nx, ny, nz, w.eos, w.t_over_tc, w.kappa, w.tau, mask=mask,
                    a=w.a, b=w.b, rho_w=w.rho_v)
    else:
        v = inputs.DROP_D2Q9_64
        lattice, nx, ny, nz = 0, 64, 64, 1
        mask = None
        rho = v.rho0()
        g = lbm.LBM(lattice, nx, ny, nz, v.eos, v.t_over_tc, v.kappa, v.tau, a=v.a, b=v.b)
    g.init(rho)
    g.step(30)
    mass, mom = g.reduce()                                 # the existing entry point
    D = 2 if lattice == 0 else 3
    f_dev = torch.empty(g.Q * g.N, dtype=torch.float64, device="cuda")
    g.get_populations(f_dev)
    mask_dev = None if mask is None else torch.from_numpy(mask).cuda()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    first = _noalloc(lbm, torch, lattice, nx, ny, nz, f_dev, mask_dev, stream)
    second = _noalloc(lbm, torch, lattice, nx, ny, nz, f_dev, mask_dev, stream)
    for got in (first, second):
        assert got[0] == pytest.approx(mass, rel=1e-13)
        assert np.allclose(got[1:1 + D], mom, rtol=0, atol=1e-12 * mass)
        if D == 2:
            assert got[3] == 0.0
    assert np.array_equal(first, second)


def test_noalloc_rejects_sizes_beyond_its_maximum(env):
    torch, lbm, _ = env
    f = torch.zeros(9, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    # checked on the host before anything is launched
    rc = lbm.lbm_reduce_noalloc(0, 8193, 8192, 1, C.c_void_p(f.data_ptr()), None,
                                C.c_void_p(out.data_ptr()), None)
    assert rc == 7                                          # LBM_ETOOBIG
    assert out.abs().sum().item() == 0.0


def test_noalloc_allocates_nothing(env):
    """After a first (warm) call, five more calls leave the device's free
    memory (cudaMemGetInfo) and the torch allocator's counters unchanged:
    the entry point allocates nothing on the device."""
    torch, lbm, inputs = env
    v = inputs.DROP_D2Q9_64
    g = lbm.LBM(0, 64, 64, 1, v.eos, v.t_over_tc, v.kappa, v.tau, a=v.a, b=v.b)
    g.init(v.rho0())
    f_dev = torch.empty(g.Q * g.N, dtype=torch.float64, device="cuda")
    g.get_populations(f_dev)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()

    def call():
        rc = lbm.lbm_reduce_noalloc(0, 64, 64, 1, C.c_void_p(f_dev.data_ptr()), None,
                                    C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == 0

    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for _ in range(5):
        call()
    stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
