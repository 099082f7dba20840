"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every function include/lbm.h declares, and validates arguments
before touching the device."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2112_01975_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_destroy",
                 "lbm_reduce", "lbm_get_populations", "lbm_set_populations"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        getattr(lib, n)


def test_required_bytes(lib):
    lib.lbm_required_bytes.restype = C.c_size_t
    n = lib.lbm_required_bytes(1, 128, 128, 128, 0)
    N = 128 ** 3
    # two FP64 population buffers + rho/psi + u + rho u^3 + mask, 256-byte aligned
    assert n >= 2 * 27 * 8 * N + 16 * N + 2 * 3 * 8 * N + N
    assert n < 2 * 27 * 8 * N + 16 * N + 2 * 3 * 8 * N + N + 64 * 1024
    assert lib.lbm_required_bytes(0, 64, 64, 2, 0) == 0      # D2Q9 needs nz = 1
    # the largest lattice: 27 N <= 4e9 (32-bit population indices)
    assert lib.lbm_required_bytes(1, 529, 529, 529, 1) > 0
    assert lib.lbm_required_bytes(1, 530, 530, 530, 1) == 0
    assert lib.lbm_required_bytes(0, 20000, 8000, 1, 1) == 0
    assert lib.lbm_required_bytes(1, 4, 64, 64, 0) == 0      # below the 2-ring minimum
    assert lib.lbm_required_bytes(1, 64, 64, 64, 7) == 0     # unknown storage


def test_default_params(lib):
    from paper_2112_01975_gb300.lbm import lbm_params
    p = lbm_params()
    assert lib.lbm_default_params(0, C.byref(p)) == 0
    assert p.a == pytest.approx(9 / 49) and p.b == pytest.approx(2 / 21)
    assert lib.lbm_default_params(1, C.byref(p)) == 0
    assert p.a == pytest.approx(2 / 49) and p.acentric == pytest.approx(0.344)
    assert lib.lbm_default_params(4, C.byref(p)) == 0 and p.b > 0    # Shan-Chen: a, b unused
    assert lib.lbm_default_params(9, C.byref(p)) == 1


@pytest.mark.parametrize("args", [
    (0, 64, 64, 2, 0, 0.8, 0.02, 1.0),     # D2Q9 with nz != 1
    (1, 64, 64, 4, 0, 0.8, 0.02, 1.0),     # nz < 5
    (1, 64, 64, 64, 6, 0.8, 0.02, 1.0),    # unknown EOS
    (1, 64, 64, 64, 0, 1.2, 0.02, 1.0),    # T/Tc >= 1
    (1, 64, 64, 64, 0, 0.8, -0.1, 1.0),    # kappa < 0
    (1, 64, 64, 64, 0, 0.8, 0.02, 0.5),    # tau <= 1/2
])
def test_create_rejects_bad_arguments_without_a_device(lib, args):
    h = C.c_void_p()
    lattice, nx, ny, nz, eos, tr, kap, tau = args
    rc = lib.lbm_create(C.byref(h), lattice, nx, ny, nz, eos, C.c_double(tr), C.c_double(kap),
                        C.c_double(tau), None, None)
    assert rc == 1 and not h.value


def test_null_handle_calls_are_errors(lib):
    assert lib.lbm_step(None, C.c_int64(1)) == 1
    assert lib.lbm_sync(None, -1) == 1
    x, y = C.c_int(-1), C.c_int(-1)
    assert lib.lbm_get_tile(None, C.byref(x), C.byref(y)) == 1 and x.value == -1
    assert lib.lbm_set_tile(None, 7) == 1
    on = C.c_int(-1)
    assert lib.lbm_set_fused_variant(None, 1) == 1
    assert lib.lbm_get_fused_variant(None, C.byref(on)) == 1 and on.value == -1
    assert lib.lbm_probe_fp64_tflops(None) == 1
    ms = C.c_double()
    assert lib.lbm_selftest_wait_timeout(C.c_longlong(1000), None, C.byref(ms)) == 1
    assert lib.lbm_selftest_wait_timeout(C.c_longlong(0), C.byref(on), C.byref(ms)) == 1
    lib.lbm_last_error.restype = C.c_char_p
    assert lib.lbm_last_error(None) == b"null handle"
    lib.lbm_destroy(None)
