"""Python binding of liblbm.so (the C ABI declared in include/lbm.h).

Argument marshalling only: every step of the update runs in the library's
CUDA kernels. PyTorch supplies device memory (a uint8 tensor bound with
``lbm_bind_device_memory``) and the CUDA stream. There is no CPU fallback:
if the compiled library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm.so")

D2Q9, D3Q27 = 0, 1
EOS_VDW, EOS_PR, EOS_RKS, EOS_CS, EOS_SC1, EOS_SC2 = 0, 1, 2, 3, 4, 5
F64, F32, F16S, BF16S = 0, 1, 2, 3
FUSED_PLAIN, FUSED_WARP_SPECIALISED, FUSED_TMEM, FUSED_WS_TMEM, FUSED_WS_TMA, FUSED_TM_TMA = 0, 1, 2, 3, 4, 5
FUSED_NAMES = {0: "plain", 1: "warp-specialised", 2: "tensor-memory",
               3: "warp-specialised, tensor-memory",
               4: "warp-specialised, tensor-memory, TMA-staged planes",
               5: "tensor-memory, TMA-staged planes (shifted storage)"}
FLAG_PHI_OFF = 1
FLAG_EOS_F64 = 2
STATUS = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_ENONFINITE",
          5: "LBM_ETIMEOUT", 6: "LBM_ESTATE", 7: "LBM_ETOOBIG"}


class lbm_params(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("acentric", C.c_double),
                ("rho_w", C.c_double), ("storage", C.c_int), ("flags", C.c_int),
                ("g", C.c_double * 3), ("tau_v", C.c_double), ("visc_rho", C.c_double * 2)]


class LBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    vp, dp, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64
    L.lbm_default_params.argtypes = [C.c_int, C.POINTER(lbm_params)]
    L.lbm_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                             C.c_double, C.c_double, C.c_double, vp, C.POINTER(lbm_params)]
    L.lbm_required_bytes.restype = C.c_size_t
    L.lbm_required_bytes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
    L.lbm_bind_device_memory.argtypes = [vp, vp, C.c_size_t]
    L.lbm_set_stream.argtypes = [vp, vp]
    L.lbm_init.argtypes = [vp, vp, vp, C.c_int]
    L.lbm_step.argtypes = [vp, i64]
    L.lbm_moments.argtypes = [vp, vp, vp, vp, C.c_int]
    L.lbm_reduce.argtypes = [vp, dp, dp]
    L.lbm_pressure_tensor.argtypes = [vp, vp, C.c_int]
    L.lbm_set_wall_distances.argtypes = [vp, vp]
    L.lbm_get_populations.argtypes = [vp, vp, C.c_int]
    L.lbm_set_populations.argtypes = [vp, vp, C.c_int]
    L.lbm_sync.argtypes = [vp, C.c_int]
    L.lbm_launch_count.restype = i64
    L.lbm_launch_count.argtypes = [vp]
    L.lbm_probe_fp64_tflops.argtypes = [dp]
    L.lbm_selftest_wait_timeout.argtypes = [C.c_longlong, C.POINTER(C.c_int), dp]
    L.lbm_time_kernels.argtypes = [vp, i64, dp]
    L.lbm_set_chunk.argtypes = [vp, C.c_int]
    L.lbm_autotune.argtypes = [vp, C.POINTER(C.c_int)]
    L.lbm_get_tile.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.lbm_set_tile.argtypes = [vp, C.c_int]
    L.lbm_set_fused_variant.argtypes = [vp, C.c_int]
    L.lbm_get_fused_variant.argtypes = [vp, C.POINTER(C.c_int)]
    L.lbm_reduce_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]
    L.lbm_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int]
    L.lbm_batch_step.argtypes = [vp, i64]
    L.lbm_batch_sync.argtypes = [vp]
    L.lbm_batch_launch_count.restype = i64
    L.lbm_batch_launch_count.argtypes = [vp]
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_last_error.argtypes = [vp]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    return L


_lib = _load()
# The C functions under their own names, for callers that marshal themselves.
lbm_default_params = _lib.lbm_default_params
lbm_create = _lib.lbm_create
lbm_required_bytes = _lib.lbm_required_bytes
lbm_bind_device_memory = _lib.lbm_bind_device_memory
lbm_set_stream = _lib.lbm_set_stream
lbm_init = _lib.lbm_init
lbm_step = _lib.lbm_step
lbm_moments = _lib.lbm_moments
lbm_reduce = _lib.lbm_reduce
lbm_get_populations = _lib.lbm_get_populations
lbm_set_populations = _lib.lbm_set_populations
lbm_sync = _lib.lbm_sync
lbm_launch_count = _lib.lbm_launch_count
lbm_time_kernels = _lib.lbm_time_kernels
lbm_set_chunk = _lib.lbm_set_chunk
lbm_autotune = _lib.lbm_autotune
lbm_get_tile = _lib.lbm_get_tile
lbm_set_tile = _lib.lbm_set_tile
lbm_set_fused_variant = _lib.lbm_set_fused_variant
lbm_get_fused_variant = _lib.lbm_get_fused_variant
lbm_reduce_noalloc = _lib.lbm_reduce_noalloc
lbm_batch_create = _lib.lbm_batch_create
lbm_batch_step = _lib.lbm_batch_step
lbm_batch_sync = _lib.lbm_batch_sync
lbm_batch_launch_count = _lib.lbm_batch_launch_count
lbm_batch_destroy = _lib.lbm_batch_destroy
lbm_last_error = _lib.lbm_last_error
lbm_destroy = _lib.lbm_destroy


def probe_fp64_tflops() -> float:
    """Measured FP64 rate of the current device in TFLOP/s (an FMA-chain
    probe; the denominator of the FP64 step's ALU roofline)."""
    v = C.c_double()
    rc = _lib.lbm_probe_fp64_tflops(C.byref(v))
    if rc:
        raise LBMError(rc, "FP64 probe failed")
    return v.value


def selftest_wait_timeout(limit_cycles: int):
    """Run the bounded-wait self-test: returns (status word, milliseconds);
    the word is 2 when the waits ran out after limit_cycles and returned."""
    st, ms = C.c_int(-1), C.c_double()
    rc = _lib.lbm_selftest_wait_timeout(int(limit_cycles), C.byref(st), C.byref(ms))
    if rc:
        raise LBMError(rc, "wait self-test failed")
    return st.value, ms.value


def default_params(eos: int) -> lbm_params:
    p = lbm_params()
    rc = _lib.lbm_default_params(eos, C.byref(p))
    if rc:
        raise LBMError(rc, "unknown eos")
    return p


def _ptr(a) -> int:
    """Address of a contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


class LBM:
    """One lattice on the GPU behind the C ABI.

    Host arrays (numpy float64) and device tensors (torch float64 on the
    handle's device) are both accepted where the C ABI takes ``on_device``.
    """

    def __init__(self, lattice: int, nx: int, ny: int, nz: int, eos: int, t_over_tc: float,
                 kappa: float, tau: float, mask=None, a: float | None = None,
                 b: float | None = None, acentric: float | None = None,
                 rho_w: float | None = None, flags: int = 0, storage: int = F64,
                 stream=None, torch_memory: bool = True, g=None, tau_v: float = 0.0,
                 visc_rho=None):
        import torch
        self.lattice, self.nx, self.ny, self.nz = lattice, nx, ny, nz
        self.D = 2 if lattice == D2Q9 else 3
        self.Q = 9 if lattice == D2Q9 else 27
        self.N = nx * ny * nz
        p = default_params(eos)
        if a is not None:
            p.a = a
        if b is not None:
            p.b = b
        if acentric is not None:
            p.acentric = acentric
        if rho_w is not None:
            p.rho_w = rho_w
        p.flags = flags
        p.storage = storage
        if g is not None:   # body acceleration (gx, gy[, gz])
            for a, v in enumerate(g):
                p.g[a] = float(v)
        if tau_v:   # density-dependent relaxation between visc_rho = (rho_v, rho_l)
            p.tau_v = float(tau_v)
            p.visc_rho[0], p.visc_rho[1] = map(float, visc_rho)
        self.params = p
        mptr = None
        if mask is not None:
            self._mask = np.ascontiguousarray(mask, dtype=np.uint8)
            if self._mask.size != self.N:
                raise ValueError("mask size != nx*ny*nz")
            mptr = self._mask.ctypes.data
        h = C.c_void_p()
        rc = _lib.lbm_create(C.byref(h), lattice, nx, ny, nz, eos, t_over_tc, kappa, tau,
                             mptr, C.byref(p))
        if rc:
            raise LBMError(rc, "lbm_create rejected the arguments")
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream
        if stream is not None:
            self._check(_lib.lbm_set_stream(h, C.c_void_p(stream.cuda_stream)))
        self._mem = None
        if torch_memory:
            nbytes = _lib.lbm_required_bytes(lattice, nx, ny, nz, storage)
            self._mem = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self._mem.data_ptr()
            off = (-base) % 256
            self._check(_lib.lbm_bind_device_memory(h, C.c_void_p(base + off), nbytes))

    # -- helpers -----------------------------------------------------------
    def _check(self, rc: int):
        if rc:
            msg = _lib.lbm_last_error(self._h).decode() if getattr(self, "_h", None) else ""
            raise LBMError(rc, msg)

    @staticmethod
    def _on_device(a) -> int:
        return 0 if a is None or isinstance(a, np.ndarray) else 1

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.lbm_destroy(h)
            self._h = None
        self._mem = None

    def __del__(self):
        self.close()

    # -- C ABI calls -------------------------------------------------------
    def init(self, rho0, u0=None):
        dev = self._on_device(rho0)
        if not dev:
            rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
            u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
        self._check(_lib.lbm_init(self._h, _ptr(rho0), None if u0 is None else _ptr(u0), dev))

    def step(self, n: int = 1):
        self._check(_lib.lbm_step(self._h, int(n)))

    def moments(self, out=None):
        """(rho, u, U). With ``out=None`` returns host numpy arrays; pass a
        tuple of three device tensors to fill them on the device."""
        if out is None:
            rho, u, U = np.empty(self.N), np.empty(self.D * self.N), np.empty(self.D * self.N)
            self._check(_lib.lbm_moments(self._h, rho.ctypes.data, u.ctypes.data, U.ctypes.data, 0))
            return rho, u, U
        rho, u, U = out
        self._check(_lib.lbm_moments(self._h, *(None if t is None else _ptr(t) for t in out), 1))
        return rho, u, U

    def set_wall_distances(self, q):
        """Wall distance q[i][n] in (0, 1] of the links from fluid node n
        along c_i into a solid (interpolated bounce-back); None clears."""
        if q is None:
            self._check(_lib.lbm_set_wall_distances(self._h, None))
            return
        qq = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
        if qq.size != self.Q * self.N:
            raise ValueError("q needs Q * N entries")
        self._check(_lib.lbm_set_wall_distances(self._h, qq.ctypes.data))

    def pressure_tensor(self, out=None):
        """Discrete pressure tensor [component][node] (xx, yy[, zz], xy[, xz,
        yz]); pass a device tensor of that many doubles to fill it on the
        device."""
        na = 6 if self.D == 3 else 3
        if out is None:
            out = np.empty(na * self.N)
            self._check(_lib.lbm_pressure_tensor(self._h, _ptr(out), 0))
            return out.reshape(na, self.N)
        self._check(_lib.lbm_pressure_tensor(self._h, _ptr(out), 1))
        return out

    def reduce(self):
        m = C.c_double()
        j = (C.c_double * 3)()
        self._check(_lib.lbm_reduce(self._h, C.byref(m), j))
        return m.value, np.array(j[: self.D])

    def get_populations(self, out=None):
        if out is None:
            out = np.empty(self.Q * self.N)
        self._check(_lib.lbm_get_populations(self._h, _ptr(out), self._on_device(out)))
        return out

    def set_populations(self, f):
        dev = self._on_device(f)
        if not dev:
            f = np.ascontiguousarray(f, dtype=np.float64)
        self._check(_lib.lbm_set_populations(self._h, _ptr(f), dev))

    def sync(self, timeout_ms: int = -1):
        self._check(_lib.lbm_sync(self._h, int(timeout_ms)))

    def time_kernels(self, n: int):
        """Mean (moments, collide) kernel durations in ms over n plain steps."""
        ms = (C.c_double * 2)()
        self._check(_lib.lbm_time_kernels(self._h, int(n), ms))
        return ms[0], ms[1]

    def set_chunk(self, chunk: int):
        self._check(_lib.lbm_set_chunk(self._h, int(chunk)))

    def autotune(self) -> int:
        """Time the fused step's chunk candidates (and, for FP32, its three
        forms and, for D3Q27, the 8- and 7-row tiles) on the current state
        (which is restored) and keep the fastest; returns the chunk (0 for
        FP64)."""
        c = C.c_int()
        self._check(_lib.lbm_autotune(self._h, C.byref(c)))
        return c.value

    def set_tile(self, tile_y: int):
        """Tile height of the D3Q27 FP32 step: 8 (default) or 7 rows."""
        self._check(_lib.lbm_set_tile(self._h, int(tile_y)))

    def set_fused_variant(self, variant: int):
        """Form of the fused step: FUSED_PLAIN, FUSED_WARP_SPECIALISED,
        FUSED_TMEM, FUSED_WS_TMEM, FUSED_WS_TMA or (shifted storage)
        FUSED_TM_TMA (bitwise the same results)."""
        self._check(_lib.lbm_set_fused_variant(self._h, int(variant)))

    @property
    def fused_variant(self) -> int:
        v = C.c_int()
        self._check(_lib.lbm_get_fused_variant(self._h, C.byref(v)))
        return v.value

    def tile(self):
        """(tile_x, tile_y) of the fused step in use; (0, 0) for FP64."""
        x, y = C.c_int(), C.c_int()
        self._check(_lib.lbm_get_tile(self._h, C.byref(x), C.byref(y)))
        return x.value, y.value

    @property
    def launches(self) -> int:
        return int(_lib.lbm_launch_count(self._h))

    @staticmethod
    def required_bytes(lattice, nx, ny, nz, storage=F64) -> int:
        return int(_lib.lbm_required_bytes(lattice, nx, ny, nz, storage))


class Batch:
    """Several FP32 lattices of one type advanced together (lbm_batch_*)."""

    def __init__(self, members):
        self.members = list(members)
        arr = (C.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        h = C.c_void_p()
        rc = _lib.lbm_batch_create(C.byref(h), arr, len(self.members))
        if rc:
            raise LBMError(rc, "lbm_batch_create rejected the members")
        self._h = h

    def step(self, n: int = 1):
        rc = _lib.lbm_batch_step(self._h, int(n))
        if rc:
            raise LBMError(rc, "lbm_batch_step failed")

    def sync(self):
        rc = _lib.lbm_batch_sync(self._h)
        if rc:
            raise LBMError(rc, "lbm_batch_sync")

    @property
    def launches(self) -> int:
        return int(_lib.lbm_batch_launch_count(self._h))

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.lbm_batch_destroy(h)
            self._h = None

    def __del__(self):
        self.close()
