"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

The C source is compiled on first use by ``oracle.build``. Arrays are numpy
float64 in the library layout: scalar fields ``[z][y][x]`` flattened, vector
fields as D planes, populations as Q planes.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

ZETA_LITERAL = 1
PHI_OFF = 2
FORCE_PRINTED_SIGN = 4
PHI_PRINTED_SIGN = 8

EOS_VDW, EOS_PR, EOS_RKS, EOS_CS, EOS_SC1, EOS_SC2 = 0, 1, 2, 3, 4, 5

# Default EOS constants (lattice units): van der Waals a = 9/49, b = 2/21;
# Peng-Robinson and Redlich-Kwong-Soave a = 2/49, b = 2/21, acentric 0.344
# (the paper's water value, Sec. 3.1); Carnahan-Starling a = 1, b = 4. The
# Shan-Chen forms (Appendix G) take no a, b: their b here only bounds the
# density range the Maxwell tools search (rho < 1/b).
DEFAULT_AB = {EOS_VDW: (9.0 / 49.0, 2.0 / 21.0), EOS_PR: (2.0 / 49.0, 2.0 / 21.0),
              EOS_RKS: (2.0 / 49.0, 2.0 / 21.0), EOS_CS: (1.0, 4.0),
              EOS_SC1: (1.0, 0.1), EOS_SC2: (1.0, 0.1)}
DEFAULT_ACENTRIC = 0.344

_libs = {}
_dp = C.POINTER(C.c_double)


def lib(openmp: bool = False):
    """The oracle library; openmp=True loads the -fopenmp build of the same
    source (all host cores, same results bit for bit)."""
    if openmp not in _libs:
        L = C.CDLL(_build.build(openmp=openmp))
        L.oracle_create.restype = C.c_void_p
        L.oracle_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                    C.c_double, C.c_double, C.c_void_p, C.c_double,
                                    C.c_double, C.c_double, C.c_double, C.c_int,
                                    C.c_double, C.c_double, C.c_double]
        L.oracle_destroy.argtypes = [C.c_void_p]
        L.oracle_init.argtypes = [C.c_void_p, _dp, _dp]
        L.oracle_step.argtypes = [C.c_void_p, C.c_long]
        L.oracle_moments.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.oracle_reduce.argtypes = [C.c_void_p, _dp, _dp]
        L.oracle_get_populations.argtypes = [C.c_void_p, _dp]
        L.oracle_set_populations.argtypes = [C.c_void_p, _dp]
        L.oracle_feq.argtypes = [C.c_void_p, C.c_double, _dp, _dp]
        L.oracle_fstar.argtypes = [C.c_void_p, C.c_double, _dp, _dp, _dp, _dp]
        L.oracle_stencil.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, _dp]
        L.oracle_weights.argtypes = [C.c_void_p, _dp, C.POINTER(C.c_int)]
        L.oracle_post_local.argtypes = [C.c_void_p, _dp, C.c_void_p, _dp]
        L.oracle_rt.restype = C.c_double
        L.oracle_rt.argtypes = [C.c_void_p]
        L.oracle_alpha.restype = C.c_double
        L.oracle_alpha.argtypes = [C.c_void_p]
        L.oracle_eos_pressure.restype = C.c_double
        L.oracle_eos_pressure.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                          C.c_double, C.c_double]
        L.oracle_eos_RTc.restype = C.c_double
        L.oracle_eos_RTc.argtypes = [C.c_int, C.c_double, C.c_double]
        L.oracle_eos_temperature.restype = C.c_double
        L.oracle_eos_temperature.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
        L.oracle_eos_alpha.restype = C.c_double
        L.oracle_eos_alpha.argtypes = [C.c_int, C.c_double, C.c_double]
        L.oracle_pressure_tensor.argtypes = [C.c_void_p, _dp]
        L.oracle_set_viscosity.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double]
        L.oracle_set_wall_distances.argtypes = [C.c_void_p, C.c_void_p]
        L.oracle_eos_pressure_array.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                                C.c_double, _dp, C.c_long, _dp]
        _libs[openmp] = L
    return _libs[openmp]


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


class EOS:
    """P(rho) at fixed T/Tc through the oracle's C equation of state."""

    def __init__(self, eos: int, t_over_tc: float, a: float | None = None,
                 b: float | None = None, acentric: float = DEFAULT_ACENTRIC):
        da, db = DEFAULT_AB[eos]
        self.eos = eos
        self.a = da if a is None else a
        self.b = db if b is None else b
        self.acentric = acentric
        self.t_over_tc = t_over_tc
        L = lib()
        self.RTc = L.oracle_eos_RTc(eos, self.a, self.b)
        self.RT = L.oracle_eos_temperature(eos, self.a, self.b, t_over_tc)
        self.alpha = L.oracle_eos_alpha(eos, acentric, t_over_tc)

    def __call__(self, rho):
        r = np.ascontiguousarray(np.atleast_1d(np.asarray(rho, dtype=np.float64)))
        out = np.empty_like(r)
        lib().oracle_eos_pressure_array(self.eos, self.a, self.b, self.RT, self.alpha,
                                        _p(r), r.size, _p(out))
        return out if np.ndim(rho) else float(out[0])


class OracleLBM:
    """One lattice on the CPU oracle."""

    def __init__(self, lattice: int, nx: int, ny: int, nz: int, eos: int, t_over_tc: float,
                 kappa: float, tau: float, mask: np.ndarray | None = None,
                 a: float | None = None, b: float | None = None,
                 acentric: float = DEFAULT_ACENTRIC, rho_w: float = 1.0, flags: int = 0,
                 g=(0.0, 0.0, 0.0), openmp: bool = False, tau_v: float = 0.0,
                 visc_rho=(0.0, 1.0)):
        """g: body acceleration (gx, gy[, gz]); the force rho g is added to the
        Korteweg force (the generic F of Eq. LBGK). openmp: run on the
        -fopenmp build (all host cores, same results). tau_v > 0: vapour
        relaxation time, nu linear in rho between visc_rho = (rho_v, rho_l)."""
        self._L = lib(openmp)
        self.lattice, self.nx, self.ny, self.nz = lattice, nx, ny, nz
        self.D = 2 if lattice == 0 else 3
        self.Q = 9 if lattice == 0 else 27
        self.N = nx * ny * nz
        da, db = DEFAULT_AB[eos]
        a = da if a is None else a
        b = db if b is None else b
        self._mask = None
        mp = None
        if mask is not None:
            self._mask = np.ascontiguousarray(mask, dtype=np.uint8)
            assert self._mask.size == self.N
            mp = self._mask.ctypes.data_as(C.c_void_p)
        gg = tuple(g) + (0.0,) * (3 - len(g))
        self._h = self._L.oracle_create(lattice, nx, ny, nz, eos, t_over_tc, kappa, tau, mp,
                                      a, b, acentric, rho_w, flags, *map(float, gg))
        if not self._h:
            raise ValueError("oracle_create rejected the arguments")
        if tau_v > 0.0:
            self._L.oracle_set_viscosity(self._h, float(tau_v), float(visc_rho[0]),
                                         float(visc_rho[1]))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.oracle_destroy(h)
            self._h = None

    def init(self, rho0: np.ndarray, u0: np.ndarray | None = None):
        r = np.ascontiguousarray(rho0, dtype=np.float64)
        u = np.ascontiguousarray(u0 if u0 is not None else np.zeros(self.D * self.N),
                                 dtype=np.float64)
        self._L.oracle_init(self._h, _p(r), _p(u))

    def step(self, n: int = 1):
        self._L.oracle_step(self._h, n)

    def moments(self):
        rho = np.empty(self.N)
        u = np.empty(self.D * self.N)
        U = np.empty(self.D * self.N)
        F = np.empty(self.D * self.N)
        self._L.oracle_moments(self._h, _p(rho), _p(u), _p(U), _p(F))
        return rho, u, U, F

    def reduce(self):
        m = C.c_double()
        j = np.zeros(3)
        self._L.oracle_reduce(self._h, C.byref(m), _p(j))
        return m.value, j[: self.D].copy()

    def get_populations(self) -> np.ndarray:
        out = np.empty(self.Q * self.N)
        self._L.oracle_get_populations(self._h, _p(out))
        return out

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == self.Q * self.N
        self._L.oracle_set_populations(self._h, _p(f))

    def feq(self, rho: float, u) -> np.ndarray:
        uu = np.zeros(3)
        uu[: self.D] = u
        out = np.empty(self.Q)
        self._L.oracle_feq(self._h, rho, _p(uu), _p(out))
        return out

    def fstar(self, rho: float, u, F, Phi) -> np.ndarray:
        uu, FF, PP = np.zeros(3), np.zeros(3), np.zeros(3)
        uu[: self.D], FF[: self.D], PP[: self.D] = u, F, Phi
        out = np.empty(self.Q)
        self._L.oracle_fstar(self._h, rho, _p(uu), _p(FF), _p(PP), _p(out))
        return out

    def stencil(self, g: np.ndarray, g1: float, g2: float) -> np.ndarray:
        g = np.ascontiguousarray(g, dtype=np.float64)
        out = np.zeros(3 * self.N)
        self._L.oracle_stencil(self._h, _p(g), g1, g2, _p(out))
        return out[: self.D * self.N].copy()

    def weights(self):
        w = np.empty(self.Q)
        c = np.empty(3 * self.Q, dtype=np.int32)
        self._L.oracle_weights(self._h, _p(w), c.ctypes.data_as(C.POINTER(C.c_int)))
        return w, c.reshape(self.Q, 3)

    def post_local(self, block: np.ndarray, mblock: np.ndarray) -> np.ndarray:
        """Post-collision populations of the centre of a 5x5(x5) block of
        populations block[dz][dy][dx][i] with solid flags mblock[dz][dy][dx]."""
        b = np.ascontiguousarray(block, dtype=np.float64)
        m = np.ascontiguousarray(mblock, dtype=np.uint8)
        out = np.empty(self.Q)
        self._L.oracle_post_local(self._h, _p(b), m.ctypes.data_as(C.c_void_p), _p(out))
        return out

    def set_wall_distances(self, q):
        """Wall distance q[i][n] in (0, 1] of each link from node n along c_i
        into a solid (interpolated bounce-back); None: halfway everywhere."""
        if q is None:
            self._L.oracle_set_wall_distances(self._h, None)
            return
        self._qw = np.ascontiguousarray(q, dtype=np.float64).reshape(self.Q * self.N)
        self._L.oracle_set_wall_distances(self._h, self._qw.ctypes.data_as(C.c_void_p))

    def pressure_tensor(self) -> np.ndarray:
        """Discrete pressure tensor (Appendix E): [component][node] with the
        components xx, yy[, zz], xy[, xz, yz]."""
        na = 6 if self.D == 3 else 3
        out = np.empty(na * self.N)
        self._L.oracle_pressure_tensor(self._h, _p(out))
        return out.reshape(na, self.N)

    @property
    def RT(self) -> float:
        return self._L.oracle_rt(self._h)
