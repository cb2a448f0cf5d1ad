"""Plain scalar FP64 CPU oracle of the MSG-MIMC hot path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
in ``paper_1907_12334_gb300``; the two meet only through the seeded input
generators in ``paper_1907_12334_gb300.inputs`` (which hold none of the
method's arithmetic).

The arithmetic lives in ``msg_oracle.c`` (compiled by :func:`build`); this
module is argument marshalling with ctypes.  Every function cites the part of
arXiv:1907.12334 it follows in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msg_oracle.c")
_LIB_PATH = os.environ.get("ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

QOI_INTEGRAL, QOI_POINT, QOI_SUBDOMAIN, QOI_FLUX = 0, 1, 2, 3
U, B, R, SOL = 0, 1, 2, 3

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile msg_oracle.c into liboracle.so next to it (plain gcc, -O2)."""
    if os.environ.get("ORACLE_LIB"):
        return _LIB_PATH  # a prebuilt variant (the mutation tests plant mistakes this way)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.orc_philox4x64_10.argtypes = [ctypes.POINTER(ctypes.c_uint64)] * 3
            L.orc_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, _dp]
            L.orc_kl_field.argtypes = [_dp, _dp, _dp, ctypes.c_int64, ctypes.c_int32, _dp]
            L.orc_hier_new.restype = ctypes.c_void_p
            L.orc_hier_new.argtypes = [ctypes.c_int, ctypes.c_int]
            L.orc_hier_free.argtypes = [ctypes.c_void_p]
            L.orc_hier_set_params.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_double, ctypes.c_double]
            L.orc_hier_set_field.argtypes = [ctypes.c_void_p, _dp]
            L.orc_hier_set_field_mode.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int]
            L.orc_hier_set_rhs.argtypes = [ctypes.c_void_p, _dp]
            L.orc_fmsg.argtypes = [ctypes.c_void_p]
            L.orc_mu_cycle.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_field_points.restype = ctypes.c_int64
            L.orc_field_points.argtypes = [ctypes.c_int, ctypes.c_int]
            L.orc_solve_sample.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_int, _dp, _ip, _dp]
            L.orc_mimc_differences.argtypes = [ctypes.c_int] * 6 + [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp]
            for name in ("orc_grid_get", "orc_grid_set"):
                getattr(L, name).argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
            L.orc_grid_apply.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp, _dp]
            L.orc_grid_smooth.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_grid_residual.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
            L.orc_grid_restrict.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_grid_interpolate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_grid_kappa.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp, _dp]
            L.orc_grid_qoi.restype = ctypes.c_double
            L.orc_grid_qoi.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
            L.orc_hier_cycles.argtypes = [ctypes.c_void_p, _ip, _dp]
            L.orc_grid_coef.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp, _dp]
            L.orc_cycle_history.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp]
            L.orc_std_block.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
            _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


# ---------------------------------------------------------------- generator --

def philox4x64_10(ctr, key) -> np.ndarray:
    """One Philox4x64-10 block (Salmon et al., SC'11)."""
    c = (ctypes.c_uint64 * 4)(*[int(v) & (2**64 - 1) for v in ctr])
    k = (ctypes.c_uint64 * 2)(*[int(v) & (2**64 - 1) for v in key])
    o = (ctypes.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return np.array(list(o), dtype=np.uint64)


def normals(seed: int, s: int, M: int) -> np.ndarray:
    """xi[0..M) ~ N(0,1) of global sample number s (Philox4x64-10 + Box-Muller)."""
    xi = np.empty(M, dtype=np.float64)
    lib().orc_normals(seed, s, M, _d(xi))
    return xi


def normals_batch(seed: int, s0: int, S: int, M: int) -> np.ndarray:
    return np.stack([normals(seed, s0 + i, M) for i in range(S)]) if S else np.zeros((0, M))


def kl_field(Phi: np.ndarray, sqrt_lambda: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Z = Phi diag(sqrt(lambda)) xi for one sample, FP64, K-ordered sum."""
    Phi = np.ascontiguousarray(Phi, dtype=np.float64)
    npts, M = Phi.shape
    Z = np.empty(npts, dtype=np.float64)
    lib().orc_kl_field(_d(Phi), _d(np.ascontiguousarray(sqrt_lambda, dtype=np.float64)),
                       _d(np.ascontiguousarray(xi, dtype=np.float64)), npts, M, _d(Z))
    return Z


def field_points(P: int, Q: int) -> int:
    return int(lib().orc_field_points(P, Q))


# ------------------------------------------------------------------- solver --

COEF_HARMONIC, COEF_INJECTION = 0, 1


class SolverParams:
    def __init__(self, mu=2, nu1=2, nu2=2, max_cycles=50, eps=1e-12, omega=1.0, qoi=QOI_INTEGRAL,
                 coef=COEF_HARMONIC):
        self.mu, self.nu1, self.nu2, self.max_cycles = mu, nu1, nu2, max_cycles
        self.eps, self.omega, self.qoi, self.coef = eps, omega, qoi, coef


def solve_sample(P: int, Q: int, Z: np.ndarray, prm: SolverParams | None = None):
    """FMSG (Algorithm 2 with W(nu1,nu2) mu-cycles of Algorithm 1) on one sample.

    Returns (Qgrid [P][Q], status, cycles [P][Q], relres [P][Q])."""
    prm = prm or SolverParams()
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    assert Z.size == field_points(P, Q)
    Qg = np.empty(P * Q, dtype=np.float64)
    cyc = (ctypes.c_int * (P * Q))()
    rr = np.empty(P * Q, dtype=np.float64)
    st = lib().orc_solve_sample(P, Q, _d(Z), prm.mu, prm.nu1, prm.nu2, prm.max_cycles, prm.eps,
                                prm.omega, prm.qoi, prm.coef, _d(Qg), cyc, _d(rr))
    if st < 0:
        raise ValueError("oracle: invalid shape")
    return Qg.reshape(P, Q), st, np.array(list(cyc)).reshape(P, Q), rr.reshape(P, Q)


def solve_batch(shapes, Zs, prm: SolverParams | None = None, threads: int | None = None):
    """solve_sample over many samples, one sample per thread (ctypes drops the GIL)."""
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda a: solve_sample(a[0][0], a[0][1], a[1], prm), zip(shapes, Zs)))


def mimc_differences(L, p0, q0, Qgrid: np.ndarray, ptau: np.ndarray | None = None):
    """dQ_tau for 0<=tau<=L (Eq. (3.2)) and Y = sum dQ_tau / p_tau (Eq. (3.6))."""
    L1, L2 = int(L[0]), int(L[1])
    Qgrid = np.ascontiguousarray(Qgrid, dtype=np.float64)
    Pn, Qn = Qgrid.shape
    dQ = np.empty((L1 + 1) * (L2 + 1), dtype=np.float64)
    Y = ctypes.c_double(np.nan)
    if ptau is not None:
        ptau = np.ascontiguousarray(ptau, dtype=np.float64)
        ld1, ld2 = ptau.shape
        pp = _d(ptau)
    else:
        ld1 = ld2 = 0
        pp = None
    rc = lib().orc_mimc_differences(L1, L2, p0, q0, Pn, Qn, _d(Qgrid), pp, ld1, ld2, _d(dQ),
                                    ctypes.byref(Y))
    if rc:
        raise ValueError("oracle: index out of the solved hierarchy")
    return dQ.reshape(L1 + 1, L2 + 1), (Y.value if ptau is not None else None)


class Hierarchy:
    """Handle on one sample's grid hierarchy, for the building-block pin tests."""

    def __init__(self, P: int, Q: int, Z: np.ndarray | None = None, prm: SolverParams | None = None,
                 rhs: np.ndarray | None = None):
        self.P, self.Q = P, Q
        self.h = lib().orc_hier_new(P, Q)
        if not self.h:
            raise ValueError("oracle: invalid shape")
        prm = prm or SolverParams()
        self.prm = prm
        lib().orc_hier_set_params(self.h, prm.mu, prm.nu1, prm.nu2, prm.max_cycles, prm.eps, prm.omega)
        if Z is None:
            Z = np.zeros(field_points(P, Q))
        self.Z = np.ascontiguousarray(Z, dtype=np.float64)
        lib().orc_hier_set_field_mode(self.h, _d(self.Z), prm.coef)
        self.set_rhs(rhs)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_hier_free(self.h)
            self.h = None

    def set_rhs(self, rhs=None):
        if rhs is None:
            lib().orc_hier_set_rhs(self.h, None)
        else:
            r = np.ascontiguousarray(rhs, dtype=np.float64)
            assert r.shape == ((1 << self.Q) + 1, (1 << self.P) + 1)
            lib().orc_hier_set_rhs(self.h, _d(r))

    @staticmethod
    def shape(p, q):
        return ((1 << q) + 1, (1 << p) + 1)

    def get(self, p, q, which=U):
        out = np.empty(self.shape(p, q))
        assert lib().orc_grid_get(self.h, p, q, which, _d(out)) == 0
        return out

    def set(self, p, q, which, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        assert a.shape == self.shape(p, q)
        assert lib().orc_grid_set(self.h, p, q, which, _d(a)) == 0

    def cycle_history(self, method: int, ncycles: int) -> np.ndarray:
        """||r_k||/||b|| on the finest grid after k = 0..ncycles cycles from u = 0, b = 1;
        method 0: MSG cycles (Algorithm 1), 1: standard coarsening."""
        h = np.empty(ncycles + 1)
        assert lib().orc_cycle_history(self.h, method, ncycles, _d(h)) == 0
        return h

    def std_restrict(self, p, q, f):
        out = np.empty(self.shape(p - 1, q - 1))
        assert lib().orc_std_block(self.h, p, q, 0, _d(np.ascontiguousarray(f, dtype=np.float64)), _d(out)) == 0
        return out

    def std_prolong(self, p, q, e):
        out = np.empty(self.shape(p, q))
        assert lib().orc_std_block(self.h, p, q, 1, _d(np.ascontiguousarray(e, dtype=np.float64)), _d(out)) == 0
        return out

    def line_solve(self, p, q, b):
        out = np.empty(self.shape(p, q))
        assert lib().orc_std_block(self.h, p, q, 2, _d(np.ascontiguousarray(b, dtype=np.float64)), _d(out)) == 0
        return out

    def coef(self, p, q):
        """(ax [(ny+1)][nx], ay [ny][nx+1]): a at the x- and y-face midpoints of grid (p,q)."""
        nx, ny = 1 << p, 1 << q
        ax = np.empty((ny + 1, nx))
        ay = np.empty((ny, nx + 1))
        assert lib().orc_grid_coef(self.h, p, q, _d(ax), _d(ay)) == 0
        return ax, ay

    def apply(self, p, q, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.empty(self.shape(p, q))
        assert lib().orc_grid_apply(self.h, p, q, _d(v), _d(out)) == 0
        return out

    def smooth(self, p, q, sweeps=1):
        assert lib().orc_grid_smooth(self.h, p, q, sweeps) == 0

    def residual(self, p, q):
        assert lib().orc_grid_residual(self.h, p, q) == 0
        return self.get(p, q, R)

    def restrict(self, p, q, src=0):
        assert lib().orc_grid_restrict(self.h, p, q, src) == 0
        return self.get(p, q, B)

    def interpolate(self, p, q, mode=0):
        assert lib().orc_grid_interpolate(self.h, p, q, mode) == 0
        return self.get(p, q, U)

    def kappa(self, p, q):
        kx = np.empty(self.shape(p, q))
        ky = np.empty(self.shape(p, q))
        assert lib().orc_grid_kappa(self.h, p, q, _d(kx), _d(ky)) == 0
        return kx, ky

    def mu_cycle(self, s):
        lib().orc_mu_cycle(self.h, s)

    def fmsg(self):
        st = lib().orc_fmsg(self.h)
        n = self.P * self.Q
        cyc = (ctypes.c_int * n)()
        rr = np.empty(n)
        lib().orc_hier_cycles(self.h, cyc, _d(rr))
        return st, np.array(list(cyc)).reshape(self.P, self.Q), rr.reshape(self.P, self.Q)

    def qoi(self, p, q, which=SOL, qoi=QOI_INTEGRAL):
        return lib().orc_grid_qoi(self.h, p, q, which, qoi, _d(self.Z))
