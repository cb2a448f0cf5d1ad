"""Thin ctypes binding of the C ABI in ``include/msg_mimc.h``.

Argument marshalling only: every step of the path runs in the CUDA library
``libmsgmimc.so``.  Loading fails loudly when the library has not been built
(``paper_1907_12334_gb300.build.build()``); there is no CPU fallback.

Device buffers are torch tensors (PyTorch provides device memory and streams);
the library sees raw pointers and the current torch CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

MSG_OK, MSG_ERR_INVALID, MSG_ERR_WORKSPACE, MSG_ERR_CUDA, MSG_ERR_UNSUPPORTED, MSG_ERR_TIMEOUT = 0, 1, 2, 3, 4, 5
MSG_SAMPLE_NOT_CONVERGED, MSG_SAMPLE_NONFINITE = 1, 2
MSG_PREC_FP64, MSG_PREC_MIXED = 0, 1
MSG_QOI_INTEGRAL, MSG_QOI_POINT, MSG_QOI_SUBDOMAIN, MSG_QOI_FLUX = 0, 1, 2, 3
MSG_GEMM_FP64, MSG_GEMM_BF16X3, MSG_GEMM_FP32, MSG_GEMM_TF32 = 0, 1, 2, 3
MSG_COEF_SERIES, MSG_COEF_INJECT = 0, 1

EXPORTED = ("msg_normals", "kl_prepared_bytes", "kl_prepare", "sample_field", "msg_workspace_bytes",
            "msg_solve_batch", "msg_solution_values", "msg_solution", "mimc_differences",
            "mimc_differences_noalloc", "msg_device_status", "msg_last_error", "msg_version",
            "msg_launch_count",
            "msg_profile_enable", "msg_profile_read", "msg_profile_read_level",
            "ce_padding", "ce_workspace_bytes", "ce_sample_field", "msg_history_workspace_bytes",
            "msg_cycle_history")
MSG_HIST_MSG, MSG_HIST_STANDARD = 0, 1
MSG_CE_NEGATIVE_EIGENVALUE = 1
KERNEL_CLASSES = ("PRE", "POST", "LOW", "RESIDUAL", "UPDATE", "INTERP", "QOI", "COEFFS", "NORMALS", "KL", "MIMC",
                  "CE")


class MsgError(RuntimeError):
    pass


class msg_params(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_int32), ("nu1", ctypes.c_int32), ("nu2", ctypes.c_int32),
                ("max_cycles", ctypes.c_int32), ("eps", ctypes.c_double), ("omega", ctypes.c_double),
                ("precision", ctypes.c_int32), ("qoi", ctypes.c_int32), ("coef", ctypes.c_int32),
                ("tune_block", ctypes.c_int32), ("tune_low_warps", ctypes.c_int32),
                ("tune_low_items", ctypes.c_int32), ("tune_low_cut", ctypes.c_int32),
                ("tune_visit_smem", ctypes.c_int32)]


@dataclass
class SolverParams:
    """W(nu1,nu2) FMSG parameters (Sec. 2 numerical setup: mu=2, nu1=nu2=2)."""
    mu: int = 2
    nu1: int = 2
    nu2: int = 2
    max_cycles: int = 200
    eps: float = 1e-10
    omega: float = 1.0
    precision: int = MSG_PREC_MIXED
    qoi: int = MSG_QOI_INTEGRAL
    coef: int = MSG_COEF_SERIES
    tune_block: int = 0      # launch shape only (no effect on results): 0 = library default
    tune_low_warps: int = 0
    tune_low_items: int = 0
    tune_low_cut: int = 0    # schedule: highest diagonal inside the low-diagonal kernel (0 = default)
    tune_visit_smem: int = 0  # schedule: KB limit of the register-cached visits (0 = default: none)

    def c(self) -> msg_params:
        return msg_params(self.mu, self.nu1, self.nu2, self.max_cycles, self.eps, self.omega, self.precision,
                          self.qoi, self.coef, self.tune_block, self.tune_low_warps,
                          self.tune_low_items, self.tune_low_cut, self.tune_visit_smem)


class msg_ce_law(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("lam", ctypes.c_double), ("eta_lo", ctypes.c_double),
                ("eta_hi", ctypes.c_double), ("theta_lo", ctypes.c_double), ("theta_hi", ctypes.c_double),
                ("L", ctypes.c_int32), ("batch", ctypes.c_int32), ("scale", ctypes.c_int32)]


@dataclass
class CeLaw:
    """Field law of the paper's experiments (Sec. 4): Matern nu = 1/2, lambda = 1/4,
    eta ~ U[1/16, 1/4], theta ~ U[-30, 30] degrees; L = 7 is ce_padding(1/2, 4, 4)."""
    nu: float = 0.5
    lam: float = 0.25
    eta_lo: float = 1.0 / 16
    eta_hi: float = 0.25
    theta_lo: float = -30.0
    theta_hi: float = 30.0
    L: int = 7
    batch: int = 8
    scale: int = 0  # 0: S as Sec. 1 prints it; 1: lambda as a length (see msg_mimc.h)

    def c(self) -> msg_ce_law:
        return msg_ce_law(self.nu, self.lam, self.eta_lo, self.eta_hi, self.theta_lo, self.theta_hi, self.L,
                          self.batch, self.scale)


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libmsgmimc.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise MsgError(f"CUDA library not built: {path} is missing (run paper_1907_12334_gb300.build.build())")
    L = ctypes.CDLL(path)
    vp, i32, i64, u64, dbl, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_double, ctypes.c_size_t)
    L.msg_normals.argtypes = [u64, u64, i64, i32, vp, vp]
    L.msg_normals.restype = i32
    L.kl_prepared_bytes.argtypes = [i64, i32, i32]
    L.kl_prepared_bytes.restype = sz
    L.kl_prepare.argtypes = [vp, vp, i64, i32, i32, vp, sz, vp]
    L.kl_prepare.restype = i32
    L.sample_field.argtypes = [vp, i64, i32, i32, vp, i64, vp, i32, vp]
    L.sample_field.restype = i32
    L.msg_workspace_bytes.argtypes = [vp, i64, ctypes.POINTER(msg_params)]
    L.msg_workspace_bytes.restype = sz
    L.msg_solve_batch.argtypes = [vp, i64, ctypes.POINTER(msg_params), vp, vp, vp, vp, vp, vp, sz, vp]
    L.msg_solve_batch.restype = i32
    L.msg_solution_values.argtypes = [vp, i64]
    L.msg_solution_values.restype = i64
    L.msg_solution.argtypes = [vp, i64, ctypes.POINTER(msg_params), vp, sz, vp, vp]
    L.msg_solution.restype = i32
    L.mimc_differences.argtypes = [vp, i64, i32, i32, vp, vp, i32, i32, vp, vp, vp]
    L.mimc_differences.restype = i32
    L.msg_device_status.argtypes = []
    L.msg_device_status.restype = i32
    L.msg_last_error.argtypes = []
    L.msg_last_error.restype = ctypes.c_char_p
    L.msg_version.argtypes = []
    L.msg_version.restype = ctypes.c_char_p
    L.msg_launch_count.argtypes = []
    L.msg_launch_count.restype = i64
    L.msg_profile_enable.argtypes = [i32]
    L.msg_profile_enable.restype = i32
    L.msg_profile_read_level.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]
    L.msg_profile_read_level.restype = i32
    L.msg_profile_read.argtypes = [i32, ctypes.POINTER(i64), ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                   ctypes.POINTER(dbl)]
    L.msg_profile_read.restype = i32
    L.ce_padding.argtypes = [dbl, i32, i32]
    L.ce_padding.restype = i32
    L.ce_workspace_bytes.argtypes = [i32, i32, ctypes.POINTER(msg_ce_law)]
    L.ce_workspace_bytes.restype = sz
    L.ce_sample_field.argtypes = [i32, i32, i64, ctypes.POINTER(msg_ce_law), u64, u64, vp, vp, vp, vp, sz, vp]
    L.ce_sample_field.restype = i32
    L.msg_history_workspace_bytes.argtypes = [i32, i32, i64, ctypes.POINTER(msg_params), i32]
    L.msg_history_workspace_bytes.restype = sz
    L.msg_cycle_history.argtypes = [i32, i32, i64, ctypes.POINTER(msg_params), i32, vp, i32, vp, vp, sz, vp]
    L.msg_cycle_history.restype = i32
    _lib = L
    return L


def _check(rc: int):
    if rc != MSG_OK:
        raise MsgError(f"libmsgmimc error {rc}: {load().msg_last_error().decode()}")


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _host_i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def field_points(P: int, Q: int) -> int:
    return ((1 << (P + 1)) + 1) * ((1 << (Q + 1)) + 1)


# ------------------------------------------------------------------- ABI ----

def msg_normals(seed: int, s0: int, S: int, M: int, xi, stream=None):
    _check(load().msg_normals(seed, s0, S, M, _ptr(xi), _stream(stream)))


def kl_prepared_bytes(npts: int, M: int, mode: int) -> int:
    return int(load().kl_prepared_bytes(npts, M, mode))


def kl_prepare(Phi, sqrt_lambda, mode: int, prepared, stream=None):
    npts, M = Phi.shape
    _check(load().kl_prepare(_ptr(Phi), _ptr(sqrt_lambda), npts, M, mode, _ptr(prepared),
                             prepared.numel() * prepared.element_size(), _stream(stream)))


def sample_field(prepared, npts: int, M: int, mode: int, xi, Z, stream=None):
    import torch

    S = xi.shape[0]
    _check(load().sample_field(_ptr(prepared), npts, M, mode, _ptr(xi), S, _ptr(Z),
                               1 if Z.dtype == torch.float32 else 0, _stream(stream)))


def ce_padding(nu: float, p0: int, q0: int) -> int:
    return int(load().ce_padding(nu, p0, q0))


def ce_workspace_bytes(P: int, Q: int, law: CeLaw) -> int:
    c = law.c()
    return int(load().ce_workspace_bytes(P, Q, ctypes.byref(c)))


def ce_sample_field(P: int, Q: int, S: int, law: CeLaw, seed: int, s0: int, Z, eta_theta=None, status=None,
                    workspace=None, stream=None):
    """Z[S][field_points(P, Q)] (device, FP64) from the circulant-embedding sampler;
    workspace: a device byte tensor of ce_workspace_bytes(P, Q, law) (allocated if None)."""
    import torch

    c = law.c()
    if workspace is None:
        workspace = torch.empty(ce_workspace_bytes(P, Q, law), dtype=torch.uint8, device=Z.device)
    _check(load().ce_sample_field(P, Q, S, ctypes.byref(c), seed, s0, _ptr(Z), _ptr(eta_theta), _ptr(status),
                                  _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream)))


def msg_history_workspace_bytes(P: int, Q: int, S: int, prm: SolverParams, method: int) -> int:
    c = prm.c()
    return int(load().msg_history_workspace_bytes(P, Q, S, ctypes.byref(c), method))


def msg_cycle_history(P: int, Q: int, S: int, prm: SolverParams, method: int, Z, ncycles: int, hist=None,
                      workspace=None, stream=None):
    """Residual history [S][ncycles + 1] of plain cycles from u = 0 (FP64): method
    MSG_HIST_MSG or MSG_HIST_STANDARD.  Returns the device tensor hist."""
    import torch

    c = prm.c()
    if hist is None:
        hist = torch.empty((S, ncycles + 1), dtype=torch.float64, device=Z.device)
    if workspace is None:
        workspace = torch.empty(msg_history_workspace_bytes(P, Q, S, prm, method), dtype=torch.uint8,
                                device=Z.device)
    _check(load().msg_cycle_history(P, Q, S, ctypes.byref(c), method, _ptr(Z), ncycles, _ptr(hist),
                                    _ptr(workspace), workspace.numel() * workspace.element_size(),
                                    _stream(stream)))
    return hist


def msg_workspace_bytes(PQ, prm: SolverParams) -> int:
    pq = _host_i32(PQ).reshape(-1, 2)
    c = prm.c()
    return int(load().msg_workspace_bytes(pq.ctypes.data_as(ctypes.c_void_p), pq.shape[0], ctypes.byref(c)))


def msg_solve_batch(PQ, prm: SolverParams, Z, Qout, status=None, cycles=None, relres=None, workspace=None,
                    stream=None):
    pq = _host_i32(PQ).reshape(-1, 2)
    c = prm.c()
    _check(load().msg_solve_batch(pq.ctypes.data_as(ctypes.c_void_p), pq.shape[0], ctypes.byref(c), _ptr(Z),
                                  _ptr(Qout), _ptr(status), _ptr(cycles), _ptr(relres), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _stream(stream)))


def msg_solution_values(PQ) -> int:
    pq = _host_i32(PQ).reshape(-1, 2)
    n = int(load().msg_solution_values(pq.ctypes.data_as(ctypes.c_void_p), pq.shape[0]))
    if n < 0:
        raise MsgError(load().msg_last_error().decode())
    return n


def msg_solution(PQ, prm: SolverParams, workspace, u_out, stream=None):
    """FP64 solutions of every grid, from a workspace msg_solve_batch has just filled."""
    pq = _host_i32(PQ).reshape(-1, 2)
    c = prm.c()
    _check(load().msg_solution(pq.ctypes.data_as(ctypes.c_void_p), pq.shape[0], ctypes.byref(c), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), _ptr(u_out), _stream(stream)))


def grid_view(u_block, P: int, Q: int, p: int, q: int):
    """Grid (p,q) of one sample's solution block (see msg_solution) as a [2^q+1, 2^p+1] array view."""
    T = lambda n: (2 << n) - 2 + n
    o = T(p - 1) * T(Q) + ((1 << p) + 1) * T(q - 1)
    return u_block[o:o + ((1 << p) + 1) * ((1 << q) + 1)].reshape((1 << q) + 1, (1 << p) + 1)


def mimc_differences(L, p0: int, q0: int, Q, dQ, ptau=None, Y=None, stream=None):
    Lh = _host_i32(L).reshape(-1, 2)
    if ptau is not None:
        pt = np.ascontiguousarray(np.asarray(ptau, dtype=np.float64))
        ld1, ld2 = pt.shape
        pp = pt.ctypes.data_as(ctypes.c_void_p)
    else:
        ld1 = ld2 = 0
        pp = None
    _check(load().mimc_differences(Lh.ctypes.data_as(ctypes.c_void_p), Lh.shape[0], p0, q0, _ptr(Q), pp, ld1, ld2,
                                   _ptr(dQ), _ptr(Y), _stream(stream)))


def msg_device_status():
    """Raise if a bounded wait inside a library kernel ran out since the last call."""
    _check(load().msg_device_status())


def msg_version() -> str:
    return load().msg_version().decode()


def msg_launch_count() -> int:
    return int(load().msg_launch_count())


def msg_profile_enable(on: bool, stride: int = 1):
    """Count every launch per kernel class and time a random 1/stride of them (on=False stops)."""
    _check(load().msg_profile_enable(int(stride) if on else 0))


def msg_profile_read(kernel_class) -> dict:
    """{launches, ms, bytes, flops} of one class since msg_profile_enable: all launches
    counted; ms, bytes and flops of the timed ones scaled to all launches."""
    k = KERNEL_CLASSES.index(kernel_class) if isinstance(kernel_class, str) else int(kernel_class)
    n = ctypes.c_int64()
    ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().msg_profile_read(k, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by), ctypes.byref(fl)))
    return {"launches": n.value, "ms": ms.value, "bytes": by.value, "flops": fl.value}


def msg_profile_read_level(kernel_class, level: int) -> dict:
    """{timed, ms, bytes} over the timed launches of one class at one multigrid diagonal."""
    k = KERNEL_CLASSES.index(kernel_class) if isinstance(kernel_class, str) else int(kernel_class)
    n = ctypes.c_int64()
    ms, by = ctypes.c_double(), ctypes.c_double()
    _check(load().msg_profile_read_level(k, int(level), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
    return {"timed": n.value, "ms": ms.value, "bytes": by.value}


# ------------------------------------------------------------ conveniences --

def packed_sizes(PQ):
    pq = _host_i32(PQ).reshape(-1, 2)
    nq = int((pq[:, 0].astype(np.int64) * pq[:, 1]).sum())
    nf = int(sum(field_points(int(P), int(Q)) for P, Q in pq))
    return nq, nf


def solve(PQ, Z, prm: SolverParams | None = None, stream=None, with_u: bool = False):
    """Allocate outputs + workspace with torch and run msg_solve_batch.

    Returns (Q, status, cycles, relres) as device tensors (Q/cycles/relres packed per sample),
    and the FP64 solutions of every grid (msg_solution layout) as a fifth item if with_u."""
    import torch

    prm = prm or SolverParams()
    pq = _host_i32(PQ).reshape(-1, 2)
    nq, nf = packed_sizes(pq)
    assert Z.numel() == nf and Z.dtype == torch.float64 and Z.is_cuda
    dev = Z.device
    Q = torch.empty(nq, dtype=torch.float64, device=dev)
    status = torch.empty(pq.shape[0], dtype=torch.int32, device=dev)
    cycles = torch.empty(nq, dtype=torch.int32, device=dev)
    relres = torch.empty(nq, dtype=torch.float64, device=dev)
    ws = torch.empty(msg_workspace_bytes(pq, prm), dtype=torch.uint8, device=dev)
    msg_solve_batch(pq, prm, Z, Q, status, cycles, relres, ws, stream)
    if with_u:
        u = torch.empty(msg_solution_values(pq), dtype=torch.float64, device=dev)
        msg_solution(pq, prm, ws, u, stream)
        return Q, status, cycles, relres, u
    return Q, status, cycles, relres


def mimc_differences_noalloc(L, p0: int, q0: int, Q, dQ, ptau=None, Y=None, stream=None):
    """Same as mimc_differences, with its scratch in the library's fixed device array."""
    lib = load()
    fn = lib.mimc_differences_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    Lh = _host_i32(L).reshape(-1, 2)
    if ptau is not None:
        pt = np.ascontiguousarray(np.asarray(ptau, dtype=np.float64))
        ld1, ld2 = pt.shape
        pp = pt.ctypes.data_as(ctypes.c_void_p)
    else:
        ld1 = ld2 = 0
        pp = None
    _check(fn(Lh.ctypes.data_as(ctypes.c_void_p), Lh.shape[0], p0, q0, _ptr(Q), pp, ld1, ld2, _ptr(dQ), _ptr(Y),
              _stream(stream)))
