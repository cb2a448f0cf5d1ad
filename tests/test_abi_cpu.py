"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every function declared in include/*.h, and its host-side argument logic
rejects bad input before touching the device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_1907_12334_gb300 import build, msg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return msg.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("msg_normals", "kl_prepare", "sample_field", "msg_workspace_bytes", "msg_solve_batch",
              "mimc_differences", "msg_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(msg.EXPORTED) <= set(declared_functions())


def test_library_is_built_for_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_and_error_strings(lib):
    assert "sm_103a" in msg.msg_version()
    assert lib.msg_last_error() == b""


def _ws(PQ, **kw):
    return msg.msg_workspace_bytes(np.array(PQ, dtype=np.int32).reshape(-1, 2), msg.SolverParams(**kw))


def test_workspace_bytes_host_logic(lib):
    one = _ws([[3, 3]])
    two = _ws([[3, 3], [3, 3]])
    assert one > 0 and two > one
    assert _ws([[8, 8]]) > _ws([[8, 7]]) > _ws([[7, 7]])
    # FP64 cycles keep 8-byte scratch and no FP32 coefficient copy
    assert _ws([[6, 6]], precision=msg.MSG_PREC_FP64) != _ws([[6, 6]], precision=msg.MSG_PREC_MIXED)
    # uneven batch is the sum of its parts up to table overhead
    mix = _ws([[2, 5], [6, 3], [1, 1]])
    assert mix > _ws([[6, 3]])


@pytest.mark.parametrize("PQ,kw", [([[0, 3]], {}), ([[3, 13]], {}), ([[3, 3]], {"mu": 0}),
                                    ([[3, 3]], {"max_cycles": 0}), ([[3, 3]], {"omega": 0.0}),
                                    ([[3, 3]], {"precision": 7}), ([[3, 3]], {"qoi": 9}),
                                    ([[3, 3]], {"eps": float("nan")}), ([[3, 3]], {"nu1": 65}),
                                    ([[3, 3]], {"tune_block": 48}), ([[3, 3]], {"tune_low_warps": 17}),
                                    ([[3, 3]], {"tune_low_items": 3}),
                                    ([[3, 3]], {"tune_low_cut": 6}), ([[3, 3]], {"tune_visit_smem": 228}),
                                    ([[3, 3]], {"tune_visit_smem": -1}),
                                    ([[3, 3]], {"tune_low_items": 8, "tune_low_warps": 8, "tune_low_cut": 5})])
def test_invalid_arguments_rejected_on_host(lib, PQ, kw):
    assert _ws(PQ, **kw) == 0
    assert lib.msg_last_error() != b""
    pq = np.array(PQ, dtype=np.int32)
    c = msg.SolverParams(**kw).c()
    rc = lib.msg_solve_batch(pq.ctypes.data_as(ctypes.c_void_p), 1, ctypes.byref(c), None, None, None, None, None,
                             None, 0, None)
    assert rc == msg.MSG_ERR_INVALID


def test_empty_batch_is_a_no_op(lib):
    c = msg.SolverParams().c()
    assert lib.msg_solve_batch(None, 0, ctypes.byref(c), None, None, None, None, None, None, 0, None) == msg.MSG_OK
    assert lib.msg_normals(0, 0, 0, 4, None, None) == msg.MSG_OK
    assert lib.msg_normals(0, 0, 3, 0, None, None) == msg.MSG_ERR_INVALID


def test_kl_prepared_bytes(lib):
    assert msg.kl_prepared_bytes(100, 16, msg.MSG_GEMM_FP64) >= 100 * 16 * 8
    assert msg.kl_prepared_bytes(100, 16, msg.MSG_GEMM_FP32) >= 100 * 16 * 4
    assert msg.kl_prepared_bytes(100, 16, 99) == 0
    # tensor-core modes: Phi padded to whole 256-point tiles and 128-byte K rows
    assert msg.kl_prepared_bytes(100, 16, msg.MSG_GEMM_BF16X3) >= 2 * 256 * 64 * 2
    assert msg.kl_prepared_bytes(100, 16, msg.MSG_GEMM_TF32) >= 256 * 32 * 4
    assert msg.kl_prepared_bytes(300, 400, msg.MSG_GEMM_TF32) >= 512 * 416 * 4


def test_mimc_rejects_bad_indices(lib):
    L = np.array([[2, 15]], dtype=np.int32)
    rc = lib.mimc_differences(L.ctypes.data_as(ctypes.c_void_p), 1, 1, 1, ctypes.c_void_p(8), None, 0, 0,
                              ctypes.c_void_p(8), None, None)
    assert rc == msg.MSG_ERR_INVALID


def test_profiling_api_host_logic(lib):
    """Counting and sampled timing: argument checks and empty reads need no GPU."""
    assert lib.msg_profile_enable(-1) == msg.MSG_ERR_INVALID
    msg.msg_profile_enable(True, stride=4)
    r = msg.msg_profile_read("PRE")
    assert r == {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0}
    assert msg.msg_profile_read_level("LOW", 4) == {"timed": 0, "ms": 0.0, "bytes": 0.0}
    n = ctypes.c_int64()
    d = ctypes.c_double()
    assert lib.msg_profile_read_level(2, -1, ctypes.byref(n), ctypes.byref(d), ctypes.byref(d)) == msg.MSG_ERR_INVALID
    assert lib.msg_profile_read(99, ctypes.byref(n), ctypes.byref(d), ctypes.byref(d), ctypes.byref(d)) == \
        msg.MSG_ERR_INVALID
    msg.msg_profile_enable(False)


def test_solution_values_count_and_grid_offsets(lib):
    """msg_solution_values = sum over samples of T(P) T(Q) nodes, T(n) = 2^(n+1) - 2 + n; grid_view
    places grid (p,q) at T(p-1) T(Q) + (2^p+1) T(q-1) and the last grid ends the block."""
    T = lambda n: (2 << n) - 2 + n
    shapes = [(3, 5), (1, 1), (8, 2)]
    assert msg.msg_solution_values(shapes) == sum(T(P) * T(Q) for P, Q in shapes)
    P, Q = 4, 3
    blk = np.arange(T(P) * T(Q), dtype=np.float64)
    seen = np.zeros(blk.size, dtype=int)
    for p in range(1, P + 1):
        for q in range(1, Q + 1):
            g = msg.grid_view(blk, P, Q, p, q)
            assert g.shape == ((1 << q) + 1, (1 << p) + 1)
            seen[g.ravel().astype(int)] += 1
    assert (seen == 1).all()  # the grids tile the block exactly
    with pytest.raises(msg.MsgError):
        msg.msg_solution_values([(0, 3)])


def test_circulant_embedding_host_logic(lib):
    """Padding (Sec. 4), workspace size, and host-side argument checks of the
    circulant-embedding sampler; no compute call."""
    assert msg.ce_padding(0.5, 4, 4) == 7
    assert msg.ce_padding(1.5, 3, 5) == 15
    assert lib.ce_padding(-1.0, 4, 4) == 0 and lib.msg_last_error() != b""
    law = msg.CeLaw(L=7, batch=3)
    P, Q = 3, 2
    M1, M2 = 7 << (P + 1), 7 << (Q + 1)
    need = 3 * (8 * M1 * M2 + 16 * M2 * (M1 // 2 + 1))
    got = msg.ce_workspace_bytes(P, Q, law)
    assert need <= got <= need + 3 * 256
    assert msg.ce_workspace_bytes(P, Q, msg.CeLaw(batch=6)) > got
    for bad in (msg.CeLaw(nu=1.0), msg.CeLaw(lam=0.0), msg.CeLaw(eta_lo=0.3, eta_hi=0.2), msg.CeLaw(L=1),
                msg.CeLaw(batch=0), msg.CeLaw(theta_lo=10.0, theta_hi=-10.0)):
        assert msg.ce_workspace_bytes(P, Q, bad) == 0 and lib.msg_last_error() != b""
    assert msg.ce_workspace_bytes(0, 3, law) == 0 and msg.ce_workspace_bytes(3, 11, law) == 0
    c = law.c()
    assert lib.ce_sample_field(P, Q, 0, ctypes.byref(c), 1, 0, None, None, None, None, 0, None) == msg.MSG_OK
    assert lib.ce_sample_field(P, Q, 2, ctypes.byref(c), 1, 0, None, None, None, None, 0, None) == msg.MSG_ERR_INVALID
    assert lib.ce_sample_field(P, Q, -1, ctypes.byref(c), 1, 0, None, None, None, None, 0, None) == msg.MSG_ERR_INVALID


def test_cycle_history_host_logic(lib):
    """Workspace size and host-side checks of the convergence-study entry point."""
    prm = msg.SolverParams()
    a = msg.msg_history_workspace_bytes(4, 3, 5, prm, msg.MSG_HIST_MSG)
    b = msg.msg_history_workspace_bytes(4, 3, 5, prm, msg.MSG_HIST_STANDARD)
    assert a > 5 * 5 * 8 * (2 ** 5 - 2 + 4) * (2 ** 4 - 2 + 3) and b > 0
    assert msg.msg_history_workspace_bytes(4, 3, 10, prm, msg.MSG_HIST_MSG) > a
    assert msg.msg_history_workspace_bytes(4, 3, 5, prm, 2) == 0 and lib.msg_last_error() != b""
    assert msg.msg_history_workspace_bytes(11, 3, 5, prm, 0) == 0
    c = prm.c()
    assert lib.msg_cycle_history(4, 3, 0, ctypes.byref(c), 0, None, 10, None, None, 0, None) == msg.MSG_OK
    assert lib.msg_cycle_history(4, 3, 2, ctypes.byref(c), 0, None, 10, None, None, 0, None) == msg.MSG_ERR_INVALID
    assert lib.msg_cycle_history(4, 3, 2, ctypes.byref(c), 0, None, 0, None, None, 0, None) == msg.MSG_ERR_INVALID
