"""The allocation-free entry point mimc_differences_noalloc.

Some callers may not allocate device memory once they are running (their own
pool already reserves all of it, or their loop cannot pay for an allocator
call).  For them the library offers a variant of mimc_differences whose
scratch lives in a fixed array of the library's own device memory.  This file
is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def msg():
    from paper_1907_12334_gb300 import build, msg as m

    build.build()
    m.load()
    return m


def _case(rng, p0, q0, Ls):
    Qs = [rng.standard_normal((p0 + a, q0 + b)) for a, b in Ls]
    nd = sum((a + 1) * (b + 1) for a, b in Ls)
    return np.concatenate([q.ravel() for q in Qs]), nd


@pytest.mark.parametrize("with_ptau", [True, False])
def test_noalloc_matches_allocating_entry_point_twice(msg, with_ptau):
    """Two calls in a row through the C ABI, each compared with mimc_differences
    on the same inputs; the results are bit-exact (same kernel, same operation order)."""
    rng = np.random.default_rng(17)
    cases = [(2, 1, [(0, 0), (2, 3), (1, 0), (0, 2), (3, 3)] * 7),
             (1, 3, [(4, 1), (0, 0), (2, 2)] * 11 + [(1, 4)])]
    for p0, q0, Ls in cases:
        Qh, nd = _case(rng, p0, q0, Ls)
        Q = torch.from_numpy(Qh).cuda()
        L = np.array(Ls, dtype=np.int32)
        ptau = np.exp(-1.7 * (np.arange(6)[:, None] + np.arange(6)[None, :])) if with_ptau else None
        out = {}
        for name, fn in (("alloc", msg.mimc_differences), ("noalloc", msg.mimc_differences_noalloc)):
            dQ = torch.full((nd,), np.nan, dtype=torch.float64, device="cuda")
            Y = torch.full((len(Ls),), np.nan, dtype=torch.float64, device="cuda")
            fn(L, p0, q0, Q, dQ, ptau=ptau, Y=Y)
            torch.cuda.synchronize()
            out[name] = (dQ.cpu().numpy(), Y.cpu().numpy())
        assert np.array_equal(out["noalloc"][0], out["alloc"][0])
        assert np.array_equal(out["noalloc"][1], out["alloc"][1])


def test_noalloc_rejects_batches_beyond_its_fixed_scratch(msg):
    """A batch whose table exceeds the fixed 16 MiB array is refused before any device work."""
    lib = msg.load()
    S = 800_000
    L = np.zeros((S, 2), dtype=np.int32)
    fn = lib.mimc_differences_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    dummy = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = fn(L.ctypes.data_as(ctypes.c_void_p), S, 1, 1, ctypes.c_void_p(dummy.data_ptr()), None, 0, 0,
            ctypes.c_void_p(dummy.data_ptr()), None, None)
    assert rc == msg.MSG_ERR_INVALID
    assert b"fixed" in lib.msg_last_error()


def _raw(msg):
    lib = msg.load()
    fn = lib.mimc_differences_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    return lib, fn


def test_noalloc_fills_its_scratch_exactly_and_rejects_one_row_more(msg):
    """The limit is the table (24 bytes per sample, rounded up to 256) plus the
    ptau table: a batch that fills the 16 MiB array exactly runs and matches
    mimc_differences; the same batch with one more ptau row is refused, and a
    ptau table larger than the whole array is refused with its own message."""
    S = 699_040  # 24 S = 16 776 960 bytes = 65 535 x 256, leaving 256 bytes = a 4 x 8 ptau table
    rng = np.random.default_rng(3)
    Ls = np.zeros((S, 2), dtype=np.int32)
    Ls[::97] = (3, 7)
    Ls[5::89] = (1, 2)
    p0 = q0 = 1
    nq = int(((p0 + Ls[:, 0]) * (q0 + Ls[:, 1])).sum())
    nd = int(((Ls[:, 0] + 1) * (Ls[:, 1] + 1)).sum())
    Q = torch.from_numpy(rng.standard_normal(nq)).cuda()
    ptau = np.exp(-1.3 * (np.arange(4)[:, None] + np.arange(8)[None, :]))
    out = {}
    for name, fn in (("alloc", msg.mimc_differences), ("noalloc", msg.mimc_differences_noalloc)):
        dQ = torch.full((nd,), np.nan, dtype=torch.float64, device="cuda")
        Y = torch.full((S,), np.nan, dtype=torch.float64, device="cuda")
        fn(Ls, p0, q0, Q, dQ, ptau=ptau, Y=Y)
        torch.cuda.synchronize()
        out[name] = (dQ.cpu().numpy(), Y.cpu().numpy())
    assert np.array_equal(out["noalloc"][0], out["alloc"][0])
    assert np.array_equal(out["noalloc"][1], out["alloc"][1])
    lib, fn = _raw(msg)
    dummy = torch.empty(1, dtype=torch.float64, device="cuda")
    dp = ctypes.c_void_p(dummy.data_ptr())
    big = np.exp(-1.3 * (np.arange(5)[:, None] + np.arange(8)[None, :]))
    rc = fn(Ls.ctypes.data_as(ctypes.c_void_p), S, p0, q0, dp, big.ctypes.data_as(ctypes.c_void_p), 5, 8, dp, dp,
            None)
    assert rc == msg.MSG_ERR_INVALID and b"fixed" in lib.msg_last_error()
    huge = np.ones((1500, 1500))
    rc = fn(Ls.ctypes.data_as(ctypes.c_void_p), 1, p0, q0, dp, huge.ctypes.data_as(ctypes.c_void_p), 1500, 1500, dp,
            dp, None)
    assert rc == msg.MSG_ERR_INVALID and b"ptau table alone" in lib.msg_last_error()
