"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (per result):
  xi (Philox4x64-10 + Box-Muller)  |d| <= 1e-14 (1 + |xi|): integer streams are
                                   identical, the FP64 transcendentals of the two
                                   math libraries may differ in the last bits;
  Z, FP64 KL contraction           |d| <= 1e-13 sum_m |Phi sqrt(lambda) xi| (summation order);
  Q per grid, FP64 cycles          relative 1e-10;
  Q per grid, mixed cycles         relative 1e-8 (FP32 cycles under FP64 refinement);
  dQ, Y                            bit-exact given the same Q (same operation order).
Inputs: seeded synthetic lognormal fields (Matern nu = 3/2, corr. lengths 0.2/0.02)
computed by the oracle from the shared KL basis.
"""
import numpy as np
import pytest

import oracle
from paper_1907_12334_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def msg():
    from paper_1907_12334_gb300 import build, msg as m

    build.build()
    m.load()
    return m


DEV = "cuda:0"


def oracle_fields(shapes, M=32, seed=0, s0=0):
    """Z of each sample by the oracle's own generator and KL sum (FP64)."""
    out = []
    for k, (P, Q) in enumerate(shapes):
        Phi, sl = inputs.kl_basis(P, Q, inputs.small_law(M))
        out.append(oracle.kl_field(Phi, sl, oracle.normals(seed, s0 + k, M)))
    return out


def run_gpu(msg, shapes, Zs, **kw):
    prm = msg.SolverParams(**kw)
    Zd = torch.from_numpy(np.concatenate(Zs)).to(DEV)
    Q, st, cyc, rr = msg.solve(np.array(shapes, dtype=np.int32), Zd, prm)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), st.cpu().numpy(), cyc.cpu().numpy(), rr.cpu().numpy()


def run_oracle(shapes, Zs, eps, max_cycles, qoi=oracle.QOI_INTEGRAL, coef=oracle.COEF_HARMONIC):
    res = oracle.solve_batch(shapes, Zs, oracle.SolverParams(eps=eps, max_cycles=max_cycles, qoi=qoi, coef=coef))
    Q = np.concatenate([r[0].ravel() for r in res])
    st = np.array([r[1] for r in res])
    cyc = np.concatenate([r[2].ravel() for r in res])
    return Q, st, cyc


# ------------------------------------------------------------------ (a1) --

def test_normals_match_oracle(msg):
    S, M = 37, 402  # ragged tail: M not a multiple of 4
    xi = torch.empty((S, M), dtype=torch.float64, device=DEV)
    msg.msg_normals(1234, 77, S, M, xi)
    g = xi.cpu().numpy()
    o = oracle.normals_batch(1234, 77, S, M)
    np.testing.assert_allclose(g, o, rtol=1e-14, atol=1e-14)


# ------------------------------------------------------------------ (a2) --

@pytest.mark.parametrize("mode,tol,M,S,zf32", [("FP64", 1e-13, 40, 70, False), ("FP32", 2e-6, 40, 70, False),
                                               ("BF16X3", 5e-5, 40, 70, False), ("BF16X3", 5e-5, 400, 300, False),
                                               ("BF16X3", 5e-5, 400, 300, True), ("TF32", 1.2e-3, 40, 70, False),
                                               ("TF32", 1.2e-3, 400, 300, False), ("TF32", 1.2e-3, 400, 300, True)])
def test_kl_contraction(msg, mode, tol, M, S, zf32):
    """BF16X3 and TF32 run on the tcgen05 tensor cores with FP32 accumulation.
    BF16X3: hi*hi + hi*lo + lo*hi of bf16 splits, error bound 3 2^-18 per product
    plus FP32 accumulation.  TF32: both operands rounded to 10-bit mantissas
    (relative error <= 2^-11 each), one product per term: bound 2^-10 + 2^-22 per
    product plus accumulation, tested at 1.2e-3.  zf32: Z written as FP32."""
    P, Q = 4, 3  # ragged: npts and S not multiples of the 256 x 128 tile
    Phi, sl = inputs.kl_basis(P, Q, inputs.small_law(M))
    npts = Phi.shape[0]
    xi_o = oracle.normals_batch(5, 0, S, M)
    Z_o = np.stack([oracle.kl_field(Phi, sl, xi_o[i]) for i in range(S)])
    m = getattr(msg, f"MSG_GEMM_{mode}")
    prep = torch.empty(msg.kl_prepared_bytes(npts, M, m), dtype=torch.uint8, device=DEV)
    msg.kl_prepare(torch.from_numpy(np.ascontiguousarray(Phi)).to(DEV), torch.from_numpy(sl.copy()).to(DEV), m, prep)
    xi = torch.empty((S, M), dtype=torch.float64, device=DEV)
    msg.msg_normals(5, 0, S, M, xi)
    Z = torch.empty((S, npts), dtype=torch.float32 if zf32 else torch.float64, device=DEV)
    msg.sample_field(prep, npts, M, m, xi, Z)
    scale = np.abs(Phi * sl[None, :]) @ np.abs(xi_o).T  # sum_m |Phi_xm sqrt(l_m) xi_sm|
    err = np.abs(Z.double().cpu().numpy() - Z_o)
    # an FP32 output adds its own rounding of |Z| <= scale
    assert np.all(err <= (tol + (6e-8 if zf32 else 0.0)) * scale.T + 1e-300)
    msg.msg_device_status()


# ------------------------------------------------------------- (a3)-(a13) --

SHAPES_SMALL = [(1, 1), (1, 4), (4, 1), (2, 3), (3, 5), (5, 5), (4, 4)]


@pytest.mark.parametrize("precision,rtol", [("FP64", 1e-10), ("MIXED", 1e-8)])
def test_solve_uneven_batch_matches_oracle(msg, precision, rtol):
    shapes = SHAPES_SMALL + [(5, 5), (3, 3)]
    Zs = oracle_fields(shapes)
    eps, mc = 1e-11, 400
    Qo, sto, cyco = run_oracle(shapes, Zs, eps, mc)
    Qg, stg, cycg, rrg = run_gpu(msg, shapes, Zs, eps=eps, max_cycles=mc,
                                 precision=getattr(msg, f"MSG_PREC_{precision}"))
    assert np.array_equal(stg, sto)
    np.testing.assert_allclose(Qg, Qo, rtol=rtol, atol=0)
    assert np.all(rrg <= eps)
    if precision == "FP64":
        # same iteration: cycle counts agree except at a tolerance boundary
        assert np.mean(cycg == cyco) > 0.9 and np.all(np.abs(cycg - cyco) <= 1)


@pytest.mark.parametrize("qoi", [1, 2, 3])
def test_other_quantities_of_interest(msg, qoi):
    shapes = [(4, 4), (3, 5), (2, 2)]
    Zs = oracle_fields(shapes, seed=3)
    Qo, _, _ = run_oracle(shapes, Zs, 1e-11, 400, qoi=qoi)
    Qg, _, _, _ = run_gpu(msg, shapes, Zs, eps=1e-11, max_cycles=400, precision=msg.MSG_PREC_MIXED, qoi=qoi)
    nan = np.isnan(Qo)
    assert np.array_equal(nan, np.isnan(Qg))
    np.testing.assert_allclose(Qg[~nan], Qo[~nan], rtol=1e-8)


def test_injected_coefficients(msg):
    shapes = [(4, 4), (2, 5), (5, 2)]
    Zs = oracle_fields(shapes, seed=5)
    Qo, sto, _ = run_oracle(shapes, Zs, 1e-11, 600, coef=oracle.COEF_INJECTION)
    Qg, stg, _, _ = run_gpu(msg, shapes, Zs, eps=1e-11, max_cycles=600, precision=msg.MSG_PREC_MIXED,
                            coef=msg.MSG_COEF_INJECT)
    assert np.array_equal(stg, sto)
    np.testing.assert_allclose(Qg, Qo, rtol=1e-8)


def test_v_cycle_and_damping_parameters(msg):
    shapes = [(4, 3), (3, 4)]
    Zs = oracle_fields(shapes, seed=9)
    prm = oracle.SolverParams(mu=1, nu1=1, nu2=3, omega=0.9, eps=1e-11, max_cycles=600)
    res = oracle.solve_batch(shapes, Zs, prm)
    Qo = np.concatenate([r[0].ravel() for r in res])
    Qg, stg, _, _ = run_gpu(msg, shapes, Zs, mu=1, nu1=1, nu2=3, omega=0.9, eps=1e-11, max_cycles=600,
                            precision=msg.MSG_PREC_FP64)
    np.testing.assert_allclose(Qg, Qo, rtol=1e-10)


def test_status_not_converged_and_nonfinite(msg):
    shapes = [(3, 3), (3, 3)]
    Zs = oracle_fields(shapes)
    NFx = (1 << 4) + 1
    Zs[1] = Zs[1].copy()
    Zs[1][8 * NFx + 7] = np.nan
    _, sto, cyco = run_oracle(shapes, Zs, 0.0, 3)
    _, stg, cycg, _ = run_gpu(msg, shapes, Zs, eps=0.0, max_cycles=3, precision=msg.MSG_PREC_FP64)
    assert np.array_equal(stg, sto)
    assert stg[0] == msg.MSG_SAMPLE_NOT_CONVERGED and stg[1] & msg.MSG_SAMPLE_NONFINITE


def test_workspace_too_small_is_reported(msg):
    pq = np.array([[3, 3]], dtype=np.int32)
    prm = msg.SolverParams()
    Z = torch.zeros(msg.field_points(3, 3), dtype=torch.float64, device=DEV)
    Q = torch.empty(9, dtype=torch.float64, device=DEV)
    ws = torch.empty(msg.msg_workspace_bytes(pq, prm) // 2, dtype=torch.uint8, device=DEV)
    with pytest.raises(msg.MsgError, match="error 2"):
        msg.msg_solve_batch(pq, prm, Z, Q, workspace=ws)


def test_result_independent_of_batch_mix(msg):
    """A sample's result is the same alone and inside a mixed batch (bit-exact)."""
    shapes = [(4, 4), (2, 5), (4, 4), (3, 2)]
    Zs = oracle_fields(shapes, seed=11)
    Qmix, _, _, _ = run_gpu(msg, shapes, Zs, eps=1e-10, max_cycles=400)
    Qalone, _, _, _ = run_gpu(msg, [shapes[1]], [Zs[1]], eps=1e-10, max_cycles=400)
    assert np.array_equal(Qmix[16:26], Qalone)


@pytest.mark.parametrize("shape", [dict(tune_low_warps=3), dict(tune_low_items=1), dict(tune_low_items=4, tune_low_warps=1),
                                   dict(tune_low_items=8, tune_low_warps=1), dict(tune_block=64, tune_low_warps=1),
                                   dict(tune_block=256, tune_low_warps=4)])
def test_launch_shapes_do_not_change_results(msg, shape):
    """Launch shapes only regroup independent per-node updates: bit-exact results.
    The batch mixes shapes (items of several low-diagonal classes in one CTA)
    and has an item count that leaves warps of the last CTA idle."""
    shapes = SHAPES_SMALL + [(2, 6), (6, 2), (5, 4)]
    Zs = oracle_fields(shapes, seed=5)
    ref = run_gpu(msg, shapes, Zs, eps=1e-10, max_cycles=300)
    got = run_gpu(msg, shapes, Zs, eps=1e-10, max_cycles=300, **shape)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("cut,shape", [(1, {}), (3, {}), (5, dict(tune_low_items=1, tune_low_warps=8))])
def test_low_kernel_cut_changes_rounding_only(msg, cut, shape):
    """The diagonal up to which the low-diagonal kernel runs the recursion (the rest
    are separate visit launches) changes only the rounding of the FP32 cycles: every
    grid still meets eps and the QoIs agree with the default cut and with the oracle
    to the mixed path's 1e-8."""
    shapes = SHAPES_SMALL + [(2, 6), (6, 2), (5, 4), (6, 6)]
    Zs = oracle_fields(shapes, seed=8)
    ref = run_gpu(msg, shapes, Zs, eps=1e-10, max_cycles=300)
    got = run_gpu(msg, shapes, Zs, eps=1e-10, max_cycles=300, tune_low_cut=cut, **shape)
    assert np.array_equal(ref[1], got[1]) and (got[1] == 0).all()
    assert np.all(got[3] <= 1e-10)
    np.testing.assert_allclose(got[0], ref[0], rtol=1e-8)
    Qo, _, _ = run_oracle(shapes, Zs, 1e-12, 600)
    np.testing.assert_allclose(got[0], Qo, rtol=1e-8)


@pytest.mark.parametrize("limit", [1, 8, 227])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_shared_memory_visits_change_rounding_only(msg, limit, precision):
    """Visits above the cut run register-cached (u in shared memory, each
    node's coefficients and right-hand side in registers) up to a shared-memory
    limit and in global memory beyond it (1 KB: every visit in global memory;
    8 KB: the two paths on different diagonals of one hierarchy; 227 KB: every
    grid small enough for the register path).  The per-node arithmetic is the
    same up to the compiler's rounding: every grid meets eps and the QoIs agree
    with the default limit and with the oracle."""
    shapes = SHAPES_SMALL + [(2, 6), (6, 2), (5, 4), (6, 6), (8, 2), (1, 8)]
    Zs = oracle_fields(shapes, seed=9)
    kw = dict(eps=1e-10, max_cycles=300)
    if precision == "fp64":
        kw.update(precision=msg.MSG_PREC_FP64, eps=1e-11)
    ref = run_gpu(msg, shapes, Zs, **kw)
    got = run_gpu(msg, shapes, Zs, tune_visit_smem=limit, **kw)
    assert (got[1] == 0).all() and (ref[1] == 0).all()
    assert np.all(got[3] <= 1e-10)
    tol = 1e-8 if precision == "mixed" else 1e-10
    np.testing.assert_allclose(got[0], ref[0], rtol=tol)
    Qo, _, _ = run_oracle(shapes, Zs, 1e-12, 600)
    np.testing.assert_allclose(got[0], Qo, rtol=tol)


# ------------------------------------------------------------------ (a14) --

def test_mimc_differences_bit_exact(msg):
    rng = np.random.default_rng(4)
    p0, q0 = 2, 1
    Ls = [(0, 0), (2, 3), (1, 0), (0, 2), (3, 3)]
    Qs = [rng.standard_normal((p0 + a, q0 + b)) for a, b in Ls]
    ptau = np.exp(-1.7 * (np.arange(5)[:, None] + np.arange(5)[None, :]))
    Qd = torch.from_numpy(np.concatenate([q.ravel() for q in Qs])).to(DEV)
    nd = sum((a + 1) * (b + 1) for a, b in Ls)
    dQ = torch.empty(nd, dtype=torch.float64, device=DEV)
    Y = torch.empty(len(Ls), dtype=torch.float64, device=DEV)
    msg.mimc_differences(np.array(Ls, dtype=np.int32), p0, q0, Qd, dQ, ptau=ptau, Y=Y)
    torch.cuda.synchronize()
    off = 0
    for k, (L, Qg) in enumerate(zip(Ls, Qs)):
        d_o, y_o = oracle.mimc_differences(L, p0, q0, Qg, ptau=ptau)
        n = d_o.size
        assert np.array_equal(dQ[off:off + n].cpu().numpy(), d_o.ravel())
        assert Y[k].item() == y_o
        off += n


# ------------------------------------------------------- full-size sample --

def test_full_size_256_sampled_against_oracle(msg):
    """The bench workload's shape (finest 256 x 256, all 64 grids, M = 400 KL terms)
    in a batch of 32, mixed cycles; three samples re-solved by the oracle."""
    P = Q = 8
    S, M = 32, 400
    Phi, sl = inputs.kl_basis(P, Q, inputs.FieldLaw(M=M))
    xi = oracle.normals_batch(0, 0, S, M)
    Zs = [oracle.kl_field(Phi, sl, xi[i]) for i in range(S)]
    eps = 1e-10
    Qg, stg, cycg, rrg = run_gpu(msg, [(P, Q)] * S, Zs, eps=eps, max_cycles=400)
    ok = stg == 0
    # every grid of a converged sample meets eps; non-convergence is rare and reported
    assert ok.mean() >= 0.9
    assert np.all(rrg.reshape(S, -1)[ok] <= eps)
    pick = [i for i in (0, 13, 31, 5, 7) if ok[i]][:3]
    Qo, sto, _ = run_oracle([(P, Q)] * len(pick), [Zs[i] for i in pick], 1e-12, 600)
    Qg = Qg.reshape(S, P * Q)[pick].ravel()
    np.testing.assert_allclose(Qg, Qo, rtol=1e-8)


def test_uneven_index_set_sampled_against_oracle(msg):
    """The uneven workload's structure (indices (a1,a2) in 0..7, grids 2^(a+2): 4..512 per
    side, shuffled in one call), reduced to 64 samples; every converged grid meets eps and
    the smaller samples are re-solved by the oracle."""
    shapes = inputs.uneven_shapes(64, k=2, amax=7, seed=3)
    M = 32
    Zs = oracle_fields(shapes, M=M, seed=7)
    eps = 1e-10
    Qg, stg, cycg, rrg = run_gpu(msg, shapes, Zs, eps=eps, max_cycles=400)
    ok = stg == 0
    assert ok.mean() >= 0.9
    offs = np.cumsum([0] + [p * q for p, q in shapes])
    for i in np.nonzero(ok)[0]:
        assert np.all(rrg[offs[i]:offs[i + 1]] <= eps)
    pick = [i for i in range(len(shapes)) if ok[i] and max(shapes[i]) <= 6][:6]
    Qo, _, _ = run_oracle([shapes[i] for i in pick], [Zs[i] for i in pick], 1e-12, 600)
    Qsel = np.concatenate([Qg[offs[i]:offs[i + 1]] for i in pick])
    np.testing.assert_allclose(Qsel, Qo, rtol=1e-8)


def test_mimc_differences_is_asynchronous_and_reads_host_tables_before_returning(msg):
    """The call enqueues its work without waiting for the stream: the host index and
    p_tau arrays are staged before it returns (overwriting them right after the call
    changes nothing), and many calls in flight on one stream, each with its own
    tables, all give the oracle's differences bit for bit."""
    rng = np.random.default_rng(12)
    p0, q0 = 1, 2
    stream = torch.cuda.Stream()
    calls = []
    with torch.cuda.stream(stream):
        for c in range(24):
            Ls = [(int(a), int(b)) for a, b in rng.integers(0, 4, size=(5 + c, 2))]
            Qs = [rng.standard_normal((p0 + a, q0 + b)) for a, b in Ls]
            Qd = torch.from_numpy(np.concatenate([q.ravel() for q in Qs])).to(DEV)
            nd = sum((a + 1) * (b + 1) for a, b in Ls)
            dQ = torch.empty(nd, dtype=torch.float64, device=DEV)
            Y = torch.empty(len(Ls), dtype=torch.float64, device=DEV)
            Lh = np.array(Ls, dtype=np.int32)
            ptau = np.exp(-0.9 * (np.arange(4)[:, None] + np.arange(4)[None, :]))
            msg.mimc_differences(Lh, p0, q0, Qd, dQ, ptau=ptau, Y=Y, stream=stream)
            Lh[:] = 7  # the library must not read these after returning
            ptau[:] = np.nan
            calls.append((Ls, Qs, Qd, dQ, Y))
    stream.synchronize()
    ptau = np.exp(-0.9 * (np.arange(4)[:, None] + np.arange(4)[None, :]))
    for Ls, Qs, _, dQ, Y in calls:
        off = 0
        for k, (L, Qg) in enumerate(zip(Ls, Qs)):
            d_o, y_o = oracle.mimc_differences(L, p0, q0, Qg, ptau=ptau)
            assert np.array_equal(dQ[off:off + d_o.size].cpu().numpy(), d_o.ravel())
            assert Y[k].item() == y_o
            off += d_o.size


def test_bf16x3_sampler_reports_through_the_status_query(msg):
    """The tensor-core sampler no longer stops the stream to read its pipeline flag;
    msg_device_status reports a bounded wait that ran out (none here)."""
    P, Q, M, S = 3, 3, 40, 130
    Phi, sl = inputs.kl_basis(P, Q, inputs.small_law(M))
    npts = Phi.shape[0]
    m = msg.MSG_GEMM_BF16X3
    prep = torch.empty(msg.kl_prepared_bytes(npts, M, m), dtype=torch.uint8, device=DEV)
    msg.kl_prepare(torch.from_numpy(np.ascontiguousarray(Phi)).to(DEV), torch.from_numpy(sl.copy()).to(DEV), m, prep)
    xi = torch.empty((S, M), dtype=torch.float64, device=DEV)
    msg.msg_normals(3, 0, S, M, xi)
    Z = torch.empty((S, npts), dtype=torch.float64, device=DEV)
    msg.sample_field(prep, npts, M, m, xi, Z)
    msg.msg_device_status()  # raises on MSG_ERR_TIMEOUT
    xo = oracle.normals_batch(3, 0, S, M)
    Zo = np.stack([oracle.kl_field(Phi, sl, xo[i]) for i in range(S)])
    scale = np.abs(xo * sl) @ np.abs(Phi).T  # sum_m |sqrt(lambda_m) xi_m Phi_xm|
    assert np.all(np.abs(Z.cpu().numpy() - Zo) <= 5e-5 * scale)
