"""Adaptive MSG-MIMC driver (host bookkeeping) and the continuous-batching server."""
import math

import numpy as np
import pytest

from paper_1907_12334_gb300.serving import MimcDriver, geometric_tail


def test_initial_law_is_algorithm3_geometric():
    """Algorithm 3: pi_L = GEOMETRIC^d(log(2)(1+4)/2), i.e. P(L_j >= k) = exp(-r k), r = 1.7329."""
    d = MimcDriver(eps=1e-3, lmax=(5, 5))
    r = 0.5 * math.log(2) * 5
    assert r == pytest.approx(1.7328679513998633)
    np.testing.assert_allclose(d.tail[:, 0], np.exp(-r * np.arange(6)), rtol=1e-14)
    np.testing.assert_allclose(d.tail, np.outer(d.tail[:, 0], d.tail[0, :]), rtol=1e-14)
    assert d.tail[1, 0] == pytest.approx(2 ** -2.5, rel=1e-14)
    pmf = d.pmf()
    assert np.all(pmf >= 0) and pmf.sum() == pytest.approx(1.0, abs=1e-12)  # truncated tail folds into lmax
    # P(L >= tau) recovered from the pmf by summing the upper-right block
    for a in range(6):
        for b in range(6):
            assert pmf[a:, b:].sum() == pytest.approx(d.tail[a, b], rel=1e-12, abs=1e-15)


def test_draws_follow_the_law():
    d = MimcDriver(eps=1e-3, lmax=(4, 4), seed=3)
    L = np.array(d.draw(200000))
    emp = np.zeros((5, 5))
    np.add.at(emp, (L[:, 0], L[:, 1]), 1)
    emp /= emp.sum()
    np.testing.assert_allclose(emp, d.pmf(), atol=3e-3)


def test_estimator_unbiased_on_synthetic_differences():
    """Unbiasedness of Eq. (3.5) (telescoping, Sec. 3): with dQ_tau of known means the
    running E converges to sum_tau E[dQ_tau] = E[Q]."""
    rng = np.random.default_rng(0)
    d = MimcDriver(eps=0.0, lmax=(3, 3), seed=1, learn_every=10**9)
    means = np.array([[1.0, 0.3, 0.1, 0.03], [0.4, 0.1, 0.02, 0.01], [0.1, 0.03, 0.01, 0.0], [0.02, 0.01, 0.0, 0.0]])
    for L in d.draw(40000):
        a, b = L[0] + 1, L[1] + 1
        dq = means[:a, :b] + 0.05 * rng.standard_normal((a, b)) * means[:a, :b]
        d.record(L, dq, d.tail)
    assert d.E == pytest.approx(means.sum(), abs=4 * math.sqrt(d.V))
    assert math.sqrt(d.V) < 0.02


def test_learned_law_is_a_monotone_tail():
    rng = np.random.default_rng(2)
    d = MimcDriver(eps=1e-6, lmax=(3, 3), learn_every=50)
    for L in d.draw(2000):
        a, b = L[0] + 1, L[1] + 1
        d.record(L, rng.standard_normal((a, b)) * 2.0 ** (-np.add.outer(np.arange(a), np.arange(b))), d.tail)
    t = d.tail
    assert t[0, 0] == 1.0
    assert np.all(np.diff(t, axis=0) <= 1e-15) and np.all(np.diff(t, axis=1) <= 1e-15)
    assert np.all(t > 0)


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    """A request's QoIs and differences are the same when it runs alone and when it
    shares concurrent batches with other requests (bit-exact: items are independent)."""
    torch = pytest.importorskip("torch")
    from paper_1907_12334_gb300 import msg
    from paper_1907_12334_gb300.serving import Request, Server

    prm = msg.SolverParams(eps=1e-10, max_cycles=300)
    drv = MimcDriver(eps=1e-3, lmax=(3, 3), seed=5)
    Ls = drv.draw(40)
    reqs = [Request(rid=i, sample=i, L=L, shape=drv.shape(L), ptau=drv.tail) for i, L in enumerate(Ls)]
    srv = Server(hbm_budget_bytes=2 << 30, max_batch=7, slots=3, M=32, prm=prm)
    mixed = {r.rid: r for r in srv.serve(reqs)}
    assert len(mixed) == len(reqs)
    for i in (0, 7, 19, 33):
        alone = Server(hbm_budget_bytes=2 << 30, max_batch=1, slots=1, M=32, prm=prm)
        one = alone.serve([Request(rid=i, sample=i, L=Ls[i], shape=drv.shape(Ls[i]), ptau=drv.tail)])[0]
        assert np.array_equal(one.Q, mixed[i].Q)
        assert np.array_equal(one.dQ, mixed[i].dQ)
    st = Server.latency_stats(list(mixed.values()))
    assert st["p99_ms"] >= st["p50_ms"] > 0
    del torch


@pytest.mark.gpu
def test_admission_respects_the_hbm_budget():
    pytest.importorskip("torch")
    from paper_1907_12334_gb300 import msg
    from paper_1907_12334_gb300.serving import Request, Server

    prm = msg.SolverParams(eps=1e-8, max_cycles=100)
    srv = Server(hbm_budget_bytes=1, max_batch=8, slots=2, M=16, prm=prm)
    out = srv.serve([Request(rid=0, sample=0, L=(0, 0), shape=(2, 2), ptau=np.ones((1, 1)))])
    assert srv.rejected == 1 and out[0].status == -1
    small = srv.request_bytes([(2, 2)])
    srv2 = Server(hbm_budget_bytes=int(2.5 * small), max_batch=8, slots=3, M=16, prm=prm)
    out2 = srv2.serve([Request(rid=i, sample=i, L=(0, 0), shape=(2, 2), ptau=np.ones((1, 1))) for i in range(6)])
    assert len(out2) == 6 and all(r.status == 0 for r in out2) and srv2.rejected == 0


def test_failed_batch_is_marked_and_skipped_by_the_driver():
    """A library error inside a batch marks every request of that batch as failed
    (status -2, no Q/dQ); the driver leaves them out of E and V and counts them per
    multi-index instead of crashing on the missing differences."""
    import contextlib
    import types

    from paper_1907_12334_gb300 import serving
    from paper_1907_12334_gb300.serving import Request, Server

    class Boom(RuntimeError):
        pass

    def fail(*a, **k):
        raise Boom("libmsgmimc error 3: simulated failure")

    fake_msg = types.SimpleNamespace(packed_sizes=fail, field_points=lambda P, Q: 1,
                                     msg_workspace_bytes=lambda pq, prm: 0)
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(stream=lambda st: contextlib.nullcontext()))
    srv = Server.__new__(Server)
    srv.torch, srv.msg, srv.prm, srv.M = fake_torch, fake_msg, None, 8
    srv.streams, srv.busy, srv.done, srv.failures = [None], [True], [], []
    srv.cv, srv.in_use, srv.batches = serving.threading.Condition(), 0, 0
    drv = MimcDriver(eps=1e-3, lmax=(2, 2))
    reqs = [Request(rid=i, sample=i, L=(i % 2, 1), shape=drv.shape((i % 2, 1)), ptau=drv.tail) for i in range(3)]
    srv._run_batch(0, reqs)
    assert [r.status for r in srv.done] == [serving.STATUS_BATCH_FAILED] * 3
    assert all(r.Q is None and r.dQ is None and "simulated" in r.error for r in srv.done)
    assert len(srv.failures) == 1 and srv.busy == [False]
    ok = Request(rid=9, sample=9, L=(0, 0), shape=drv.shape((0, 0)), ptau=drv.tail, dQ=np.ones((1, 1)))
    for r in srv.done + [ok]:
        drv.take(r)
    assert drv.n == 1 and drv.E == 1.0
    assert drv.skipped_report() == {"batch_failed": {(0, 1): 2, (1, 1): 1}}
    nc = Request(rid=10, sample=10, L=(2, 2), shape=drv.shape((2, 2)), ptau=drv.tail, status=1)
    nf = Request(rid=11, sample=11, L=(2, 0), shape=drv.shape((2, 0)), ptau=drv.tail, status=3)
    drv.take(nc)
    drv.take(nf)
    rep = drv.skipped_report()
    assert rep["not_converged"] == {(2, 2): 1} and rep["nonfinite"] == {(2, 0): 1}


@pytest.mark.gpu
def test_served_results_match_the_oracle():
    """Requests served through continuous batching (several concurrent batches,
    uneven shapes) against the oracle solving the same fields: each grid's Q to the
    mixed path's relative 1e-8, and dQ to 1e-8 max|Q| (differences tend to zero, so
    they are compared absolutely at the scale of Q)."""
    pytest.importorskip("torch")
    import oracle
    from paper_1907_12334_gb300 import inputs, msg
    from paper_1907_12334_gb300.serving import Request, Server

    M, seed = 24, 4
    prm = msg.SolverParams(eps=1e-10, max_cycles=400)
    drv = MimcDriver(eps=1e-3, lmax=(3, 3), seed=11)
    Ls = drv.draw(18)
    reqs = [Request(rid=i, sample=100 + i, L=L, shape=drv.shape(L), ptau=drv.tail) for i, L in enumerate(Ls)]
    srv = Server(hbm_budget_bytes=2 << 30, max_batch=5, slots=3, M=M, seed=seed, prm=prm)
    done = {r.rid: r for r in srv.serve(reqs)}
    assert len(done) == len(reqs) and not srv.failures
    checked = 0
    for r in reqs:
        got = done[r.rid]
        if got.status != 0:
            continue
        P, Qn = r.shape
        Phi, sl = inputs.kl_basis(P, Qn, inputs.FieldLaw(M=M))
        Z = oracle.kl_field(Phi, sl, oracle.normals(seed, r.sample, M))
        Qo, st, _, _ = oracle.solve_sample(P, Qn, Z, oracle.SolverParams(eps=1e-12, max_cycles=600))
        assert st == 0
        np.testing.assert_allclose(got.Q, Qo, rtol=1e-8)
        dQo, _ = oracle.mimc_differences(r.L, srv.p0, srv.q0, Qo)
        np.testing.assert_allclose(got.dQ, dQo, rtol=0, atol=1e-8 * np.abs(Qo).max())
        checked += 1
    assert checked >= 0.9 * len(reqs)


def test_measured_cost_and_learned_law_use_it():
    """The measured work of a solve weights each grid's cycles by the W-cycle work of
    that grid as top (p q 2^(p+q)); once solves at an index are timed, Algorithm 3's
    update uses their mean measured cost in place of the 2^(p+q) prior."""
    from paper_1907_12334_gb300.serving import measured_cost

    cyc = np.array([[1, 2], [3, 4]])
    assert measured_cost(cyc) == 1 * 1 * 1 * 4 + 2 * 1 * 2 * 8 + 3 * 2 * 1 * 8 + 4 * 2 * 2 * 16
    rng = np.random.default_rng(1)
    a = MimcDriver(eps=1e-6, lmax=(2, 2), learn_every=10**9)
    b = MimcDriver(eps=1e-6, lmax=(2, 2), learn_every=10**9)
    for L in a.draw(3000):
        dq = rng.standard_normal((L[0] + 1, L[1] + 1)) * 0.5 ** np.add.outer(np.arange(L[0] + 1), np.arange(L[1] + 1))
        a.record(L, dq, a.tail)
        # index (1, 1) measured 64x more expensive than the prior says, the others as the prior
        c = b.cost[L[0], L[1]] * (64.0 if L == (1, 1) else 1.0)
        b.record(L, dq, b.tail, cost=c)
    a.learn()
    b.learn()
    assert b.tail[1, 1] < a.tail[1, 1]  # the costlier index is drawn less often
    assert b.tail[0, 0] == a.tail[0, 0] == 1.0
