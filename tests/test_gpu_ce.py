"""Parity of the circulant-embedding sampler (ce_sample_field, through the C ABI)
with its oracle (oracle/circulant.py), on the same seeded inputs.

eta, theta: the same 53-bit uniforms; FP64 affine maps -> relative 1e-15.
Z: the GPU takes the eigenvalues in FP64 (as the oracle), then forms
a = sqrt(Lambda / M) (xi1 + i xi2) and its transform in FP32.  The transform's
rounding error per output is at most about u log2(M) ||a||_2 (u = 2^-24), and
the single-precision Box-Muller adds at most a few u of each |xi| <= 8.6, whose
contribution is again bounded by u ||a||_2-sized terms; ||a||_2^2 = sum_k
Lambda_k |xi_k|^2 / M is computed here from the oracle.  The test allows
4 u (log2 M + 8) ||a||_2 per node.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import circulant as ce

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def msg():
    from paper_1907_12334_gb300 import build, msg as m

    build.build()
    m.load()
    return m


def _bound(P, Q, law, eta, theta, seed, s):
    lam = ce.eigenvalues(ce.generating_array(P, Q, law, eta, theta))
    M1, M2 = ce.embed_size(P, Q, law.L)
    xi = oracle.normals(seed, s, 2 * M1 * M2)
    a2 = np.sum(np.maximum(lam.ravel(), 0) / lam.size * (xi[0::2] ** 2 + xi[1::2] ** 2))
    return 4 * 2.0 ** -24 * (math.log2(M1 * M2) + 8) * math.sqrt(a2)


def _run(msg, P, Q, S, law_kw, seed, s0, batch):
    gl = msg.CeLaw(batch=batch, **law_kw)
    ol = ce.CeLaw(**law_kw)
    nf = oracle.field_points(P, Q)
    Z = torch.full((S, nf), float("nan"), dtype=torch.float64, device=DEV)
    et = torch.empty((S, 2), dtype=torch.float64, device=DEV)
    st = torch.full((S,), -1, dtype=torch.int32, device=DEV)
    msg.ce_sample_field(P, Q, S, gl, seed, s0, Z, et, st)
    torch.cuda.synchronize()
    Z, et, st = Z.cpu().numpy(), et.cpu().numpy(), st.cpu().numpy()
    for i in range(S):
        Zo, eta, theta, ratio = ce.ce_field(P, Q, ol, seed, s0 + i)
        # both sides set negative eigenvalues to zero; the flag marks one below -1e-10 of the largest
        assert st[i] == (msg.MSG_CE_NEGATIVE_EIGENVALUE if ratio < -1e-10 else 0), (i, st[i], ratio)
        assert et[i, 0] == pytest.approx(eta, rel=1e-15) and et[i, 1] == pytest.approx(theta, rel=1e-15, abs=1e-16)
        err = np.max(np.abs(Z[i] - Zo))
        tol = _bound(P, Q, ol, eta, theta, seed, s0 + i)
        assert err <= tol, (i, err, tol)
    return Z


@pytest.mark.parametrize("P,Q,S,batch,law_kw", [(3, 3, 5, 2, {}), (2, 4, 3, 3, {}), (4, 1, 4, 4, dict(nu=1.5)),
                                                (1, 1, 2, 1, dict(nu=2.5, lam=0.1, L=5)), (3, 4, 3, 2, dict(scale=1))])
def test_ce_fields_match_oracle(msg, P, Q, S, batch, law_kw):
    """Ragged last batch (S not a multiple of batch), anisotropic grids, the three
    smoothness values, a smaller padding."""
    _run(msg, P, Q, S, law_kw, seed=11, s0=3, batch=batch)


def test_ce_fields_full_size_256(msg):
    """The bench's field shape (256 x 256 grids: 513 x 513 field nodes) with the
    bench's padding L = 9 (a 4608 x 4608 periodic grid), two samples in one batch:
    positive definite, no flag."""
    _run(msg, 8, 8, 2, dict(L=9), seed=20190729, s0=40, batch=2)


def test_ce_negative_eigenvalues_flagged_like_the_oracle(msg):
    """With the paper's padding L = 7 at a 1/512 field spacing these two samples'
    embeddings have eigenvalues down to -2e-7 of the largest: both sides set them
    to zero, the GPU flags the samples, and the fields still agree."""
    Z = _run(msg, 8, 8, 2, dict(L=7), seed=20190729, s0=40, batch=2)
    assert np.isfinite(Z).all()


def test_ce_field_solves_like_the_oracle(msg):
    """A circulant-embedding field through msg_solve_batch agrees with the
    oracle's solve of the oracle's field (sampler and solver error together)."""
    P = Q = 4
    Z = _run(msg, P, Q, 2, {}, seed=5, s0=0, batch=2)
    prm = msg.SolverParams(eps=1e-10, max_cycles=400)
    Qg, stg, _, _ = msg.solve(np.array([[P, Q]] * 2, dtype=np.int32), torch.from_numpy(Z.ravel()).to(DEV), prm)
    torch.cuda.synchronize()
    res = oracle.solve_batch([(P, Q)] * 2, [ce.ce_field(P, Q, ce.CeLaw(), 5, s)[0] for s in range(2)],
                             oracle.SolverParams(eps=1e-12, max_cycles=600))
    Qo = np.concatenate([r[0].ravel() for r in res])
    assert (stg.cpu().numpy() == 0).all()
    np.testing.assert_allclose(Qg.cpu().numpy(), Qo, rtol=1e-4)
