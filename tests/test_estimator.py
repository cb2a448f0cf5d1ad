"""Host logic of the reuse analysis (paper_1907_12334_gb300/estimator.py, Sec. 3)
against what Theorem 1 and the estimator's definition fix.

* Theorem 1 in closed form for d = 2, (1 - x1)(1 - x2), and the Table 1
  ratios (0.753 / 0.515 / 0.387) from the golden rates file.
* On exact product-model data (A1)-(A3) over a box large enough that its edge
  carries no weight, the cost ratio of the two sample allocations equals
  Theorem 1's, and the fitted rates are the model's.
* The reuse allocation N' supplies exactly N samples to every index:
  sum_{L >= tau} N'_L = N_tau.
* Unbiasedness of the reuse estimator Y = sum_{tau <= L} dQ_tau / p_tau with
  the driver's own law (p_tau = P(L >= tau), pi = its mass function):
  sum_L pi_L Y(L) = sum_tau dQ_tau exactly, for an arbitrary dQ box.
"""
import os

import numpy as np
import pytest

from paper_1907_12334_gb300 import estimator as est
from paper_1907_12334_gb300.serving import MimcDriver

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_theorem1_closed_form_and_table1():
    for b, g in [((4.0, 4.0), (1.0, 1.0)), ((2.5, 1.7), (1.2, 0.9))]:
        x = [2 ** (-(g[j] + b[j]) / 2) for j in range(2)]
        assert est.theorem1_ratio(b, g) == pytest.approx((1 - x[0]) * (1 - x[1]), rel=1e-14)
    rows = [l.split() for l in open(os.path.join(GOLD, "table1_rates.txt")) if l.strip() and l[0] != "#"]
    got = {r[0]: est.theorem1_ratio((float(r[3]), float(r[4])), (float(r[5]), float(r[6]))) for r in rows}
    assert got["Q1"] == pytest.approx(0.753, abs=1e-3)
    assert got["Q2"] == pytest.approx(0.515, abs=1e-3)
    assert got["Q3"] == pytest.approx(0.387, abs=1e-3)
    assert est.theorem1_ratio((3.0,), (1.0,)) == pytest.approx(1 - 2 ** -2, rel=1e-14)  # d = 1


def _product(K, a, b, g):
    l1, l2 = np.meshgrid(np.arange(K + 1), np.arange(K + 1), indexing="ij")
    E = 0.3 * 2.0 ** (-a[0] * l1 - a[1] * l2)
    V = 0.7 * 2.0 ** (-b[0] * l1 - b[1] * l2)
    C = 5.0 * 2.0 ** (g[0] * l1 + g[1] * l2)
    return E, V, C


@pytest.mark.parametrize("a,b,g", [((2.0, 2.0), (4.0, 4.0), (1.0, 1.0)), ((1.5, 1.0), (3.0, 2.2), (1.1, 0.8))])
def test_cost_ratio_equals_theorem1_on_the_product_model(a, b, g):
    E, V, C = _product(60, a, b, g)
    no, yes, N, Nr = est.costs(V, C, tol=1e-3)
    assert yes / no == pytest.approx(est.theorem1_ratio(b, g), rel=1e-9)
    r = est.rates(E, V, C)
    assert r["alpha"] == pytest.approx(a, rel=1e-12)
    assert r["beta"] == pytest.approx(b, rel=1e-12)
    assert r["gamma"] == pytest.approx(g, rel=1e-12)


def test_reuse_allocation_supplies_every_index():
    rng = np.random.default_rng(1)
    N = np.cumsum(np.cumsum(rng.uniform(0, 3, (6, 5))[::-1, ::-1], 0), 1)[::-1, ::-1]  # decreasing in both
    Nr = est.reuse_samples(N)
    supplied = np.array([[Nr[i:, j:].sum() for j in range(N.shape[1])] for i in range(N.shape[0])])
    np.testing.assert_allclose(supplied, N, rtol=1e-12)


def test_optimal_samples_meet_the_tolerance():
    _, V, C = _product(8, (1, 1), (3.0, 2.0), (1.0, 1.0))
    N = est.optimal_samples(V, C, tol=2e-3)
    assert np.sum(V / N) == pytest.approx(4e-6, rel=1e-12)


def test_reuse_estimator_is_unbiased_under_the_driver_law():
    d = MimcDriver(eps=1e-2, lmax=(4, 3), seed=0)
    pi, tail = d.pmf(), d.tail
    assert pi.sum() == pytest.approx(tail[0, 0], rel=1e-14)
    rng = np.random.default_rng(7)
    dQ = rng.standard_normal(tail.shape)
    n1, n2 = tail.shape
    expect = 0.0
    for a in range(n1):
        for b in range(n2):
            Y = float((dQ[: a + 1, : b + 1] / tail[: a + 1, : b + 1]).sum())
            expect += pi[a, b] * Y
    # the mass function pads the tail with zeros beyond lmax, so inside the box its
    # own tail P(L >= tau) is exactly the p_tau that Y divides by
    box_tail = np.array([[pi[i:, j:].sum() for j in range(n2)] for i in range(n1)])
    np.testing.assert_allclose(box_tail, tail, rtol=1e-12)
    assert expect == pytest.approx(float(dQ.sum()), rel=1e-12)
