"""Pins of the circulant-embedding oracle (oracle/circulant.py) against what the
paper and the mathematics fix, independently of the oracle's own code path.

* Exactness (Sec. 4: "exact samples ... using circulant embedding"): the map
  from (xi1, xi2) to the field is linear, Z = Re(A (xi1 + i xi2)), so the
  field's covariance is Re(A) Re(A)^T + Im(A) Im(A)^T.  Built column by column
  from the oracle's own sampling call, it must equal the Matern covariance of
  Eq. (1.2) evaluated directly between every pair of field nodes, whenever the
  embedding's eigenvalues are non-negative.
* Eq. (1.2) closed forms for nu = 1/2, 3/2, 5/2 against the general formula
  with the modified Bessel function K_nu (scipy).
* The distance of Sec. 1 at special angles (theta = 0, 90 degrees).
* The padding formula of Sec. 4.
Planted mistakes (an unsigned periodic offset, a missing 1/M, swapped grid
spacings, a rotation of the wrong sign) must fail these pins.
"""
import math

import numpy as np
import pytest

from oracle import circulant as ce


def _field_covariance(P, Q, law, eta, theta):
    M1, M2 = ce.embed_size(P, Q, law.L)
    lam = ce.eigenvalues(ce.generating_array(P, Q, law, eta, theta))
    n = M1 * M2
    cols = []
    z = np.zeros(n)
    for k in range(n):
        e = z.copy()
        e[k] = 1.0
        cols.append(ce.sample_from_normals(P, Q, lam, e, z))
        cols.append(ce.sample_from_normals(P, Q, lam, z, e))
    A = np.stack(cols, axis=1)
    return A @ A.T, lam


@pytest.mark.parametrize("P,Q,nu,eta,theta_deg,scale", [(1, 1, 0.5, 0.125, 20.0, 0), (1, 2, 0.5, 1 / 16, -30.0, 0),
                                                        (2, 1, 1.5, 0.25, 25.0, 0), (1, 1, 2.5, 0.2, 0.0, 0),
                                                        (1, 2, 0.5, 1 / 16, 10.0, 1), (2, 1, 1.5, 0.1, -20.0, 1)])
def test_embedding_reproduces_the_matern_covariance_exactly(P, Q, nu, eta, theta_deg, scale):
    law = ce.CeLaw(nu=nu, L=7, scale=scale)
    th = math.radians(theta_deg)
    cov, lam = _field_covariance(P, Q, law, eta, th)
    assert lam.min() >= -1e-12 * lam.max()
    ref = ce.covariance_matrix(P, Q, law, eta, th)
    np.testing.assert_allclose(cov, ref, rtol=0, atol=1e-12)


def test_matern_closed_forms_match_the_bessel_formula():
    sp = pytest.importorskip("scipy.special")
    r = np.array([1e-3, 0.05, 0.3, 1.0, 2.7])
    for nu in (0.5, 1.5, 2.5):
        x = 2 * math.sqrt(nu) * r
        general = 2 ** (1 - nu) / math.gamma(nu) * x ** nu * sp.kv(nu, x)
        np.testing.assert_allclose(ce.matern(r, nu), general, rtol=1e-13)
    assert ce.matern(0.0, 0.5) == 1.0


def test_distance_at_special_angles():
    lam, eta, dx = 0.25, 0.1, 0.3
    assert ce.distance(dx, 0.0, lam, eta, 0.0) == pytest.approx(dx / math.sqrt(eta * lam), rel=1e-15)
    assert ce.distance(0.0, dx, lam, eta, 0.0) == pytest.approx(dx / math.sqrt(lam), rel=1e-15)
    # a quarter turn sends the x offset onto the second axis
    assert ce.distance(dx, 0.0, lam, eta, math.pi / 2) == pytest.approx(dx / math.sqrt(lam), rel=1e-14)
    # +30 degrees moves (cos 30, sin 30) onto the first axis only for theta = -30 degrees
    v = (math.cos(math.radians(30)), math.sin(math.radians(30)))
    assert ce.distance(*v, lam, eta, math.radians(-30)) == pytest.approx(1 / math.sqrt(eta * lam), rel=1e-14)


def test_distance_length_scale_reading():
    """scale 1 reads lambda as a length: r = |rotated offset| / (eta lambda) along x'."""
    lam, eta, dx = 0.25, 0.1, 0.3
    assert ce.distance(dx, 0.0, lam, eta, 0.0, 1) == pytest.approx(dx / (eta * lam), rel=1e-15)
    assert ce.distance(0.0, dx, lam, eta, math.pi / 2, 1) == pytest.approx(dx / (eta * lam), rel=1e-14)


def test_padding_formula():
    assert ce.padding(0.5, 4, 4) == 7          # 1 + 2 ceil(sqrt(1/2) 4) = 1 + 2*3
    assert ce.padding(1.5, 3, 5) == 15         # 1 + 2 ceil(1.2247 * 5)
    assert ce.padding(0.5, 0, 0) == 1


def test_hyperparameters_lie_in_the_paper_ranges():
    law = ce.CeLaw()
    eta, th = zip(*[ce.hyper(3, s, law) for s in range(200)])
    assert 1 / 16 <= min(eta) and max(eta) <= 1 / 4
    assert math.radians(-30) <= min(th) and max(th) <= math.radians(30)
    assert np.std(eta) > 0.03 and np.std(th) > 0.2  # spread over the ranges, not constant


@pytest.mark.parametrize("mistake", ["unsigned_offset", "no_normalisation", "swapped_spacing", "rotation_sign"])
def test_planted_mistakes_fail_the_pins(monkeypatch, mistake):
    P, Q, eta, th = 1, 2, 0.1, math.radians(25.0)
    law = ce.CeLaw(nu=0.5, L=7)
    if mistake == "unsigned_offset":
        monkeypatch.setattr(ce, "_offsets", lambda M: (np.arange(M), np.arange(M)))
    elif mistake == "no_normalisation":
        orig = ce.sample_from_normals
        monkeypatch.setattr(ce, "sample_from_normals",
                            lambda P_, Q_, lam, a, b: orig(P_, Q_, lam * lam.size, a, b))
    elif mistake == "swapped_spacing":
        orig_g = ce.generating_array
        monkeypatch.setattr(ce, "generating_array", lambda P_, Q_, law_, e, t: orig_g(Q_, P_, law_, e, t).T)
    if mistake == "rotation_sign":
        orig_d = ce.distance
        monkeypatch.setattr(ce, "distance", lambda dx, dy, lam, e, t: orig_d(dx, dy, lam, e, -t))
        # the direct matrix (unplanted) against the planted embedding, and the special-angle pin
        v = (math.cos(math.radians(30)), math.sin(math.radians(30)))
        assert ce.distance(*v, 0.25, 0.1, math.radians(-30)) != pytest.approx(1 / math.sqrt(0.1 * 0.25), rel=1e-6)
        return
    if mistake == "swapped_spacing":
        with pytest.raises((AssertionError, ValueError)):
            cov, _ = _field_covariance(P, Q, law, eta, th)
            np.testing.assert_allclose(cov, ce.covariance_matrix(P, Q, law, eta, th), rtol=0, atol=1e-12)
        return
    cov, _ = _field_covariance(P, Q, law, eta, th)
    assert np.max(np.abs(cov - ce.covariance_matrix(P, Q, law, eta, th))) > 1e-6
