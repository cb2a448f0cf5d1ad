"""Cost of the multi-index estimator with and without sample reuse (Sec. 3).

From per-index means E_tau and variances V_tau of the differences dQ_tau
(Eq. (3.2)) and per-sample costs C_tau, on an index box 0 <= tau <= K:

* without reuse (standard MIMC): N_tau proportional to sqrt(V_tau / C_tau)
  samples on index tau, scaled so that sum_tau V_tau / N_tau = tol^2; cost
  sum_tau N_tau C_tau = (sum_tau sqrt(V_tau C_tau))^2 / tol^2;
* with reuse (MSG-MIMC): one FMSG solve at index L gives dQ_tau for every
  tau <= L, so only the samples not already supplied by higher indices are
  drawn on tau: N'_tau = N_tau - N_{tau+e1} - N_{tau+e2} + N_{tau+e1+e2}
  (inclusion-exclusion, N = 0 outside the box), cost sum_tau N'_tau C_tau;
* Theorem 1 (Eq. (3.9)): under the product model (A1)-(A3) the ratio of the
  two costs is 1 - sum over non-empty u of (-1)^(|u|+1) prod_{j in u} x_j,
  x_j = 2^(-(gamma_j + beta_j)/2); for d = 2 that is (1 - x1)(1 - x2);
* rates alpha_j, beta_j, gamma_j by least squares on log2 |E|, log2 V and
  log2 C along each axis (tau_j = 1..K_j, the other index 0; index 0 is left
  out, its "difference" being the coarsest value itself).
Host arithmetic only (numpy); the measurements come from the batched solver.
"""
from __future__ import annotations

import itertools

import numpy as np


def theorem1_ratio(beta, gamma) -> float:
    """Eq. (3.9) for any dimension d = len(beta)."""
    x = [2.0 ** (-(g + b) / 2.0) for b, g in zip(beta, gamma)]
    s = 0.0
    for k in range(1, len(x) + 1):
        for u in itertools.combinations(range(len(x)), k):
            s += (-1) ** (k + 1) * float(np.prod([x[j] for j in u]))
    return 1.0 - s


def optimal_samples(V, C, tol: float) -> np.ndarray:
    """N_tau = sqrt(V_tau / C_tau) sum(sqrt(V C)) / tol^2 (continuous, unrounded)."""
    V, C = np.asarray(V, float), np.asarray(C, float)
    return np.sqrt(V / C) * np.sum(np.sqrt(V * C)) / tol ** 2


def reuse_samples(N) -> np.ndarray:
    """N'_tau: samples to draw on tau when every sample at L >= tau also supplies tau (d = 2)."""
    N = np.asarray(N, float)
    Np = np.pad(N, ((0, 1), (0, 1)))
    return Np[:-1, :-1] - Np[1:, :-1] - Np[:-1, 1:] + Np[1:, 1:]


def costs(V, C, tol: float):
    """(cost without reuse, cost with reuse, N, N'); N' below zero (noisy V, C) count as zero."""
    N = optimal_samples(V, C, tol)
    Nr = reuse_samples(N)
    C = np.asarray(C, float)
    return float(np.sum(N * C)), float(np.sum(np.maximum(Nr, 0.0) * C)), N, Nr


def fit_rates(A) -> tuple[float, float]:
    """Rates of |A| along each axis: A[l, 0] ~ 2^(-r1 l), A[0, l] ~ 2^(-r2 l), l >= 1,
    least squares on log2 (a decay gives a positive rate)."""
    A = np.abs(np.asarray(A, float))
    out = []
    for axis in range(2):
        line = A[1:, 0] if axis == 0 else A[0, 1:]
        l = np.arange(1, line.size + 1)
        ok = line > 0
        if ok.sum() < 2:
            out.append(float("nan"))
            continue
        slope = np.polyfit(l[ok], np.log2(line[ok]), 1)[0]
        out.append(float(-slope))
    return out[0], out[1]


def rates(E, V, C) -> dict:
    """alpha_j, beta_j (decay of |E| and V) and gamma_j (growth of C) along each axis."""
    a1, a2 = fit_rates(E)
    b1, b2 = fit_rates(V)
    g1, g2 = fit_rates(C)
    return {"alpha": (a1, a2), "beta": (b1, b2), "gamma": (-g1, -g2)}
