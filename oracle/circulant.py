"""Circulant-embedding sampler of the paper's field law (oracle; test infrastructure).

Sec. 4 (numerical experiments) samples the lognormal coefficient a = exp(Z) with
Z a zero-mean Gaussian field of Matern covariance (Eq. (1.2) of Sec. 1) whose
distance is r = ||T (x1 - x2)||, T = S R with S = diag(1/sqrt(eta lambda),
1/sqrt(lambda)) and R the rotation by theta (Sec. 1).  The anisotropic ratio eta
and the rotation theta are hyper-parameters drawn per sample, so the
eigenvalues of the embedding are recomputed for every sample by an FFT.  The
field is sampled exactly on a periodic domain L times larger than [0,1]^2 in
each direction, L = 1 + 2 ceil(sqrt(nu) log2(max(2^p0, 2^q0))).

Readings (where the text leaves a choice):
* the field lives on the nodes of the finest grid of the solver's field,
  x_i = i hx, y_j = j hy, hx = 2^-(P+1), hy = 2^-(Q+1); the periodic domain
  [0, L)^2 is sampled with the same spacing: M1 = L 2^(P+1) by M2 = L 2^(Q+1)
  points;
* the generating array is c(k1, k2) = C(d1 hx, d2 hy) with d the signed
  periodic offset (k, or k - M above M/2).  At an offset of exactly M/2 the two
  signs are averaged, which keeps the embedding symmetric under a rotation;
* eigenvalues Lambda = DFT2(c) (real); a negative one, possible only when L is
  too small, is set to zero and reported;
* a sample is the real part of DFT2(sqrt(Lambda / (M1 M2)) (xi1 + i xi2)),
  forward transform (exp(-2 pi i jk/M)), restricted to the field's nodes;
  xi1, xi2 at embedding point k = k2 M1 + k1 are normals 2k and 2k+1 of the
  sample's Philox4x64-10 + Box-Muller stream;
* the scaling S: the text prints S = diag(1/sqrt(eta lambda), 1/sqrt(lambda))
  (scale 0, the default), under which lambda acts as a squared length; with
  lambda read as a length, S = diag(1/(eta lambda), 1/lambda) (scale 1), the
  standard-coarsening multigrid of Sec. 2 fails at eta = 1/16 as the paper
  reports, while under the printed form it converges;
* eta and theta of global sample s come from one Philox4x64-10 block with
  counter (0, s, 1, 0) and key (seed, 0): u = (w >> 11) 2^-53 of words 0 and
  1, eta = eta_lo + (eta_hi - eta_lo) u0, theta = theta_lo + (theta_hi -
  theta_lo) u1 (degrees).
The FFTs are numpy's (FP64), used as a library primitive.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import normals, philox4x64_10


@dataclass
class CeLaw:
    nu: float = 0.5          # Matern smoothness (closed forms for 1/2, 3/2, 5/2)
    lam: float = 0.25        # length scale lambda
    eta_lo: float = 1.0 / 16
    eta_hi: float = 0.25
    theta_lo: float = -30.0  # degrees
    theta_hi: float = 30.0
    L: int = 7               # periodic domain side in domain lengths
    scale: int = 0           # 0: S = diag(1/sqrt(eta lam), 1/sqrt(lam)) as printed; 1: lambda as a length


def padding(nu: float, p0: int, q0: int) -> int:
    """L = 1 + 2 ceil(sqrt(nu) log2(max(2^p0, 2^q0))) (Sec. 4)."""
    return 1 + 2 * math.ceil(math.sqrt(nu) * max(p0, q0))


def matern(r, nu: float):
    """Eq. (1.2) for half-integer nu, written out: x = 2 sqrt(nu) r and
    nu = 1/2: exp(-x); 3/2: (1 + x) exp(-x); 5/2: (1 + x + x^2/3) exp(-x)."""
    r = np.asarray(r, dtype=np.float64)
    x = 2.0 * math.sqrt(nu) * r
    if nu == 0.5:
        return np.exp(-x)
    if nu == 1.5:
        return (1.0 + x) * np.exp(-x)
    if nu == 2.5:
        return (1.0 + x + x * x / 3.0) * np.exp(-x)
    raise ValueError("nu must be 1/2, 3/2 or 5/2")


def distance(dx, dy, lam: float, eta: float, theta: float, scale: int = 0):
    """r = ||S R (dx, dy)||, theta in radians (Sec. 1).  scale 0: S = diag(1/sqrt(eta
    lambda), 1/sqrt(lambda)) as printed; 1: S = diag(1/(eta lambda), 1/lambda)."""
    ct, st = math.cos(theta), math.sin(theta)
    rx = ct * dx - st * dy
    ry = st * dx + ct * dy
    if scale:
        return np.sqrt((rx / (eta * lam)) ** 2 + (ry / lam) ** 2)
    return np.sqrt(rx * rx / (eta * lam) + ry * ry / lam)


def hyper(seed: int, s: int, law: CeLaw):
    """(eta, theta in radians) of global sample s."""
    w = philox4x64_10((0, s, 1, 0), (seed, 0))
    u0 = float(int(w[0]) >> 11) * 2.0 ** -53
    u1 = float(int(w[1]) >> 11) * 2.0 ** -53
    eta = law.eta_lo + (law.eta_hi - law.eta_lo) * u0
    theta = law.theta_lo + (law.theta_hi - law.theta_lo) * u1
    return eta, math.radians(theta)


def embed_size(P: int, Q: int, L: int):
    return L << (P + 1), L << (Q + 1)


def _offsets(M: int):
    """Signed periodic offsets of k = 0..M-1 as (first, second) candidates; they
    differ only at k = M/2, where both signs are averaged."""
    k = np.arange(M)
    d = np.where(k <= M // 2, k, k - M)
    d2 = np.where(k == M // 2, -k, d)
    return d, d2


def generating_array(P: int, Q: int, law: CeLaw, eta: float, theta: float) -> np.ndarray:
    """c[k2, k1] (rows: y offset, columns: x offset) of the block-circulant embedding."""
    M1, M2 = embed_size(P, Q, law.L)
    hx, hy = 2.0 ** -(P + 1), 2.0 ** -(Q + 1)
    a1, b1 = _offsets(M1)
    a2, b2 = _offsets(M2)
    c = np.zeros((M2, M1))
    for ox in (a1, b1):
        for oy in (a2, b2):
            c += matern(distance(ox[None, :] * hx, oy[:, None] * hy, law.lam, eta, theta, law.scale), law.nu)
    return c / 4.0


def eigenvalues(c: np.ndarray) -> np.ndarray:
    return np.fft.fft2(c).real


def sample_from_normals(P: int, Q: int, lam_eig: np.ndarray, xi1: np.ndarray, xi2: np.ndarray) -> np.ndarray:
    """Field on the (2^(Q+1)+1) x (2^(P+1)+1) nodes, row-major (x fastest)."""
    M2, M1 = lam_eig.shape
    a = np.sqrt(np.maximum(lam_eig, 0.0) / (M1 * M2))
    y = np.fft.fft2(a * (xi1.reshape(M2, M1) + 1j * xi2.reshape(M2, M1)))
    return np.ascontiguousarray(y.real[: (1 << (Q + 1)) + 1, : (1 << (P + 1)) + 1]).ravel()


def ce_field(P: int, Q: int, law: CeLaw, seed: int, s: int):
    """(Z, eta, theta, min eigenvalue / largest) of global sample s."""
    eta, theta = hyper(seed, s, law)
    lam_eig = eigenvalues(generating_array(P, Q, law, eta, theta))
    M1, M2 = embed_size(P, Q, law.L)
    xi = normals(seed, s, 2 * M1 * M2)
    Z = sample_from_normals(P, Q, lam_eig, xi[0::2], xi[1::2])
    return Z, eta, theta, float(lam_eig.min() / lam_eig.max())


def covariance_matrix(P: int, Q: int, law: CeLaw, eta: float, theta: float) -> np.ndarray:
    """Eq. (1.2) between every pair of field nodes, evaluated directly."""
    nx, ny = (1 << (P + 1)) + 1, (1 << (Q + 1)) + 1
    X, Y = np.meshgrid(np.arange(nx) * 2.0 ** -(P + 1), np.arange(ny) * 2.0 ** -(Q + 1))
    X, Y = X.ravel(), Y.ravel()
    return matern(distance(X[:, None] - X[None, :], Y[:, None] - Y[None, :], law.lam, eta, theta, law.scale),
                  law.nu)
