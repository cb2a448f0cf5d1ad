"""Seeded synthetic inputs shared by the CUDA path, the oracle, tests and bench.

This module holds none of the hot path's arithmetic.  It builds the *inputs*
of the path: the truncated Karhunen-Loeve basis (Phi, sqrt(lambda)) of the
Matern covariance that ``sample_field`` contracts with xi, and batch layouts
(grid shapes and multi-indices).  The random normals xi themselves are drawn
by each side's own counter-based generator (Philox4x64-10), never here.

Field law (Sec. 1, Eq. (1.2) of arXiv:1907.12334): a = exp(Z), Z a zero-mean
Gaussian field with Matern covariance
    C(r) = sigma^2 2^(1-nu)/Gamma(nu) (2 sqrt(nu) r)^nu K_nu(2 sqrt(nu) r),
r = ||T (x1 - x2)||.  The default law is nu = 3/2, sigma^2 = 1 with correlation
lengths 0.2 along x and 0.02 along y, read as r = sqrt((dx/0.2)^2 + (dy/0.02)^2)
(theta rotates the axes as the paper's T does).

The KL basis comes from a Nystrom discretisation of the covariance operator on
a uniform midpoint quadrature grid of the unit square: eigenpairs of (w C_q),
w = 1/n_q, eigenfunctions normalised in L2 and carried to the field points by
bilinear interpolation.  It is set-up work, untimed, and its accuracy as a
model of the Matern field is not part of any parity claim: both sides of every
parity test contract the very same (Phi, sqrt(lambda)) arrays.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class FieldLaw:
    nu: float = 1.5
    sigma2: float = 1.0
    ell_x: float = 0.2
    ell_y: float = 0.02
    theta: float = 0.0  # radians
    M: int = 400


def matern(r: np.ndarray, nu: float, sigma2: float = 1.0) -> np.ndarray:
    """Matern covariance of Eq. (1.2) as a function of the scaled distance r."""
    z = 2.0 * math.sqrt(nu) * np.asarray(r, dtype=np.float64)
    if nu == 0.5:
        return sigma2 * np.exp(-z)
    if nu == 1.5:
        return sigma2 * (1.0 + z) * np.exp(-z)
    if nu == 2.5:
        return sigma2 * (1.0 + z + z * z / 3.0) * np.exp(-z)
    from scipy.special import gamma, kv

    out = np.empty_like(z)
    small = z < 1e-12
    out[small] = 1.0
    zz = z[~small]
    out[~small] = 2.0 ** (1.0 - nu) / gamma(nu) * zz**nu * kv(nu, zz)
    return sigma2 * out


def scaled_distance(dx, dy, law: FieldLaw):
    c, s = math.cos(law.theta), math.sin(law.theta)
    rx = c * dx - s * dy
    ry = s * dx + c * dy
    return np.sqrt((rx / law.ell_x) ** 2 + (ry / law.ell_y) ** 2)


def _quad_grid(law: FieldLaw):
    # enough points per correlation length along each axis for M modes
    nqx = int(min(48, max(12, math.ceil(2.5 / law.ell_x) + 4)))
    nqy = int(min(192, max(12, math.ceil(2.5 / law.ell_y) + 4)))
    while nqx * nqy < 2 * law.M:
        nqx += 4
        nqy += 4
    return nqx, nqy


@functools.lru_cache(maxsize=8)
def _nystrom(law: FieldLaw):
    from scipy.linalg import eigh

    nqx, nqy = _quad_grid(law)
    xs = (np.arange(nqx) + 0.5) / nqx
    ys = (np.arange(nqy) + 0.5) / nqy
    X, Y = np.meshgrid(xs, ys)  # [nqy][nqx]
    px, py = X.ravel(), Y.ravel()
    n = px.size
    C = matern(scaled_distance(px[:, None] - px[None, :], py[:, None] - py[None, :], law), law.nu, law.sigma2)
    w = 1.0 / n
    M = min(law.M, n)
    vals, vecs = eigh(w * C, subset_by_index=[n - M, n - 1])
    order = np.argsort(vals)[::-1]
    lam = np.clip(vals[order], 0.0, None)
    phi_q = vecs[:, order] / math.sqrt(w)  # L2-normalised eigenfunctions at the nodes
    # fix the sign of each eigenfunction so the basis is deterministic
    sgn = np.sign(phi_q[np.argmax(np.abs(phi_q), axis=0), np.arange(M)])
    phi_q = phi_q * sgn[None, :]
    return nqx, nqy, lam, phi_q.reshape(nqy, nqx, M)


def field_grid_shape(P: int, Q: int):
    """(NFy, NFx): the field is given on the nodes of G^(P+1,Q+1)."""
    return (1 << (Q + 1)) + 1, (1 << (P + 1)) + 1


@functools.lru_cache(maxsize=16)
def kl_basis(P: int, Q: int, law: FieldLaw = FieldLaw()):
    """(Phi [npts][M] float64 row-major, sqrt_lambda [M]) on the field grid of (P,Q).

    Point index = Fy * NFx + Fx with Fx the x node index (x fastest)."""
    nqx, nqy, lam, phi_q = _nystrom(law)
    NFy, NFx = field_grid_shape(P, Q)
    fx = np.arange(NFx) / (NFx - 1)
    fy = np.arange(NFy) / (NFy - 1)

    def weights(f, nq):
        t = np.clip(f * nq - 0.5, 0.0, nq - 1.0)
        i0 = np.minimum(np.floor(t).astype(np.int64), nq - 2) if nq > 1 else np.zeros_like(t, dtype=np.int64)
        a = t - i0
        return i0, a

    ix, axw = weights(fx, nqx)
    iy, ayw = weights(fy, nqy)
    M = lam.size
    Phi = np.empty((NFy, NFx, M), dtype=np.float64)
    for r in range(NFy):
        row0 = phi_q[iy[r]]
        row1 = phi_q[iy[r] + 1]
        rowv = (1.0 - ayw[r]) * row0 + ayw[r] * row1  # [nqx][M]
        Phi[r] = (1.0 - axw)[:, None] * rowv[ix] + axw[:, None] * rowv[ix + 1]
    Phi = Phi.reshape(NFy * NFx, M)
    Phi.setflags(write=False)
    sl = np.sqrt(lam)
    sl.setflags(write=False)
    return Phi, sl


def kl_basis_nodes(nx: int, ny: int, law: FieldLaw = FieldLaw(), rows=None):
    """(Phi [len(rows) * nx][M] float64, sqrt_lambda [M]) at the nodes (i/(nx-1), j/(ny-1))
    of an nx x ny grid, x fastest; `rows` (default all) selects the j of the returned
    rows so that large grids can be built in pieces."""
    nqx, nqy, lam, phi_q = _nystrom(law)
    rows = np.arange(ny) if rows is None else np.asarray(rows)

    def weights(f, nq):
        t = np.clip(f * nq - 0.5, 0.0, nq - 1.0)
        i0 = np.minimum(np.floor(t).astype(np.int64), nq - 2) if nq > 1 else np.zeros_like(t, dtype=np.int64)
        return i0, t - i0

    ix, axw = weights(np.arange(nx) / (nx - 1), nqx)
    iy, ayw = weights(rows / (ny - 1), nqy)
    M = lam.size
    Phi = np.empty((rows.size, nx, M), dtype=np.float64)
    for k in range(rows.size):
        rowv = (1.0 - ayw[k]) * phi_q[iy[k]] + ayw[k] * phi_q[iy[k] + 1]  # [nqx][M]
        Phi[k] = (1.0 - axw)[:, None] * rowv[ix] + axw[:, None] * rowv[ix + 1]
    return Phi.reshape(rows.size * nx, M), np.sqrt(lam)


def small_law(M: int = 32) -> FieldLaw:
    """The default law truncated to M terms (cheap set-up for small test cases)."""
    return FieldLaw(M=M)


def smooth_field(P: int, Q: int, amp: float = 0.5) -> np.ndarray:
    """A smooth deterministic Z on the field grid (used by convergence pins)."""
    NFy, NFx = field_grid_shape(P, Q)
    x = np.arange(NFx) / (NFx - 1)
    y = np.arange(NFy) / (NFy - 1)
    X, Y = np.meshgrid(x, y)
    return (amp * np.sin(2 * np.pi * X) * np.cos(np.pi * Y) + 0.3 * amp * X * Y).ravel()


# ------------------------------------------------------------------ batches --

def pr1_indices():
    """Multi-indices (l1,l2) in 0..3 x 0..3 with base grid (3,3): finest 64x64 cells."""
    return [(l1, l2) for l1 in range(4) for l2 in range(4)]


def uneven_shapes(S: int, k: int = 2, amax: int = 7, seed: int = 0):
    """Grid exponents (P,Q) = (a1+k, a2+k), a in 0..amax, S/(amax+1)^2 per index, shuffled."""
    idx = [(a1 + k, a2 + k) for a1 in range(amax + 1) for a2 in range(amax + 1)]
    per = S // len(idx)
    shapes = [pq for pq in idx for _ in range(per)]
    rng = np.random.default_rng(seed)
    rng.shuffle(shapes)
    return shapes
