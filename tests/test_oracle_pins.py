"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a closed form, an independent
library implementation, an invariant of the method, or a value printed in
arXiv:1907.12334.  Chosen so that a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at
least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1907_12334_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------- generator --

@pytest.mark.parametrize("ctr,key", [((0, 0, 0, 0), (0, 0)), ((5, 7, 0, 0), (123, 0)), ((0, 3, 0, 0), (2**63 + 11, 0)),
                                     ((2**40, 2**33, 9, 2**62), (1, 2**64 - 1))])
def test_philox_matches_numpy(ctr, key):
    """numpy.random.Philox is an independent Philox4x64-10; it pre-increments its counter."""
    c = np.array(ctr, dtype=np.uint64)
    prev = c.copy()
    # counter - 1 with borrow, so numpy's first block is exactly `ctr`
    for w in range(4):
        if prev[w] > 0:
            prev[w] -= np.uint64(1)
            break
        prev[w] = np.uint64(2**64 - 1)
    bg = np.random.Philox(counter=prev, key=np.array(key, dtype=np.uint64))
    assert [int(x) for x in bg.random_raw(4)] == [int(x) for x in oracle.philox4x64_10(ctr, key)]


def test_normals_distribution():
    """Box-Muller output is N(0,1): moments and a Kolmogorov-Smirnov test."""
    from scipy import stats

    z = np.concatenate([oracle.normals(0, s, 400) for s in range(500)])
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # consecutive pairs share a radius: z_a^2 + z_b^2 = -2 ln(1 - U_a)
    w = oracle.philox4x64_10((0, 3, 0, 0), (0, 0))
    ua = float(int(w[0]) >> 11) * 2.0**-53
    xi = oracle.normals(0, 3, 4)
    assert xi[0] ** 2 + xi[1] ** 2 == pytest.approx(-2 * math.log(1 - ua), rel=1e-14)


def test_normals_ragged_tail_and_independence():
    """Terms of a block do not depend on M; different samples differ."""
    a = oracle.normals(7, 11, 10)
    b = oracle.normals(7, 11, 13)
    assert np.array_equal(a, b[:10])
    assert not np.allclose(oracle.normals(7, 12, 10), a)


def test_kl_field_is_the_matrix_product():
    """Z = Phi diag(sqrt(lambda)) xi; numpy's matmul is an independent evaluation."""
    rng = np.random.default_rng(1)
    Phi = rng.standard_normal((37, 9))
    sl = rng.random(9)
    xi = rng.standard_normal(9)
    np.testing.assert_allclose(oracle.kl_field(Phi, sl, xi), Phi @ (sl * xi), rtol=1e-13, atol=1e-14)


# --------------------------------------------------------- discretisation --

def test_coefficient_injection_faces():
    """Injection reading: a = exp(Z) at face midpoints x-face (i+1/2, j), y-face (i, j+1/2), every grid."""
    P, Q = 4, 3
    NFy, NFx = inputs.field_grid_shape(P, Q)
    X, Y = np.meshgrid(np.arange(NFx) / (NFx - 1), np.arange(NFy) / (NFy - 1))
    f = lambda x, y: 0.3 * x - 0.7 * y + 0.1 + 0.2 * x * y
    H = oracle.Hierarchy(P, Q, f(X, Y).ravel(), oracle.SolverParams(coef=oracle.COEF_INJECTION))
    for p in range(1, P + 1):
        for q in range(1, Q + 1):
            nx, ny = 1 << p, 1 << q
            ax, ay = H.coef(p, q)
            i, j = np.meshgrid(np.arange(nx), np.arange(ny + 1))
            np.testing.assert_allclose(ax, np.exp(f((i + 0.5) / nx, j / ny)), rtol=1e-14)
            i, j = np.meshgrid(np.arange(nx + 1), np.arange(ny))
            np.testing.assert_allclose(ay, np.exp(f(i / nx, (j + 0.5) / ny)), rtol=1e-14)


def test_coefficient_series_mean_faces():
    """Default reading: a coarse face carries the series mean of the finest-face values
    it covers along the flux direction.  For Z = c x + g(y) the x-face values are the
    geometric sequence exp(c x_k) (g(y) factored out) with the closed-form harmonic
    mean; a transverse-only variation (Z = h(y)) is passed through unchanged on x-faces."""
    P, Q = 4, 3
    NFy, NFx = inputs.field_grid_shape(P, Q)
    X, Y = np.meshgrid(np.arange(NFx) / (NFx - 1), np.arange(NFy) / (NFy - 1))
    c = 1.3
    g = lambda y: 0.4 * np.cos(3 * y)
    H = oracle.Hierarchy(P, Q, (c * X + g(Y)).ravel())
    for p in range(1, P + 1):
        for q in range(1, Q + 1):
            nx, ny = 1 << p, 1 << q
            sx = 1 << (P - p)
            h = 1.0 / (1 << P)  # finest x-face spacing
            ax, _ = H.coef(p, q)
            for i in (0, nx - 1):
                for j in (0, ny // 2, ny):
                    x0 = i * sx * h + h / 2  # first finest face midpoint in the segment
                    # sx / sum_k exp(-(c (x0 + k h) + g)) = sx e^{c x0 + g} (1 - e^{-c h}) / (1 - e^{-c h sx})
                    expect = sx * np.exp(c * x0 + g(j / ny)) * (1 - np.exp(-c * h)) / (1 - np.exp(-c * h * sx))
                    assert ax[j, i] == pytest.approx(expect, rel=1e-13)
    H2 = oracle.Hierarchy(P, Q, g(Y).ravel())
    for p in range(1, P + 1):
        ax, _ = H2.coef(p, 2)
        np.testing.assert_allclose(ax, np.exp(g(np.arange(5) / 4))[:, None] * np.ones((1, 1 << p)), rtol=1e-14)


def _dense(H, p, q):
    sh = H.shape(p, q)
    n = (sh[0] - 2) * (sh[1] - 2)
    A = np.zeros((n, n))
    for k in range(n):
        v = np.zeros(sh)
        v[1:-1, 1:-1].flat[k] = 1.0
        A[:, k] = H.apply(p, q, v)[1:-1, 1:-1].ravel()
    return A


def test_operator_symmetric_positive_definite():
    """The conservative 5-point operator is symmetric positive definite; a face
    coefficient taken from the wrong side breaks the symmetry."""
    P, Q = 3, 3
    Phi, sl = inputs.kl_basis(P, Q, inputs.small_law(24))
    Z = oracle.kl_field(Phi, sl, oracle.normals(0, 0, 24))
    H = oracle.Hierarchy(P, Q, Z)
    for p, q in [(3, 3), (3, 1), (1, 3), (2, 3)]:
        A = _dense(H, p, q)
        np.testing.assert_allclose(A, A.T, rtol=1e-13, atol=1e-12 * np.abs(A).max())
        assert np.linalg.eigvalsh(A).min() > 0


def _dst_solution(p, q):
    """Discrete solution of A u = 1 for a = 1 by the sine eigenbasis (textbook)."""
    from scipy.fft import dstn, idstn

    nx, ny = 1 << p, 1 << q
    k = np.arange(1, nx)
    l = np.arange(1, ny)
    lam = 4 * nx**2 * np.sin(k * np.pi / (2 * nx))[None, :] ** 2 + 4 * ny**2 * np.sin(l * np.pi / (2 * ny))[:, None] ** 2
    b = np.ones((ny - 1, nx - 1))
    return idstn(dstn(b, type=1) / lam, type=1)


def test_constant_coefficient_fmsg_matches_sine_solution():
    """a = 1: every grid's FMSG solution equals the sine-series discrete solution."""
    P, Q = 5, 4
    H = oracle.Hierarchy(P, Q, np.zeros(oracle.field_points(P, Q)), oracle.SolverParams(eps=1e-13, max_cycles=100))
    st, cyc, rr = H.fmsg()
    assert st == 0
    for p in range(1, P + 1):
        for q in range(1, Q + 1):
            u = H.get(p, q, oracle.SOL)[1:-1, 1:-1]
            np.testing.assert_allclose(u, _dst_solution(p, q), rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("p,q,integral,center", [(1, 1, 0.015625, 1 / 16), (2, 2, 0.0288086, 0.0703125),
                                                 (3, 3, 0.0334230, None), (3, 6, 0.0342545, None),
                                                 (6, 6, 0.0351164, 0.0736572)])
def test_constant_coefficient_printed_values(p, q, integral, center):
    """Integral and midpoint values of the a = 1 discrete solutions: the discrete
    sine-series (DST) closed form summed to 7 digits, and 1/64 and 1/16 on G^(1,1)
    by hand (one unknown, A = 8 + 8 = 16, u = 1/16, integral = u / 4)."""
    Qg, st, _, _ = oracle.solve_sample(p, q, np.zeros(oracle.field_points(p, q)),
                                       oracle.SolverParams(eps=1e-12, max_cycles=100))
    assert Qg[p - 1, q - 1] == pytest.approx(integral, abs=6e-8)
    if center is not None:
        Qc, _, _, _ = oracle.solve_sample(p, q, np.zeros(oracle.field_points(p, q)),
                                          oracle.SolverParams(eps=1e-12, max_cycles=100, qoi=oracle.QOI_POINT))
        assert Qc[p - 1, q - 1] == pytest.approx(center, abs=6e-8)


def test_constant_coefficient_second_order_to_continuum():
    """Integral of u and u(1/2,1/2) converge at O(h^2) to the continuum values
    0.0351443 and 0.0736714 (double sine series of -Laplace u = 1)."""
    errs_i, errs_c = [], []
    for n in (3, 4, 5, 6):
        z = np.zeros(oracle.field_points(n, n))
        Qi, _, _, _ = oracle.solve_sample(n, n, z, oracle.SolverParams(eps=1e-12))
        Qc, _, _, _ = oracle.solve_sample(n, n, z, oracle.SolverParams(eps=1e-12, qoi=oracle.QOI_POINT))
        errs_i.append(abs(Qi[-1, -1] - 0.0351443))
        errs_c.append(abs(Qc[-1, -1] - 0.0736714))
    for e in (errs_i, errs_c):
        ratios = [e[k] / e[k + 1] for k in range(len(e) - 1)]
        assert all(3.3 < r < 4.7 for r in ratios[:2]), ratios


def test_manufactured_solution_second_order():
    """Variable a = exp(Z) with smooth Z, u* = sin(pi x) sin(pi y), f = -div(a grad u*)
    by symbolic differentiation: the discrete solution converges at O(h^2)."""
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    Zs = 0.5 * sp.sin(2 * sp.pi * x) * sp.cos(sp.pi * y) + 0.15 * x * y
    us = sp.sin(sp.pi * x) * sp.sin(sp.pi * y)
    a = sp.exp(Zs)
    f = -(sp.diff(a * sp.diff(us, x), x) + sp.diff(a * sp.diff(us, y), y))
    fl = sp.lambdify((x, y), f, "numpy")
    ul = sp.lambdify((x, y), us, "numpy")
    errs = []
    for n in (3, 4, 5, 6):
        Z = inputs.smooth_field(n, n, amp=0.5)
        H = oracle.Hierarchy(n, n, Z, oracle.SolverParams(eps=1e-12, max_cycles=200))
        N = 1 << n
        X, Y = np.meshgrid(np.arange(N + 1) / N, np.arange(N + 1) / N)
        H.set_rhs(fl(X, Y))
        st, _, _ = H.fmsg()
        assert st == 0
        errs.append(np.abs(H.get(n, n, oracle.SOL) - ul(X, Y)).max())
    ratios = [errs[k] / errs[k + 1] for k in range(3)]
    assert all(3.5 < r < 4.5 for r in ratios[1:]), ratios


# ------------------------------------------------------- transfer operators --

def test_rhs_restriction_of_one_is_one():
    """Full weighting of h = 1 averaged over two parents gives exactly 1 (Alg. 2 restriction)."""
    P, Q = 4, 3
    H = oracle.Hierarchy(P, Q)
    for s in range(P + Q - 3, -1, -1):
        for p in range(1, P + 1):
            q = s + 2 - p
            if 1 <= q <= Q:
                b = H.restrict(p, q, src=1)
                assert np.all(b[1:-1, 1:-1] == 1.0)


def test_restriction_combination_closed_form():
    """Eq. (2.3): one parent on the q = Q / p = P edges, the average of both
    otherwise; full weighting maps x^2 to x^2 + dx_fine^2 / 2."""
    P, Q = 3, 3
    H = oracle.Hierarchy(P, Q)

    def grid_xy(p, q):
        nx, ny = 1 << p, 1 << q
        return np.meshgrid(np.arange(nx + 1) / nx, np.arange(ny + 1) / ny)

    def set_b(p, q, fn):
        X, Y = grid_xy(p, q)
        v = fn(X, Y)
        v[0, :] = v[-1, :] = v[:, 0] = v[:, -1] = 0
        H.set(p, q, oracle.B, v)

    fx = lambda X, Y: X**2 + 3 * Y
    fy = lambda X, Y: Y**2 - X
    for p in range(1, P + 1):
        for q in range(1, Q + 1):
            set_b(p, q, fx if (p + q) % 2 else fy)
    # (2,3): q = Q, only the x-parent (3,3), which holds fy (linear in x: R_x is exact)
    X, Y = grid_xy(2, 3)
    b = H.restrict(2, 3, src=1)
    np.testing.assert_allclose(b[1:-1, 1:-1], fy(X, Y)[1:-1, 1:-1], rtol=1e-14, atol=1e-14)
    # (3,2): p = P, only the y-parent (3,3) (fy): R_y y^2 = y^2 + dy_f^2 / 2
    X, Y = grid_xy(3, 2)
    b = H.restrict(3, 2, src=1)
    np.testing.assert_allclose(b[1:-1, 1:-1], (Y**2 + (1 / 8) ** 2 / 2 - X)[1:-1, 1:-1], rtol=1e-13, atol=1e-14)
    # (2,2): both parents (3,2) and (2,3), reset to fx, via R_x and R_y
    set_b(3, 2, fx)
    set_b(2, 3, fx)
    X, Y = grid_xy(2, 2)
    b = H.restrict(2, 2, src=1)
    rx = X**2 + (1 / 8) ** 2 / 2 + 3 * Y  # R_x of fx from (3,2): dx_f = 1/8
    ry = X**2 + 3 * Y  # R_y of fx from (2,3): linear in y -> exact
    np.testing.assert_allclose(b[1:-1, 1:-1], (0.5 * rx + 0.5 * ry)[1:-1, 1:-1], rtol=1e-13, atol=1e-14)


def test_linear_prolongation_reproduces_piecewise_linear_and_weights():
    """Eq. (2.4) with linear P: a coarse hat in x (kink on a coarse node) is
    reproduced; with equal children the weights sum to one (u += omega g); with
    a = 1 and dx = dy, kappa_x = kappa_y = 1/2 (Mulder's weights, Sec. 2)."""
    P, Q = 3, 3
    omega = 0.8
    H = oracle.Hierarchy(P, Q, prm=oracle.SolverParams(omega=omega))
    p, q = 3, 3
    g = lambda X, Y: np.minimum(X, 1 - X) * (1 + Y) * Y * (1 - Y)
    for (cp, cq) in [(2, 3), (3, 2)]:
        nx, ny = 1 << cp, 1 << cq
        X, Y = np.meshgrid(np.arange(nx + 1) / nx, np.arange(ny + 1) / ny)
        H.set(cp, cq, oracle.U, g(X, Y) if cp == 2 else np.zeros_like(X))
    H.set(p, q, oracle.U, np.zeros(H.shape(p, q)))
    u = H.interpolate(p, q, 0)
    nx = 1 << p
    X, Y = np.meshgrid(np.arange(nx + 1) / nx, np.arange(nx + 1) / nx)
    np.testing.assert_allclose(u, omega * 0.5 * g(X, Y), rtol=1e-13, atol=1e-15)


def test_kappa_closed_forms():
    """Eq. (2.5) with a = const: kappa_x = 1 / (1 + (dx/dy)^4); with random a the
    weights lie in [0,1] and sum to 1."""
    P, Q = 4, 4
    H = oracle.Hierarchy(P, Q)
    for p, q in [(4, 4), (4, 2), (1, 4), (3, 1)]:
        kx, ky = H.kappa(p, q)
        expect = 1.0 / (1.0 + (2.0 ** (q - p)) ** 4)
        np.testing.assert_allclose(kx[1:-1, 1:-1], expect, rtol=1e-14)
        np.testing.assert_allclose(ky[1:-1, 1:-1], 1 - expect, rtol=1e-12)
    Phi, sl = inputs.kl_basis(P, Q, inputs.small_law(16))
    H = oracle.Hierarchy(P, Q, oracle.kl_field(Phi, sl, oracle.normals(1, 0, 16)))
    kx, ky = H.kappa(3, 4)
    assert np.all((kx[1:-1, 1:-1] >= 0) & (kx[1:-1, 1:-1] <= 1))
    np.testing.assert_allclose((kx + ky)[1:-1, 1:-1], 1.0, rtol=1e-14)
    assert kx[1:-1, 1:-1].std() > 1e-3  # matrix dependent


def test_cubic_interpolation_exactness():
    """FMSG cubic interpolation: fine odd nodes with four coarse neighbours are exact
    for cubics; the boundary stencil 1/16[10 16 9 0 -1] is exact for cubics odd
    about the boundary (a x + b x^3)."""
    P, Q = 4, 1  # grid (4,1) has only the x-child (3,1)
    H = oracle.Hierarchy(P, Q)
    nxc = 1 << 3
    xc = np.arange(nxc + 1) / nxc
    xf = np.arange(2 * nxc + 1) / (2 * nxc)
    f_gen = lambda x: 1 - 2 * x + 3 * x**2 - 5 * x**3
    f_odd = lambda x: 0.7 * x - 2.0 * x**3
    # fine 4..12 only use interior coarse nodes 1..7; fine 1 uses the boundary stencil
    for f, check in [(f_gen, slice(4, 2 * nxc - 3)), (f_odd, slice(1, 2))]:
        c = np.zeros((3, nxc + 1))
        c[1, 1:-1] = f(xc[1:-1])
        H.set(3, 1, oracle.SOL, c)
        u = H.interpolate(4, 1, 1)
        np.testing.assert_allclose(u[1, check], f(xf[check]), rtol=1e-13, atol=1e-15)


# ----------------------------------------------------------- solver pins --

def test_fmsg_solutions_match_dense_solves():
    """Random lognormal field: the saved FMSG solution of every grid equals the
    dense LU solution of that grid's system (to the residual tolerance)."""
    P, Q = 3, 4
    M = 24
    Phi, sl = inputs.kl_basis(P, Q, inputs.small_law(M))
    Z = oracle.kl_field(Phi, sl, oracle.normals(3, 5, M))
    H = oracle.Hierarchy(P, Q, Z, oracle.SolverParams(eps=1e-13, max_cycles=500))
    st, cyc, rr = H.fmsg()
    assert st == 0 and np.all(rr <= 1e-13)
    for p in range(1, P + 1):
        for q in range(1, Q + 1):
            A = _dense(H, p, q)
            u = np.linalg.solve(A, np.ones(A.shape[0]))
            np.testing.assert_allclose(H.get(p, q, oracle.SOL)[1:-1, 1:-1].ravel(), u, rtol=1e-9)


def test_w_cycle_contraction_constant_coefficient():
    """MSG W(2,2) on the top grid of a = 1 contracts the residual by far more than
    a smoother alone (textbook multigrid rate; a wrong transfer operator fails)."""
    P = Q = 5
    H = oracle.Hierarchy(P, Q, np.zeros(oracle.field_points(P, Q)))
    r0 = np.linalg.norm(H.residual(P, Q))
    H.mu_cycle(P + Q - 2)
    r1 = np.linalg.norm(H.residual(P, Q))
    H.mu_cycle(P + Q - 2)
    r2 = np.linalg.norm(H.residual(P, Q))
    assert r1 / r0 < 0.05 and r2 / r1 < 0.05


def test_solve_sample_status_and_cycles():
    P, Q = 3, 3
    Z = np.zeros(oracle.field_points(P, Q))
    Qg, st, cyc, rr = oracle.solve_sample(P, Q, Z, oracle.SolverParams(eps=1e-12, max_cycles=50))
    assert st == 0 and np.all(cyc >= 1) and np.all(rr <= 1e-12)
    assert cyc[0, 0] == 1  # the one-unknown grid is solved exactly
    _, st2, cyc2, _ = oracle.solve_sample(P, Q, Z, oracle.SolverParams(eps=0.0, max_cycles=3))
    assert st2 & 1 and cyc2.max() == 3
    Zbad = Z.copy()
    NFx = (1 << (P + 1)) + 1
    Zbad[8 * NFx + 7] = np.nan  # field node (7, 8): x-face (3+1/2, 4) of the finest grid
    _, st3, _, _ = oracle.solve_sample(P, Q, Zbad, oracle.SolverParams(eps=1e-12, max_cycles=5))
    assert st3 & 2


# ------------------------------------------------------------------ QoIs --

def test_qoi_closed_forms():
    """Q on analytic nodal fields: integral (trapezoid of x(1-x)y(1-y) = (1/6 - dx^2/6)(1/6 - dy^2/6)),
    Q1 = value at the centre, Q2 = mean of x over [1/4,1/2]^2 = 0.375 (trapezoid is exact),
    Q3 = dy sum_j a v_{nx-1,j} / dx with a = 1."""
    P, Q = 4, 3
    H = oracle.Hierarchy(P, Q)
    nx, ny = 1 << P, 1 << Q
    X, Y = np.meshgrid(np.arange(nx + 1) / nx, np.arange(ny + 1) / ny)
    v = X * (1 - X) * Y * (1 - Y)
    H.set(P, Q, oracle.SOL, v)
    dx, dy = 1 / nx, 1 / ny
    assert H.qoi(P, Q, qoi=oracle.QOI_INTEGRAL) == pytest.approx((1 / 6 - dx**2 / 6) * (1 / 6 - dy**2 / 6), rel=1e-13)
    assert H.qoi(P, Q, qoi=oracle.QOI_POINT) == pytest.approx(0.25 * 0.25, rel=1e-14)
    assert H.qoi(P, Q, qoi=oracle.QOI_FLUX) == pytest.approx((1 - dx) * (1 / 6 - dy**2 / 6), rel=1e-13)
    H.set(P, Q, oracle.SOL, X.copy())
    assert H.qoi(P, Q, qoi=oracle.QOI_SUBDOMAIN) == pytest.approx(0.375, rel=1e-14)


def test_flux_qoi_reads_the_boundary_column_of_a_varying_field():
    """Q3 of Sec. 4 takes a(1, y_j) from the field's boundary column x = 1.  With
    Z(x, y) = 3x + log(1 + y) on the field nodes, a(1, y) = e^3 (1 + y), and the nodal
    v = x(1-x) y(1-y) on grid (p,q) gives v_{nx-1,j}/dx = (1 - dx) y_j (1 - y_j), so
    Q3 = e^3 (1 - dx) dy sum_j (y_j - y_j^3) = e^3 (1 - dx) [(1 - dy)/2 - (1 - dy)^2/4]
    (sum_j j = n(n-1)/2, sum_j j^3 = (n(n-1)/2)^2).  A column one node inside (a(1-h, y))
    or a row shifted by one field node changes the value; grids coarser than the
    field's finest (sy > 1) check the row stride."""
    P, Q = 3, 4
    NFx, NFy = (1 << (P + 1)) + 1, (1 << (Q + 1)) + 1
    FX, FY = np.meshgrid(np.arange(NFx) / (NFx - 1), np.arange(NFy) / (NFy - 1))
    Z = 3.0 * FX + np.log1p(FY)
    H = oracle.Hierarchy(P, Q, Z=Z.ravel())
    for p, q in [(P, Q), (2, 3), (3, 1), (1, 2)]:
        nx, ny = 1 << p, 1 << q
        X, Y = np.meshgrid(np.arange(nx + 1) / nx, np.arange(ny + 1) / ny)
        H.set(p, q, oracle.SOL, X * (1 - X) * Y * (1 - Y))
        dx, dy = 1 / nx, 1 / ny
        want = np.exp(3.0) * (1 - dx) * ((1 - dy) / 2 - (1 - dy) ** 2 / 4)
        assert H.qoi(p, q, qoi=oracle.QOI_FLUX) == pytest.approx(want, rel=1e-13), (p, q)


def test_grid_above_the_zero_guess_after_one_cycle_keeps_cycling():
    """Divergence reading: a grid stops as diverged only when a cycle leaves its
    relative residual above both 1 (the zero guess) and its initial guess's.  On this
    deterministic field (sharp variation along y, a 16 x 128 finest grid) the
    interpolated initial guess of grid (3,4) starts far above 1 and is still above 1
    after its first cycle; it must keep cycling, and every grid then meets eps and
    agrees with a dense direct solve of its own system."""
    P, Q = 4, 7
    NFy, NFx = inputs.field_grid_shape(P, Q)
    X, Y = np.meshgrid(np.arange(NFx) / (NFx - 1), np.arange(NFy) / (NFy - 1))
    Z = (2.0 * np.sin(14 * np.pi * Y + 1.3) * np.cos(2 * np.pi * X) + np.sin(16 * np.pi * X * Y)).ravel()
    prm = oracle.SolverParams(eps=1e-10, max_cycles=400)
    Qg, st, cyc, rr = oracle.solve_sample(P, Q, Z, prm)
    assert st == 0 and np.all(rr <= 1e-10)
    assert cyc[2, 3] > 10  # the grid that a stop at 1 would have abandoned after one cycle
    H = oracle.Hierarchy(P, Q, Z, prm)
    st2, cyc2, _ = H.fmsg()
    assert st2 == 0 and np.array_equal(cyc2, cyc)
    for p, q in [(3, 4), (3, 5)]:
        A = _dense(H, p, q)
        u = np.linalg.solve(A, np.ones(A.shape[0]))
        got = H.get(p, q, oracle.SOL)[1:-1, 1:-1].ravel()
        assert np.max(np.abs(got - u)) <= 1e-6 * np.max(np.abs(u))


# ------------------------------------------------------------------- MIMC --

def test_mixed_difference_worked_example():
    """Sec. 3 worked example: dQ_(3,4) = Q_(3,4) - Q_(2,4) - Q_(3,3) + Q_(2,3)."""
    p0, q0 = 2, 3
    L = (3, 4)
    rng = np.random.default_rng(0)
    Qg = rng.standard_normal((p0 + L[0], q0 + L[1]))
    Ql = lambda l1, l2: Qg[p0 + l1 - 1, q0 + l2 - 1]
    dQ, _ = oracle.mimc_differences(L, p0, q0, Qg)
    assert dQ[3, 4] == pytest.approx(Ql(3, 4) - Ql(2, 4) - Ql(3, 3) + Ql(2, 3), rel=1e-14, abs=1e-14)
    assert dQ[0, 0] == Ql(0, 0)
    assert dQ[2, 0] == pytest.approx(Ql(2, 0) - Ql(1, 0), abs=1e-15)
    assert dQ[0, 3] == pytest.approx(Ql(0, 3) - Ql(0, 2), abs=1e-15)


def test_telescoping_and_unit_probabilities():
    """Sum over 0 <= tau <= L of dQ_tau = Q_L (telescoping used in the unbiasedness
    proof, Sec. 3); with p_tau = 1 the estimator term Y equals Q_L."""
    rng = np.random.default_rng(2)
    for L in [(0, 0), (2, 0), (0, 3), (3, 2)]:
        Qg = rng.standard_normal((1 + L[0], 2 + L[1]))
        dQ, Y = oracle.mimc_differences(L, 1, 2, Qg, ptau=np.ones((5, 5)))
        assert dQ.sum() == pytest.approx(Qg[-1, -1], rel=1e-13, abs=1e-13)
        assert Y == pytest.approx(Qg[-1, -1], rel=1e-13, abs=1e-13)


def test_estimator_term_weights():
    """Y = sum dQ_tau / p_tau (Eq. (3.6)) with a geometric p_tau = exp(-r (tau1 + tau2))."""
    r = 0.5 * math.log(2) * 5  # Algorithm 3 initial law, beta = 4, gamma = 1
    pt = np.exp(-r * (np.arange(4)[:, None] + np.arange(4)[None, :]))
    Qg = np.arange(1.0, 1 + 3 * 4).reshape(3, 4) ** 1.5
    dQ, Y = oracle.mimc_differences((1, 2), 2, 2, Qg, ptau=pt)
    assert Y == pytest.approx(sum(dQ[a, b] / pt[a, b] for a in range(2) for b in range(3)), rel=1e-14)
    assert pt[1, 0] == pytest.approx(0.17677669529663687, rel=1e-14)  # 2^(-5/2)


def test_theorem1_cost_ratio_from_table1():
    """Theorem 1 with the Table 1 rates: (1 - x1)(1 - x2), x_j = 2^(-(gamma_j + beta_j)/2)."""
    rows = [l.split() for l in open(os.path.join(GOLD, "table1_rates.txt")) if l.strip() and l[0] != "#"]
    ratios = {}
    for r in rows:
        a1, a2, b1, b2, g1, g2 = map(float, r[1:])
        x1, x2 = 2 ** (-(g1 + b1) / 2), 2 ** (-(g2 + b2) / 2)
        # inclusion-exclusion form of Eq. (3.9) for d = 2
        ratios[r[0]] = 1 - (x1 + x2 - x1 * x2)
        assert ratios[r[0]] == pytest.approx((1 - x1) * (1 - x2), rel=1e-14)
    assert ratios["Q1"] == pytest.approx(0.753, abs=1e-3)
    assert ratios["Q2"] == pytest.approx(0.515, abs=1e-3)
    assert ratios["Q3"] == pytest.approx(0.387, abs=1e-3)
    assert ratios["Q3"] < ratios["Q2"] < ratios["Q1"]  # largest benefit for Q3 (Sec. 4)


# ----------------------------------------------- convergence study (Sec. 2) --

def test_std_transfer_adjoint():
    """Full weighting is 1/4 of the transpose of bilinear interpolation on
    vertex-centred grids: 4 <R f, e>_coarse = <f, P e>_fine over interior nodes,
    for random f and e (a wrong stencil weight breaks it)."""
    rng = np.random.default_rng(3)
    for P, Q in [(3, 3), (4, 2), (2, 5)]:
        H = oracle.Hierarchy(P, Q)
        f = np.zeros(H.shape(P, Q))
        f[1:-1, 1:-1] = rng.standard_normal((f.shape[0] - 2, f.shape[1] - 2))
        e = np.zeros(H.shape(P - 1, Q - 1))
        e[1:-1, 1:-1] = rng.standard_normal((e.shape[0] - 2, e.shape[1] - 2))
        Rf, Pe = H.std_restrict(P, Q, f), H.std_prolong(P, Q, e)
        assert 4.0 * np.sum(Rf * e) == pytest.approx(np.sum(f * Pe), rel=1e-13)
        # interpolation reproduces bilinear functions exactly (and restriction preserves constants inside)
        yy, xx = np.meshgrid(np.arange(e.shape[0]) / (e.shape[0] - 1), np.arange(e.shape[1]) / (e.shape[1] - 1),
                             indexing="ij")
        lin = 1.0 + 2.0 * xx - 3.0 * yy + 0.5 * xx * yy
        yf, xf = np.meshgrid(np.arange(f.shape[0]) / (f.shape[0] - 1), np.arange(f.shape[1]) / (f.shape[1] - 1),
                             indexing="ij")
        np.testing.assert_allclose(H.std_prolong(P, Q, lin)[1:-1, 1:-1],
                                   (1.0 + 2.0 * xf - 3.0 * yf + 0.5 * xf * yf)[1:-1, 1:-1], rtol=1e-14)


def test_std_line_solve_is_exact():
    """The coarsest standard-coarsening grid (one interior line) is solved exactly."""
    rng = np.random.default_rng(5)
    law = inputs.small_law(16)
    for P, Q, p, q in [(4, 3, 1, 3), (4, 3, 4, 1), (2, 2, 1, 1)]:
        Phi, sl = inputs.kl_basis(P, Q, law)
        H = oracle.Hierarchy(P, Q, Z=oracle.kl_field(Phi, sl, rng.standard_normal(16)))
        b = np.zeros(H.shape(p, q))
        b[1:-1, 1:-1] = rng.standard_normal((b.shape[0] - 2, b.shape[1] - 2))
        u = H.line_solve(p, q, b)
        Au = H.apply(p, q, u)
        np.testing.assert_allclose(Au[1:-1, 1:-1], b[1:-1, 1:-1], rtol=1e-12, atol=1e-12 * np.abs(b).max())


def test_std_convergence_textbook_poisson():
    """a = 1 on square grids: the standard-coarsening W(2,2) cycle with red-black
    Gauss-Seidel reduces the residual by well under 0.1 per cycle (textbook
    behaviour) and reaches the rounding floor, i.e. its fixed point is A^-1 b."""
    for P in (3, 5, 6):
        h = oracle.Hierarchy(P, P).cycle_history(1, 40)
        rho = (h[8] / h[0]) ** (1 / 8)
        assert rho < 0.1, (P, rho)
        assert h[-1] < 1e-12


def test_msg_robust_where_std_coarsening_degrades():
    """Sec. 2: multigrid with standard coarsening and a point smoother degrades
    on anisotropic problems; MSG does not.  With a = 1 on 64 x 4 cells (couplings
    256:1) the standard cycle's rate is poor while MSG's stays small."""
    H = oracle.Hierarchy(6, 2)
    hs, hm = H.cycle_history(1, 10), H.cycle_history(0, 10)
    rho_s = (hs[10] / hs[0]) ** 0.1
    rho_m = (hm[6] / hm[0]) ** (1 / 6)
    assert rho_s > 0.4 and rho_m < 0.1, (rho_s, rho_m)
