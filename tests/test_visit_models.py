"""Host model of the register-cached visit kernel (k_visit_reg in csrc/solver.cu).

The kernel keeps a grid's u in shared memory with the columns split by parity
(even i in slots 0..nx/2, odd i after them) and gives thread t colour slot
t + m blockDim of each colour.  The model below replays its index arithmetic
(colour slot -> node and split slots, prolongation from the slot's (i, j),
residual into a second plane, restriction slots) in exact host arithmetic and
must give, bit for bit, the phase-by-phase visit written from Algorithm 1
(red-black Gauss-Seidel, residual, Eq. (2.3) restriction; Eq. (2.4)/(2.5)
prolongation) in the natural node layout.  Every child right-hand-side entry
must be written: a wrong row or slot shift leaves entries out and fails the
key-set comparison.
"""
import itertools

import numpy as np
import pytest

def split_slot(h, i):
    return h + (i >> 1) if i & 1 else i >> 1


# ------------------------------------------------------- phase-by-phase --

def ref_smooth(u, b, ax, ay, nx, ny, sweeps):
    W = nx + 1
    for _ in range(sweeps):
        for colour in (0, 1):
            for j in range(1, ny):
                for i in range(1, nx):
                    if (i + j) & 1 != colour:
                        continue
                    c = j * W + i
                    aw, ae, as_, an = ax[c - 1], ax[c], ay[c - W], ay[c]
                    nb = (aw * u[c - 1] + ae * u[c + 1]) + (as_ * u[c - W] + an * u[c + W])
                    u[c] = (b[c] + nb) * (1.0 / (aw + ae + as_ + an))


def ref_pre(u, b, ax, ay, nx, ny, nu, zero):
    W = nx + 1
    u = np.zeros_like(u) if zero else u.copy()
    ref_smooth(u, b, ax, ay, nx, ny, nu)
    r = np.zeros_like(u)
    for j in range(1, ny):
        for i in range(1, nx):
            c = j * W + i
            aw, ae, as_, an = ax[c - 1], ax[c], ay[c - W], ay[c]
            Au = (aw + ae + as_ + an) * u[c] - (aw * u[c - 1] + ae * u[c + 1]) - (as_ * u[c - W] + an * u[c + W])
            r[c] = b[c] - Au
    ncx, Wc = nx // 2, nx // 2 + 1
    cxb = {}
    if nx > 2:
        for j in range(1, ny):
            for ic in range(1, ncx):
                c = j * W + 2 * ic
                cxb[j * Wc + ic] = 0.25 * (r[c - 1] + 2.0 * r[c] + r[c + 1])
    cyb = {}
    if ny > 2:
        for jc in range(1, ny // 2):
            for i in range(1, nx):
                c = 2 * jc * W + i
                cyb[jc * W + i] = 0.25 * (r[c - W] + 2.0 * r[c] + r[c + W])
    return u, cxb, cyb


def ref_post(u, b, ax, ay, nx, ny, nu, ucx, ucy, omega):
    W = nx + 1
    u = u.copy()
    for j in range(1, ny):
        for i in range(1, nx):
            c = j * W + i
            u[c] += omega * prolong_corr(ax, ay, c, W, i, j, nx, ucx, ucy, ax[c - 1], ax[c], ay[c - W], ay[c])
    ref_smooth(u, b, ax, ay, nx, ny, nu)
    return u


def prolong_corr(ax, ay, c, W, i, j, nx, ucx, ucy, aw, ae, as_, an):
    vx = vy = 0.0
    if ucx is not None:
        Wc = nx // 2 + 1
        r = j * Wc + (i >> 1)
        vx = 0.5 * (ucx[r] + ucx[r + 1]) if i & 1 else ucx[r]
    if ucy is not None:
        r = (j >> 1) * W + i
        vy = 0.5 * (ucy[r] + ucy[r + W]) if j & 1 else ucy[r]
    if ucx is not None and ucy is not None:
        cxv, cyv = aw + ae, as_ + an
        x2, y2 = cxv * cxv, cyv * cyv
        sc = 1.0 / (x2 + y2)
        return (x2 * sc) * vx + (y2 * sc) * vy
    return vx if ucx is not None else vy


def _grid(nx, ny, seed):
    rng = np.random.default_rng(seed)
    n = (nx + 1) * (ny + 1)
    u = rng.standard_normal(n)
    W = nx + 1
    for j in range(ny + 1):  # boundary nodes hold zeros, as in the solver's scratch
        for i in (0, nx):
            u[j * W + i] = 0.0
    u[:W] = 0.0
    u[ny * W:] = 0.0
    return u, rng.standard_normal(n), rng.uniform(0.5, 2.0, n), rng.uniform(0.5, 2.0, n), rng




def colour_node(k, colour, p):
    sh = p - 1
    half = 1 << sh
    j = 1 + (k >> sh)
    kk = k & (half - 1)
    odd = (j + colour) & 1
    i = 2 * kk + 1 if odd else 2 * kk + 2
    return (odd or kk != half - 1), i, j


def reg_visit(pre, u, b, ax, ay, p, q, nu, zero=False, ucx=None, ucy=None, omega=1.0, threads=64, npt=2):
    nx, ny = 1 << p, 1 << q
    W, hs = nx + 1, nx // 2 + 1
    nslot = (ny - 1) << (p - 1)
    assert threads * npt >= nslot
    U = np.full(W * (ny + 1), np.nan)
    Rs = np.full(W * (ny + 1), np.nan)
    for j in range(ny + 1):
        for i in range(nx + 1):
            U[j * W + split_slot(hs, i)] = 0.0 if (pre and zero) else u[j * W + i]
    nodes = []  # per thread, per colour, per m: (s, w, aw, ae, as, an, dg, iv, b, i, j)
    for t in range(threads):
        for c in (0, 1):
            for m in range(npt):
                k = t + m * threads
                if k >= nslot:
                    continue
                ok, i, j = colour_node(k, c, p)
                if not ok:
                    continue
                g = j * W + i
                aw, ae, as_, an = ax[g - 1], ax[g], ay[g - W], ay[g]
                dg = aw + ae + as_ + an
                nodes.append((c, j * W + split_slot(hs, i), j * W + split_slot(hs, i - 1), aw, ae, as_, an, dg,
                              1.0 / dg, b[g], i, j))
    if not pre:
        for c, s, w, aw, ae, as_, an, dg, iv, bb, i, j in nodes:
            U[s] += omega * prolong_corr(None, None, None, W, i, j, nx, ucx, ucy, aw, ae, as_, an)
    for _ in range(nu):
        for colour in (0, 1):
            for c, s, w, aw, ae, as_, an, dg, iv, bb, i, j in nodes:
                if c == colour:
                    nb = (aw * U[w] + ae * U[w + 1]) + (as_ * U[s - W] + an * U[s + W])
                    U[s] = (bb + nb) * iv
    cxb, cyb = {}, {}
    if pre:
        for c, s, w, aw, ae, as_, an, dg, iv, bb, i, j in nodes:
            Rs[s] = bb - (dg * U[s] - (aw * U[w] + ae * U[w + 1]) - (as_ * U[s - W] + an * U[s + W]))
        if p > 1:
            shc, ncx = p - 1, nx >> 1
            for k in range((ny - 1) << shc):
                ic, j = k & (ncx - 1), 1 + (k >> shc)
                if ic:
                    base = j * W
                    cxb[j * (ncx + 1) + ic] = 0.25 * (Rs[base + hs + ic - 1] + 2.0 * Rs[base + ic] + Rs[base + hs + ic])
        if q > 1:
            for k in range(((ny >> 1) - 1) << p):
                i, jc = k & (nx - 1), 1 + (k >> p)
                if i:
                    s = 2 * jc * W + split_slot(hs, i)
                    cyb[jc * W + i] = 0.25 * (Rs[s - W] + 2.0 * Rs[s] + Rs[s + W])
    gu = np.array([U[j * W + split_slot(hs, i)] for j in range(ny + 1) for i in range(nx + 1)])
    return gu, cxb, cyb


CASES = [(1, 3, 2), (2, 2, 2), (3, 4, 2), (2, 5, 2), (4, 3, 2), (5, 2, 2), (3, 3, 1), (4, 4, 0), (2, 1, 2), (1, 1, 2),
         (6, 1, 2)]


def _launch(p, q):
    """Threads and nodes per thread as the host picks them (128-thread target)."""
    nslot = ((1 << q) - 1) << (p - 1)
    npt = 1
    while npt < 4 and -(-nslot // npt) > 128:
        npt *= 2
    per = -(-nslot // npt)  # ceil
    return max(32, -(-per // 32) * 32), npt


@pytest.mark.parametrize("p,q,nu", CASES)
def test_register_visit_pre_equals_phase_order(p, q, nu):
    nx, ny = 1 << p, 1 << q
    u, b, ax, ay, _ = _grid(nx, ny, 5 * p + q)
    for threads, npt in (_launch(p, q), (32, 4 if ((ny - 1) << (p - 1)) > 64 else 2)):
        if threads * npt < ((ny - 1) << (p - 1)):
            continue
        for zero in (False, True):
            ru, rcx, rcy = ref_pre(u, b, ax, ay, nx, ny, nu, zero)
            gu, gcx, gcy = reg_visit(True, u, b, ax, ay, p, q, nu, zero, threads=threads, npt=npt)
            assert np.array_equal(gu, ru)
            assert gcx == rcx and gcy == rcy


@pytest.mark.parametrize("p,q,nu", CASES)
def test_register_visit_post_equals_phase_order(p, q, nu):
    nx, ny = 1 << p, 1 << q
    u, b, ax, ay, rng = _grid(nx, ny, 13 * p + q)
    threads, npt = _launch(p, q)
    for has_x, has_y in itertools.product((False, True), repeat=2):
        if (has_x and p == 1) or (has_y and q == 1) or not (has_x or has_y):
            continue
        ucx = rng.standard_normal((nx // 2 + 1) * (ny + 1)) if has_x else None
        ucy = rng.standard_normal((nx + 1) * (ny // 2 + 1)) if has_y else None
        gu, _, _ = reg_visit(False, u, b, ax, ay, p, q, nu, ucx=ucx, ucy=ucy, omega=0.9, threads=threads, npt=npt)
        assert np.array_equal(gu, ref_post(u, b, ax, ay, nx, ny, nu, ucx, ucy, 0.9))


def test_a_wrong_restriction_shift_is_caught():
    """The x-restriction enumerates (row, ic) with 2^(p-1) slots a row; with
    2^(p-2) it leaves entries of the child's right-hand side unwritten."""
    p, q, nu = 3, 4, 2
    nx, ny = 1 << p, 1 << q
    u, b, ax, ay, _ = _grid(nx, ny, 1)
    _, rcx, _ = ref_pre(u, b, ax, ay, nx, ny, nu, False)
    shc, ncx = p - 2, nx >> 1
    keys = set()
    for k in range((ny - 1) << shc):
        ic, j = k & (ncx - 1), 1 + (k >> shc)
        if ic:
            keys.add(j * (ncx + 1) + ic)
    assert keys != set(rcx)
