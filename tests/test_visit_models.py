"""Host models of the shared-memory visit kernels (csrc/solver.cu).

Resident visits (k_pre_res, k_post_res): the whole grid sits in shared memory
with the columns split by parity; the model below replays their index
arithmetic (colour-slot mapping, residual in place of b, restriction and
prolongation slots) and must give, bit for bit, the phase-by-phase visit.

Streamed visits (k_visit_stream): a grid too large for shared memory is swept through a ring of rows; in step t
operation k of the visit's chain (PRE: 2 nu1 red-black colour phases, then the
residual; POST: the prolongation, then 2 nu2 colour phases) works on row
t - 2k, u row t - 2(2nu+1) is written back and PRE restricts the residual row
finished one step earlier.  This test replays exactly that index arithmetic
(row slots, work-item mapping, write-back and restriction rows, loads
kStreamAhead rows ahead into a ring of R = kStreamAhead + 2(2nu+1) + 3 rows)
on the host, and checks, for many grid shapes and sweep counts:

* every ring read finds the grid row it expects (no slot reloaded too early);
* within a step no work item writes a location another item of the step reads
  or writes, so one barrier per step suffices;
* a row loaded at the start of a step is not read by the previous step, which
  runs without a barrier before those loads;
* the result (u, the children's right-hand sides) equals, bit for bit, the
  phase-by-phase visit of Algorithm 1 (red-black Gauss-Seidel, residual,
  Eq. (2.3) restriction; Eq. (2.4)/(2.5) prolongation).

The phase-by-phase reference below is written from Algorithm 1 directly, in the
natural node layout, independent of the schedule being checked.
"""
import itertools

import numpy as np
import pytest

AHEAD = 4  # kStreamAhead


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


# ---------------------------------------------------------------- stream --

class Ring:
    """Ring planes with a row tag per ring row; logs each access of a step."""

    def __init__(self, R, W):
        self.R, self.W = R, W
        self.p = {k: np.full(R * W, np.nan) for k in "UBXY"}
        self.tag = [-1] * R
        self.log = None

    def idx(self, j, slot):
        assert self.tag[j % self.R] == j, f"ring row {j % self.R} holds row {self.tag[j % self.R]}, not {j}"
        return (j % self.R) * self.W + slot

    def rd(self, who, plane, j, slot):
        k = self.idx(j, slot)
        self.log.append((who, plane, k, "r"))
        return self.p[plane][k]

    def wr(self, who, plane, j, slot, v):
        k = self.idx(j, slot)
        self.log.append((who, plane, k, "w"))
        self.p[plane][k] = v


def check_step(log):
    """No location written by one work item is touched by another of the step."""
    writers, touched = {}, {}
    for who, plane, k, m in log:
        touched.setdefault((plane, k), set()).add(who)
        if m == "w":
            writers.setdefault((plane, k), set()).add(who)
    for key, ws in writers.items():
        assert len(ws) == 1 and touched[key] == ws, f"hazard on {key}: writers {ws}, touched by {touched[key]}"


def stream_visit(pre, u, b, ax, ay, nx, ny, nu, zero, ucx=None, ucy=None, omega=1.0, ring=None):
    W, hs, half = nx + 1, nx // 2 + 1, nx // 2
    p = nx.bit_length() - 1
    nops = 2 * nu + 1
    R = AHEAD + 2 * nops + 3 if ring is None else ring
    Rr = min(R, ny + 1)
    ring = Ring(Rr, W)
    gu = u.copy()
    cxb, cyb = {}, {}
    ncol = 2 * nu * half
    prev_reads = set()

    def load_row(j):
        ring.tag[j % Rr] = j
        for i in range(nx + 1):
            s = (j % Rr) * W + split_slot(hs, i)
            assert ("U", s) not in prev_reads and ("B", s) not in prev_reads and ("X", s) not in prev_reads \
                and ("Y", s) not in prev_reads, f"row {j} loaded over a location the previous step reads"
            c = j * W + i
            ring.p["U"][s] = 0.0 if (pre and zero) else u[c]
            ring.p["B"][s] = b[c]
            ring.p["X"][s] = ax[c]
            ring.p["Y"][s] = ay[c]

    for j in range(AHEAD):
        if j <= ny:
            load_row(j)
    for st in range(ny + 2 * nops + 1):
        if st + AHEAD <= ny:
            load_row(st + AHEAD)
        ring.log = []
        for w in range(ncol + nx):
            if pre:
                k, m = (w >> (p - 1), w & (half - 1)) if w < ncol else (2 * nu, w - ncol)
            else:
                k, m = (0, w) if w < nx else (1 + ((w - nx) >> (p - 1)), (w - nx) & (half - 1))
            j = st - 2 * k
            if j < 1 or j > ny - 1:
                continue
            who = ("op", w)
            if (k < 2 * nu) if pre else (k > 0):
                colour = (k & 1) if pre else ((k - 1) & 1)
                odd = (j + colour) & 1
                if not odd and m == half - 1:
                    continue
                s, wv = (hs + m, m) if odd else (m + 1, hs + m)
                aw, ae = ring.rd(who, "X", j, wv), ring.rd(who, "X", j, s)
                as_, an = ring.rd(who, "Y", j - 1, s), ring.rd(who, "Y", j, s)
                nb = (aw * ring.rd(who, "U", j, wv) + ae * ring.rd(who, "U", j, wv + 1)) + \
                     (as_ * ring.rd(who, "U", j - 1, s) + an * ring.rd(who, "U", j + 1, s))
                ring.wr(who, "U", j, s, (ring.rd(who, "B", j, s) + nb) * (1.0 / (aw + ae + as_ + an)))
            elif pre:
                colour = int(m >= half)
                kk = m - colour * half
                odd = (j + colour) & 1
                if not odd and kk == half - 1:
                    continue
                s, wv = (hs + kk, kk) if odd else (kk + 1, hs + kk)
                aw, ae = ring.rd(who, "X", j, wv), ring.rd(who, "X", j, s)
                as_, an = ring.rd(who, "Y", j - 1, s), ring.rd(who, "Y", j, s)
                Au = (aw + ae + as_ + an) * ring.rd(who, "U", j, s) - \
                     (aw * ring.rd(who, "U", j, wv) + ae * ring.rd(who, "U", j, wv + 1)) - \
                     (as_ * ring.rd(who, "U", j - 1, s) + an * ring.rd(who, "U", j + 1, s))
                ring.wr(who, "B", j, s, ring.rd(who, "B", j, s) - Au)
            else:
                i = m
                if i == 0:
                    continue
                s, wv = split_slot(hs, i), split_slot(hs, i - 1)
                aw, ae = ring.rd(who, "X", j, wv), ring.rd(who, "X", j, s)
                as_, an = ring.rd(who, "Y", j - 1, s), ring.rd(who, "Y", j, s)
                corr = prolong_corr(None, None, None, W, i, j, nx, ucx, ucy, aw, ae, as_, an)
                ring.wr(who, "U", j, s, ring.rd(who, "U", j, s) + omega * corr)
        jw = st - 2 * nops
        if 0 <= jw <= ny:
            for i in range(nx + 1):
                gu[jw * W + i] = ring.rd(("wb", i), "U", jw, split_slot(hs, i))
        jr = jw + 1
        if pre and nx > 2 and 1 <= jr <= ny - 1:
            Wc = half + 1
            for ic in range(1, half):
                who = ("rx", ic)
                cxb[jr * Wc + ic] = 0.25 * (ring.rd(who, "B", jr, hs + ic - 1) + 2.0 * ring.rd(who, "B", jr, ic)
                                            + ring.rd(who, "B", jr, hs + ic))
        if pre and ny > 2 and (jr & 1) and 3 <= jr <= ny - 1:
            jc = (jr - 1) >> 1
            for i in range(1, nx):
                who, s = ("ry", i), split_slot(hs, i)
                cyb[jc * W + i] = 0.25 * (ring.rd(who, "B", jr - 2, s) + 2.0 * ring.rd(who, "B", jr - 1, s)
                                          + ring.rd(who, "B", jr, s))
        check_step(ring.log)
        prev_reads = {(pl, k) for _, pl, k, _ in ring.log}
    return gu, cxb, cyb


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


@pytest.mark.parametrize("p,q,nu", [(1, 3, 2), (2, 2, 2), (3, 4, 2), (4, 5, 2), (5, 3, 2), (2, 6, 2), (3, 5, 1),
                                    (3, 5, 3), (4, 4, 0), (2, 1, 2), (4, 2, 2)])
def test_streamed_pre_equals_phase_order(p, q, nu):
    nx, ny = 1 << p, 1 << q
    u, b, ax, ay, _ = _grid(nx, ny, 7 * p + q)
    for zero in (False, True):
        ru, rcx, rcy = ref_pre(u, b, ax, ay, nx, ny, nu, zero)
        gu, gcx, gcy = stream_visit(True, u, b, ax, ay, nx, ny, nu, zero)
        assert np.array_equal(gu, ru)
        assert gcx == rcx and gcy == rcy


@pytest.mark.parametrize("p,q,nu", [(1, 3, 2), (2, 2, 2), (3, 4, 2), (4, 5, 2), (5, 3, 2), (2, 6, 2), (3, 5, 1),
                                    (3, 5, 3), (4, 4, 0), (2, 1, 2), (4, 2, 2)])
def test_streamed_post_equals_phase_order(p, q, nu):
    nx, ny = 1 << p, 1 << q
    u, b, ax, ay, rng = _grid(nx, ny, 11 * p + q)
    for has_x, has_y in itertools.product((False, True), repeat=2):
        if (has_x and p == 1) or (has_y and q == 1) or not (has_x or has_y):
            continue
        ucx = rng.standard_normal((nx // 2 + 1) * (ny + 1)) if has_x else None
        ucy = rng.standard_normal((nx + 1) * (ny // 2 + 1)) if has_y else None
        ru = ref_post(u, b, ax, ay, nx, ny, nu, ucx, ucy, 0.9)
        gu, _, _ = stream_visit(False, u, b, ax, ay, nx, ny, nu, False, ucx, ucy, 0.9)
        assert np.array_equal(gu, ru)


def test_a_ring_one_row_short_is_caught():
    """The checks see a ring one row smaller than the kernel's: a row is then
    loaded over one the previous step still reads (PRE: the residual row the
    y-restriction reads; POST, which has no restriction, needs two rows less to
    clash with the write-back, and the kernel keeps the PRE size for both)."""
    nx, ny, nu = 8, 32, 2
    u, b, ax, ay, _ = _grid(nx, ny, 3)
    with pytest.raises(AssertionError):
        stream_visit(True, u, b, ax, ay, nx, ny, nu, False, ring=AHEAD + 2 * (2 * nu + 1) + 2)
    with pytest.raises(AssertionError):
        stream_visit(False, u, b, ax, ay, nx, ny, nu, False, ucx=np.zeros((nx // 2 + 1) * (ny + 1)),
                     ring=AHEAD + 2 * (2 * nu + 1) + 1)


# ------------------------------------------------------------- resident --

def _colour_slots(p, ny, colour, h, W):
    """(self, west) slots of the nodes of one colour, in the kernels' order."""
    half, sh = (1 << p) >> 1, p - 1
    for k in range((ny - 1) << sh):
        j, kk = 1 + (k >> sh), k & (half - 1)
        odd = (j + colour) & 1
        if not odd and kk == half - 1:
            continue
        yield j * W + (h + kk if odd else kk + 1), j * W + (kk if odd else h + kk)


def _res_load(u, b, ax, ay, p, q, zero):
    nx, ny = 1 << p, 1 << q
    W, h = nx + 1, nx // 2 + 1
    S = {k: np.full(W * (ny + 1), np.nan) for k in "UBXY"}
    for j in range(ny + 1):
        for i in range(nx + 1):
            c, s = j * W + i, j * W + split_slot(h, i)
            S["U"][s], S["B"][s], S["X"][s], S["Y"][s] = 0.0 if zero else u[c], b[c], ax[c], ay[c]
    return S, nx, ny, W, h


def _res_smooth(S, p, ny, W, h, sweeps):
    U, B, X, Y = S["U"], S["B"], S["X"], S["Y"]
    for _ in range(sweeps):
        for colour in (0, 1):
            for s, w in list(_colour_slots(p, ny, colour, h, W)):
                aw, ae, as_, an = X[w], X[s], Y[s - W], Y[s]
                nb = (aw * U[w] + ae * U[w + 1]) + (as_ * U[s - W] + an * U[s + W])
                U[s] = (B[s] + nb) * (1.0 / (aw + ae + as_ + an))


def _res_store(S, nx, ny, W, h):
    return np.array([S["U"][j * W + split_slot(h, i)] for j in range(ny + 1) for i in range(nx + 1)])


def resident_pre(u, b, ax, ay, p, q, nu, zero):
    S, nx, ny, W, h = _res_load(u, b, ax, ay, p, q, zero)
    _res_smooth(S, p, ny, W, h, nu)
    U, B, X, Y = S["U"], S["B"], S["X"], S["Y"]
    for colour in (0, 1):
        for s, w in list(_colour_slots(p, ny, colour, h, W)):
            aw, ae, as_, an = X[w], X[s], Y[s - W], Y[s]
            B[s] = B[s] - ((aw + ae + as_ + an) * U[s] - (aw * U[w] + ae * U[w + 1]) - (as_ * U[s - W] + an * U[s + W]))
    cxb, cyb = {}, {}
    if p > 1:  # k = (row, ic) with ncx = 2^(p-1) slots a row
        shc, ncx = p - 1, nx >> 1
        for k in range((ny - 1) << shc):
            ic, j = k & (ncx - 1), 1 + (k >> shc)
            if ic:
                base = j * W
                cxb[j * (ncx + 1) + ic] = 0.25 * (B[base + h + ic - 1] + 2.0 * B[base + ic] + B[base + h + ic])
    if q > 1:
        for k in range(((ny >> 1) - 1) << p):
            i, jc = k & (nx - 1), 1 + (k >> p)
            if i:
                s = 2 * jc * W + split_slot(h, i)
                cyb[jc * W + i] = 0.25 * (B[s - W] + 2.0 * B[s] + B[s + W])
    return _res_store(S, nx, ny, W, h), cxb, cyb


def resident_post(u, b, ax, ay, p, q, nu, ucx, ucy, omega):
    S, nx, ny, W, h = _res_load(u, b, ax, ay, p, q, False)
    U, X, Y = S["U"], S["X"], S["Y"]
    for k in range((ny - 1) << p):
        i, j = k & (nx - 1), 1 + (k >> p)
        if i == 0:
            continue
        s, w = j * W + split_slot(h, i), j * W + split_slot(h, i - 1)
        U[s] += omega * prolong_corr(None, None, None, W, i, j, nx, ucx, ucy, X[w], X[s], Y[s - W], Y[s])
    _res_smooth(S, p, ny, W, h, nu)
    return _res_store(S, nx, ny, W, h)


RES_CASES = [(1, 3, 2), (2, 2, 2), (3, 4, 2), (2, 5, 2), (4, 3, 2), (5, 2, 2), (3, 3, 1), (4, 4, 0), (2, 1, 2),
             (1, 1, 2)]


@pytest.mark.parametrize("p,q,nu", RES_CASES)
def test_resident_pre_equals_phase_order(p, q, nu):
    """Every child right-hand-side entry is written (same key sets) with the
    phase-order value; a wrong row/slot shift in the restriction fails here."""
    nx, ny = 1 << p, 1 << q
    u, b, ax, ay, _ = _grid(nx, ny, 5 * p + q)
    for zero in (False, True):
        ru, rcx, rcy = ref_pre(u, b, ax, ay, nx, ny, nu, zero)
        gu, gcx, gcy = resident_pre(u, b, ax, ay, p, q, nu, zero)
        assert np.array_equal(gu, ru)
        assert gcx == rcx and gcy == rcy


@pytest.mark.parametrize("p,q,nu", RES_CASES)
def test_resident_post_equals_phase_order(p, q, nu):
    nx, ny = 1 << p, 1 << q
    u, b, ax, ay, rng = _grid(nx, ny, 13 * p + q)
    for has_x, has_y in itertools.product((False, True), repeat=2):
        if (has_x and p == 1) or (has_y and q == 1) or not (has_x or has_y):
            continue
        ucx = rng.standard_normal((nx // 2 + 1) * (ny + 1)) if has_x else None
        ucy = rng.standard_normal((nx + 1) * (ny // 2 + 1)) if has_y else None
        assert np.array_equal(resident_post(u, b, ax, ay, p, q, nu, ucx, ucy, 0.9),
                              ref_post(u, b, ax, ay, nx, ny, nu, ucx, ucy, 0.9))
