"""Element-by-element parity of the solutions on every grid (Algorithm 2 returns
one solution per grid of the hierarchy) between the CUDA path and the oracle.

Both sides stop when their own FP64 residual satisfies ||1 - A u||_h <=
relres ||1||_h, so their difference e = u_gpu - u_oracle obeys
    ||e||_h <= (relres_gpu + relres_oracle) ||1||_h / lambda_min(A).
A is a sum of a_face (difference)^2 / h^2 terms with every face coefficient >=
a_min = exp(min Z) (the series mean of values >= a_min is >= a_min), so
A >= a_min L_h with L_h the Dirichlet five-point Laplacian, whose smallest
eigenvalue is 4 sin^2(pi dx/2)/dx^2 + 4 sin^2(pi dy/2)/dy^2 >= 8 + 8 (each term
decreases in the mesh width and equals 8 at width 1/2).  The test therefore
checks ||e||_h <= 1.01 (relres_gpu + relres_oracle) ||1||_h / (16 a_min) on
every grid, with the relres values each side reports, and that boundary nodes
are exactly zero.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1907_12334_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def msg():
    from paper_1907_12334_gb300 import build, msg as m

    build.build()
    m.load()
    return m


def _oracle_solutions(P, Q, Z, eps):
    H = oracle.Hierarchy(P, Q, Z=Z, prm=oracle.SolverParams(eps=eps, max_cycles=600))
    st, _, rr = H.fmsg()
    sols = {(p, q): H.get(p, q, oracle.SOL) for p in range(1, P + 1) for q in range(1, Q + 1)}
    return st, rr, sols


def _check(msg, shapes, Zs, eps_gpu=1e-10, eps_orc=1e-12, precision=None):
    prm = msg.SolverParams(eps=eps_gpu, max_cycles=400, **({} if precision is None else {"precision": precision}))
    pq = np.array(shapes, dtype=np.int32)
    Qd, st, cyc, rr, u = msg.solve(pq, torch.from_numpy(np.concatenate(Zs)).cuda(), prm, with_u=True)
    torch.cuda.synchronize()
    st, rr, u = st.cpu().numpy(), rr.cpu().numpy(), u.cpu().numpy()
    with ThreadPoolExecutor(max_workers=len(shapes)) as ex:
        orc = list(ex.map(lambda a: _oracle_solutions(a[0][0], a[0][1], a[1], eps_orc), zip(shapes, Zs)))
    uo = qo = 0
    compared = 0
    for i, ((P, Q), Z) in enumerate(zip(shapes, Zs)):
        n_u = msg.msg_solution_values(pq[i:i + 1])
        block = u[uo:uo + n_u]
        ost, orr, osol = orc[i]
        # the GPU must meet its eps; the oracle's own target is tighter than it can always
        # reach in 600 cycles on the widest grids, and the bound uses the residual it reports
        assert st[i] == 0, (i, st[i])
        assert np.all(orr <= 1e-10), (i, ost, orr.max())
        amin = float(np.exp(np.min(Z)))
        for p in range(1, P + 1):
            for q in range(1, Q + 1):
                g = msg.grid_view(block, P, Q, p, q)
                o = osol[(p, q)]
                nx, ny = 1 << p, 1 << q
                dxdy = 1.0 / (nx * ny)
                assert not g[0].any() and not g[-1].any() and not g[:, 0].any() and not g[:, -1].any()
                rg, ro = rr[qo + (p - 1) * Q + (q - 1)], orr[p - 1, q - 1]
                norm1 = np.sqrt((nx - 1) * (ny - 1) * dxdy)
                bound = 1.01 * (rg + ro) * norm1 / (16.0 * amin)
                err = np.sqrt(dxdy * np.sum((g - o) ** 2))
                assert err <= bound, (i, p, q, err, bound)
                compared += g.size
        uo += n_u
        qo += P * Q
    return compared


def test_solution_fields_full_size_256(msg):
    """Four samples of the bench workload's shape (256 x 256, all 64 grids, M = 400),
    mixed cycles, every node of every grid."""
    P = Q = 8
    S, M = 4, 400
    Phi, sl = inputs.kl_basis(P, Q, inputs.FieldLaw(M=M))
    xi = oracle.normals_batch(11, 0, S, M)
    Zs = [oracle.kl_field(Phi, sl, xi[i]) for i in range(S)]
    assert _check(msg, [(P, Q)] * S, Zs) > 4 * 260_000


def test_solution_fields_uneven_with_a_512_side(msg):
    """Uneven shapes in one call, one of them 512 cells wide (the uneven workload's
    largest extent), FP64 and mixed cycles."""
    shapes = [(9, 3), (2, 7), (5, 5), (3, 2), (1, 6)]
    M = 32
    Zs = []
    for k, (P, Q) in enumerate(shapes):
        Phi, sl = inputs.kl_basis(P, Q, inputs.small_law(M))
        Zs.append(oracle.kl_field(Phi, sl, oracle.normals(5, k, M)))
    _check(msg, shapes, Zs)
    _check(msg, shapes, Zs, precision=0)
