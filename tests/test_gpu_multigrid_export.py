"""The multigrid set-up's products read back from the device
(pgo_graph_multigrid_export) against a plain numpy construction from the
exported inputs of each step, level by level.  The PCG tests check the
hierarchy only through convergence; these check what k_amg_setup writes.

With A_0 = H + lambda I over the free vertices (H from pg.linearize in the
same precision, the gauge vertex's rows and columns dropped) and, for
l >= 1, A_l the exported Galerkin operator:
  D_l^-1     the inverse of each diagonal block of A_l;
  T_0        Adj(S_v S_r^-1) for vertex v and the first vertex r of its
             aggregate (the rigid motion of the aggregate in the left
             tangent), from the oracle's Sim(3) functions;
  P_l        (I - 4 / (3 rho_l) D_l^-1 A_l) T_l, T_l placed by the aggregates;
  Q_l        P_l - (1 / rho_l) D_l^-1 A_l P_l;
  A_{l+1}    P_l^T A_l P_l;
  W          Q_d A_L^-1 Q_d^T on the level d = L - 1 next to the coarsest.
Each comparison is relative to the largest entry of the reference:
1e-10 for the FP64 set-up; for the FP32 set-up 2e-5 (products of FP32 blocks
summed in FP32 over tens of terms), and 2e-4 for W, which passes through the
coarsest operator's inverse.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_17201_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def dense(ptr, col, blocks, nrows, ncols):
    M = np.zeros((7 * nrows, 7 * ncols))
    for r in range(nrows):
        for k in range(ptr[r], ptr[r + 1]):
            M[7 * r:7 * r + 7, 7 * col[k]:7 * col[k] + 7] = blocks[k]
    return M


def block_diag_inv(A, n, live):
    Dinv = np.zeros_like(A)
    for v in range(n):
        if live[v]:
            s = slice(7 * v, 7 * v + 7)
            Dinv[s, s] = np.linalg.inv(A[s, s])
    return Dinv


def close(got, ref, tol, what):
    err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert err <= tol, f"{what}: {err:.2e} > {tol:.0e}"
    return err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_setup_products_match_plain_construction(precision):
    from paper_2603_17201_gb300 import PoseGraph
    g = syn.make_graph("figure8", 300, seed=5, window=6, n_loops=2, meas_noise=True)
    g.fixed_vertex = 7
    pg = PoseGraph.from_synthetic(g)
    lin = pg.linearize(precision, jacobians=False)
    Hd, Ho = lin["h_diag"], lin["h_off"]
    N = g.n_vertices
    lam = 1e-3 * max(np.diag(Hd[v]).max() for v in range(N))
    pg.precondition_async(lam, precision=precision)
    torch.cuda.synchronize()
    info = pg.multigrid_info()
    Lc = len(info) - 1
    assert Lc >= 2, info
    tol = 1e-10 if precision == "fp64" else 2e-5
    ex = lambda l, name: pg.multigrid_export(l, name, precision)  # noqa: E731

    # level 0 operator: H + lambda I on the free vertices
    live = np.ones(N, bool)
    live[g.fixed_vertex] = False
    A = np.zeros((7 * N, 7 * N))
    for v in range(N):
        A[7 * v:7 * v + 7, 7 * v:7 * v + 7] = Hd[v] + lam * np.eye(7)
    for e, (i, j) in enumerate(zip(g.edge_i, g.edge_j)):
        A[7 * i:7 * i + 7, 7 * j:7 * j + 7] += Ho[e]
        A[7 * j:7 * j + 7, 7 * i:7 * i + 7] += Ho[e].T
    keep = np.repeat(live, 7)
    A[~keep, :] = 0.0
    A[:, ~keep] = 0.0

    # tentative blocks of level 0 from the poses (oracle Sim(3) functions)
    agg0 = ex(0, "agg")
    T0 = ex(0, "t")
    first = {}
    for v in range(N):
        if agg0[v] >= 0 and agg0[v] not in first:
            first[agg0[v]] = v
    for v in range(N):
        if agg0[v] < 0:
            continue
        r = first[agg0[v]]
        ref = O.adj(O.compose(g.poses_init[v], O.inverse(g.poses_init[r])))
        close(T0[v], ref, tol, f"T_0 vertex {v}")

    n = N
    for l in range(Lc):
        n_next = info[l + 1]["nodes"]
        agg = ex(l, "agg")
        rho = ex(l, "rho")[0]
        Dinv = block_diag_inv(A, n, agg >= 0)
        close(dense(np.arange(n + 1), np.arange(n), ex(l, "dinv"), n, n), Dinv, tol, f"D^-1 level {l}")
        T = np.zeros((7 * n, 7 * n_next))
        Tb = ex(l, "t")
        for v in range(n):
            if agg[v] >= 0:
                T[7 * v:7 * v + 7, 7 * agg[v]:7 * agg[v] + 7] = Tb[v]
        P = dense(ex(l, "p_ptr"), ex(l, "p_col"), ex(l, "p"), n, n_next)
        close(P, T - (4.0 / (3.0 * rho)) * Dinv @ (A @ T), tol, f"P level {l}")
        AP = A @ P
        Q = dense(ex(l, "ap_ptr"), ex(l, "ap_col"), ex(l, "q"), n, n_next)
        close(Q, P - (1.0 / rho) * Dinv @ AP, tol, f"Q level {l}")
        A_next = dense(ex(l + 1, "a_ptr"), ex(l + 1, "a_col"), ex(l + 1, "a"), n_next, n_next)
        close(A_next, P.T @ AP, tol, f"A level {l + 1}")
        if l == Lc - 1:
            W = ex(l, "w").reshape(n, n, 7, 7).transpose(0, 2, 1, 3).reshape(7 * n, 7 * n)
            close(W, Q @ np.linalg.solve(A_next, Q.T), 1e-10 if precision == "fp64" else 2e-4, "W")
        A, n = A_next, n_next


def test_export_rejects_what_a_level_does_not_have():
    from paper_2603_17201_gb300 import PGOError, PoseGraph
    g = syn.make_graph("figure8", 120, seed=3, window=5, n_loops=1)
    pg = PoseGraph.from_synthetic(g)
    pg.linearize("fp64", jacobians=False)
    with pytest.raises(PGOError) as ei:   # no set-up yet in this precision
        pg.multigrid_export(0, "p", "fp64")
    assert ei.value.status == 6
    pg.precondition_async(1.0, precision="fp64")
    torch.cuda.synchronize()
    Lc = len(pg.multigrid_info()) - 1
    with pytest.raises(PGOError):          # level 0 has no Galerkin operator
        pg.multigrid_export(0, "a", "fp64")
    with pytest.raises(PGOError):          # the coarsest level has no prolongation
        pg.multigrid_export(Lc, "p", "fp64")
    with pytest.raises(PGOError):          # the FP32 set-up has not run
        pg.multigrid_export(0, "p", "mixed")
