"""Pins of the oracle's graph-level arithmetic (residuals, Jacobians, normal
equations, exact solve, LM, adjoint) against facts fixed by the mathematics:
finite differences, zero-cost consistent graphs, gauge invariance, the
closed-form scale-only ring, dense/scipy solves and brute-force finite
differences of the whole solve.  The problem is the pose graph optimisation
of the essential graph (Sec. III-B, Sec. IV-F)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from paper_2603_17201_gb300 import synthetic as syn

RNG = np.random.default_rng(777)


def small_graph(n=24, window=3, meas_noise=True, seed=5, n_loops=1):
    """A small figure-8-like graph with a loop (first lap revisited)."""
    g = syn.make_graph("circle", n, seed=seed, n_loops=n_loops, meas_noise=meas_noise)
    return g


def consistent_meas(g, poses):
    return syn.compose(poses[g.edge_j], syn.inverse(poses[g.edge_i]))


def test_residual_matches_definition(oracle_mod):
    g = syn.make_config("c1_circle200")
    og = O.OracleGraph.from_synthetic(g)
    F, r = og.cost(g.poses_init, residuals=True)
    for e in RNG.choice(g.n_edges, 20, replace=False).tolist() + [g.n_edges - 1]:
        i, j = g.edge_i[e], g.edge_j[e]
        T = syn.compose(g.meas[e], syn.compose(g.poses_init[i], syn.inverse(g.poses_init[j])))
        assert np.allclose(O.exp(r[e]), T * np.sign(np.dot(O.exp(r[e])[:4], T[:4])), atol=1e-13)
    assert np.isclose(F, np.sum(r * r), rtol=1e-15)
    # tree / covisibility edges are consistent with the drifted estimate
    assert np.abs(r[:-1]).max() < 1e-12
    assert np.abs(r[-1]).max() > 0.05


@pytest.mark.parametrize("cfg", ["c1_circle200", "noisy"])
def test_edge_jacobians_fd(oracle_mod, cfg):
    if cfg == "noisy":
        g = small_graph(40, meas_noise=True)
    else:
        g = syn.make_config(cfg)
    og = O.OracleGraph.from_synthetic(g)
    Ai, Aj = og.jacobians(g.poses_init)
    h = 1e-6
    edges = list(RNG.choice(g.n_edges, 8, replace=False)) + [g.n_edges - 1]
    for e in edges:
        i, j = g.edge_i[e], g.edge_j[e]
        for v, A in ((i, Ai[e]), (j, Aj[e])):
            num = np.zeros((7, 7))
            for k in range(7):
                d = np.zeros(7)
                d[k] = h
                pp = g.poses_init.copy()
                pm = g.poses_init.copy()
                pp[v] = syn.compose(O.exp(d), pp[v])
                pm[v] = syn.compose(O.exp(-d), pm[v])
                rp = og.cost(pp, residuals=True)[1][e]
                rm = og.cost(pm, residuals=True)[1][e]
                num[:, k] = (rp - rm) / (2 * h)
            err = np.abs(num - A).max() / max(1.0, np.abs(A).max())
            assert err < 1e-7, (e, err)


def test_normal_equations_from_jacobians(oracle_mod):
    g = small_graph(30, meas_noise=True)
    og = O.OracleGraph.from_synthetic(g)
    F, Hd, Ho, b = og.linearize(g.poses_init)
    Ai, Aj = og.jacobians(g.poses_init)
    _, r = og.cost(g.poses_init, residuals=True)
    # dense Jacobian of the stacked residual vector
    J = np.zeros((7 * g.n_edges, 7 * g.n_vertices))
    for e in range(g.n_edges):
        J[7 * e:7 * e + 7, 7 * g.edge_i[e]:7 * g.edge_i[e] + 7] += Ai[e]
        J[7 * e:7 * e + 7, 7 * g.edge_j[e]:7 * g.edge_j[e] + 7] += Aj[e]
    H = J.T @ J
    bb = J.T @ r.reshape(-1)
    for v in range(g.n_vertices):
        assert np.allclose(Hd[v], H[7 * v:7 * v + 7, 7 * v:7 * v + 7], atol=1e-12)
    for e in range(g.n_edges):
        i, j = g.edge_i[e], g.edge_j[e]
        assert np.allclose(Ho[e], Ai[e].T @ Aj[e], atol=1e-12)
    assert np.allclose(b.reshape(-1), bb, atol=1e-12)
    assert np.isclose(F, r.ravel() @ r.ravel())


def dense_system(g, Hd, Ho, lam):
    N = g.n_vertices
    H = np.zeros((7 * N, 7 * N))
    for v in range(N):
        H[7 * v:7 * v + 7, 7 * v:7 * v + 7] += Hd[v] + lam * np.eye(7)
    for e in range(g.n_edges):
        i, j = g.edge_i[e], g.edge_j[e]
        H[7 * i:7 * i + 7, 7 * j:7 * j + 7] += Ho[e]
        H[7 * j:7 * j + 7, 7 * i:7 * i + 7] += Ho[e].T
    keep = np.ones(7 * N, bool)
    keep[7 * g.fixed_vertex:7 * g.fixed_vertex + 7] = False
    return H, keep


@pytest.mark.parametrize("cfg", ["c1_circle200", "noisy"])
def test_exact_solve_vs_dense_and_scipy(oracle_mod, cfg):
    g = syn.make_config(cfg) if cfg != "noisy" else small_graph(60, meas_noise=True)
    og = O.OracleGraph.from_synthetic(g)
    _, Hd, Ho, b = og.linearize(g.poses_init)
    lam = 1e-3
    d = og.solve_system(Hd, Ho, b, lam)
    H, keep = dense_system(g, Hd, Ho, lam)
    ref = np.linalg.solve(H[np.ix_(keep, keep)], -b.reshape(-1)[keep])
    assert np.abs(d.reshape(-1)[keep] - ref).max() < 1e-9 * np.abs(ref).max()
    assert np.abs(d[g.fixed_vertex]).max() == 0.0
    ref2 = spla.spsolve(sp.csc_matrix(H[np.ix_(keep, keep)]), -b.reshape(-1)[keep])
    assert np.abs(d.reshape(-1)[keep] - ref2).max() < 1e-9 * np.abs(ref2).max()


def test_consistent_graph_converges_to_zero_cost(oracle_mod):
    """All measurements from the ground truth: LM from the drifted estimate
    reaches zero cost and the ground truth (vertex 0 is exact and fixed)."""
    g = syn.make_config("c1_circle200")
    meas = consistent_meas(g, g.poses_gt)
    og = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, meas, None, None, 0)
    assert og.cost(g.poses_init) > 1.0
    p, rep = og.lm(g.poses_init, max_iters=50)
    assert rep["final_cost"] < 1e-20
    err = O.pose_error(p, g.poses_gt)
    assert err.max() < 1e-9


def test_tree_graph_reaches_zero_cost(oracle_mod):
    """An acyclic graph can always satisfy every measurement exactly."""
    g = small_graph(50, meas_noise=True)
    tree = (g.edge_j - g.edge_i) == 1
    og = O.OracleGraph(g.n_vertices, g.edge_i[tree], g.edge_j[tree], g.meas[tree], None, None, 0)
    init = g.poses_init.copy()
    init[1:, 4:7] += RNG.normal(size=(g.n_vertices - 1, 3)) * 0.3
    p, rep = og.lm(init, max_iters=50)
    assert rep["final_cost"] < 1e-20


def test_gauge_invariance(oracle_mod):
    """Right-multiplying every pose by G^-1 leaves every residual, and hence
    the final cost, unchanged."""
    g = syn.make_config("c1_circle200")
    og = O.OracleGraph.from_synthetic(g)
    _, rep0 = og.lm(g.poses_init, max_iters=20)
    q = RNG.normal(size=4)
    q /= np.linalg.norm(q)
    G = np.concatenate([q, RNG.normal(size=3) * 3, [1.7]])
    moved = syn.compose(g.poses_init, np.broadcast_to(syn.inverse(G), g.poses_init.shape))
    assert np.isclose(og.cost(moved), og.cost(g.poses_init), rtol=1e-12)
    _, rep1 = og.lm(moved, max_iters=20)
    assert abs(rep1["final_cost"] - rep0["final_cost"]) <= 1e-12 * rep0["final_cost"]


def scale_ring(n, seed=3, weights=None):
    """Ring of n vertices with identity rotations, zero translations and
    scale-only measurements; edges k -> k+1 and the loop n-1 -> 0."""
    rng = np.random.default_rng(seed)
    sz = rng.normal(0, 0.05, size=n)
    ei = np.arange(n, dtype=np.int32)
    ej = ((np.arange(n) + 1) % n).astype(np.int32)
    meas = np.zeros((n, 8))
    meas[:, 3] = 1.0
    meas[:, 7] = np.exp(sz)
    poses = np.zeros((n, 8))
    poses[:, 3] = 1.0
    poses[:, 7] = 1.0
    return ei, ej, meas, poses, sz


def test_scale_ring_closed_form(oracle_mod):
    """Residual r_k = sigma_Z,k + sigma_k - sigma_{k+1} is linear in the log
    scales and the rotation/translation gradient vanishes, so the optimum has
    every residual equal to c/n (c = sum of measured log scales) and cost
    c^2 / n."""
    n = 17
    ei, ej, meas, poses, sz = scale_ring(n)
    og = O.OracleGraph(n, ei, ej, meas, None, None, 0)
    p, rep = og.lm(poses, max_iters=30)
    c = sz.sum()
    assert abs(rep["final_cost"] - c * c / n) < 1e-14
    # cost-based stopping resolves the optimum to sqrt(eps); polishing
    # (undamped Newton steps kept while |b| drops) pins the stationary point
    p, rep = og.lm(poses, max_iters=30, polish_iters=5)
    _, r = og.cost(p, residuals=True)
    assert np.abs(r[:, 6] - c / n).max() < 1e-12
    assert np.abs(r[:, :6]).max() < 1e-13
    sig = np.log(p[:, 7])
    ref = np.concatenate([[0.0], np.cumsum(sz[:-1] - c / n)])
    assert np.abs(sig - ref).max() < 1e-12


def test_scale_ring_adjoint_closed_form(oracle_mod):
    """Closed-form sensitivities of L = 1/2 sum sigma_v^2 (ground truth
    s = 1) for the scale-only ring, against the oracle's implicit adjoint."""
    n = 9
    ei, ej, meas, poses, sz = scale_ring(n, seed=11)
    og = O.OracleGraph(n, ei, ej, meas, None, None, 0)
    p, _ = og.lm(poses, max_iters=50, ftol=0.0, polish_iters=5)
    gt = poses.copy()
    L, dLdx = og.pose_loss(p, gt)
    dz, dw, _ = og.adjoint(p, dLdx)
    c = sz.sum()
    v = np.arange(n)
    sig = np.concatenate([[0.0], np.cumsum(sz[:-1] - c / n)])
    for m in range(n):
        ref_z = np.sum(sig * ((m < v).astype(float) - v / n))
        ref_w = np.sum(sig * (-(v * c / n ** 2 - (m < v) * c / n)))
        assert abs(dz[m, 6] - ref_z) < 1e-8
        assert np.abs(dz[m, :6]).max() < 1e-8
        assert abs(dw[m] - ref_w) < 1e-8


@pytest.mark.slow
def test_adjoint_brute_force(oracle_mod):
    """dL/dw and dL/dz of the converged solution against central differences
    of the whole LM solve (tiny noisy graph)."""
    g = small_graph(14, meas_noise=True, seed=21)
    base = dict(max_iters=200, ftol=0.0, gtol=1e-15, polish_iters=10)

    def solve(meas, w):
        og = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, meas, w, None, 0)
        p, _ = og.lm(g.poses_init, **base)
        return og, p

    og, p = solve(g.meas, g.weight)
    L, dLdx = og.pose_loss(p, g.poses_gt)
    dz, dw, _ = og.adjoint(p, dLdx)
    hw, hz = 1e-5, 1e-5
    for e in RNG.choice(g.n_edges, 6, replace=False):
        w = g.weight.copy()
        w[e] += hw
        ogp, pp = solve(g.meas, w)
        Lp = ogp.pose_loss(pp, g.poses_gt)[0]
        w[e] -= 2 * hw
        ogm, pm = solve(g.meas, w)
        Lm = ogm.pose_loss(pm, g.poses_gt)[0]
        fd_w = (Lp - Lm) / (2 * hw)
        assert abs(fd_w - dw[e]) <= 1e-5 * max(abs(fd_w), 1e-3 * np.abs(dw).max())
        fd_z = np.zeros(7)
        for k in range(7):
            d = np.zeros(7)
            d[k] = hz
            mp = g.meas.copy()
            mm = g.meas.copy()
            mp[e] = syn.compose(O.exp(d), mp[e])
            mm[e] = syn.compose(O.exp(-d), mm[e])
            ogp, pp = solve(mp, g.weight)
            ogm, pm = solve(mm, g.weight)
            fd_z[k] = (ogp.pose_loss(pp, g.poses_gt)[0] - ogm.pose_loss(pm, g.poses_gt)[0]) / (2 * hz)
        assert np.linalg.norm(fd_z - dz[e]) <= 1e-5 * max(np.linalg.norm(fd_z), 1e-3 * np.abs(dz).max())


def test_lm_single_step_rules(oracle_mod):
    """One LM iteration equals: lambda_0 = tau max diag(H), exact damped
    solve, exp update, and the gain-ratio accept rule."""
    g = small_graph(40, meas_noise=True)
    og = O.OracleGraph.from_synthetic(g)
    F0, Hd, Ho, b = og.linearize(g.poses_init)
    lam = 1e-5 * max(np.diag(Hd[v]).max() for v in range(1, g.n_vertices))
    d = og.solve_system(Hd, Ho, b, lam)
    pn = og.apply_update(g.poses_init, d)
    F1 = og.cost(pn)
    pred = float(np.sum(d * (lam * d - b)))
    rho = (F0 - F1) / pred
    p, rep = og.lm(g.poses_init, max_iters=1)
    assert rep["iterations"] == 1
    if rho > 0:
        assert rep["accepted"] == 1
        assert np.isclose(rep["final_cost"], F1, rtol=1e-14)
        f = 1 - (2 * rho - 1) ** 3
        assert np.isclose(rep["final_lambda"], lam * max(1 / 3, f), rtol=1e-12)
    else:
        assert rep["accepted"] == 0
        assert np.isclose(rep["final_lambda"], 2 * lam, rtol=1e-12)
