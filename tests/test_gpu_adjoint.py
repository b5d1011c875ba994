"""GPU implicit adjoint against the oracle's adjoint, closed forms and
brute-force finite differences of the whole solve, through the C ABI and the
torch.autograd.Function.

Tolerances: GPU vs oracle adjoint 1e-6 relative to the largest gradient (the
oracle takes its second derivatives by central differences, the GPU by exact
nested duals); against finite differences of the solve 1e-5 relative, per
edge on vector norms with a floor of 1e-3 x the largest gradient."""
import numpy as np
import pytest

import oracle as O
from paper_2603_17201_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

POLISH = dict(max_iters=60, polish_iters=10, gtol=1e-15, pcg_tol=1e-12, pcg_max_iters=20000)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def PG(*a, **k):
    from paper_2603_17201_gb300 import PoseGraph
    return PoseGraph(*a, **k)


def small(n=40, seed=21, info=False):
    g = syn.make_graph("figure8", n, seed=seed, window=4, n_loops=2, meas_noise=True,
                       loop_min_gap=n // 3, loop_max_dist=4.0)
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 2.0, g.n_edges)
    I = None
    if info:
        M = rng.normal(size=(g.n_edges, 7, 7)) * 0.3
        I = np.einsum("eij,ekj->eik", M, M) + np.eye(7)[None] * 0.5
    return g, w, I


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("info", [False, True])
def test_adjoint_matches_oracle(info):
    g, w, I = small(info=info)
    og = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, w, I, 0)
    p_ref, _ = og.lm(g.poses_init, max_iters=60, ftol=0.0, gtol=1e-15, polish_iters=10)
    _, dLdx_ref = og.pose_loss(p_ref, g.poses_gt)
    dz_ref, dw_ref, _ = og.adjoint(p_ref, dLdx_ref)
    pg = PG(g.n_vertices, g.edge_i, g.edge_j, g.meas, w, I, g.poses_init, 0)
    rep = pg.solve(**POLISH)
    assert rep["grad_inf_norm"] < 1e-10, rep
    p = pg.get_poses()
    assert O.pose_error(p, p_ref).max() < 1e-9
    _, dLdx = og.pose_loss(p, g.poses_gt)
    dz, dw = pg.backward(dLdx, layout="tangent")
    assert rel_err(dw, dw_ref) < 1e-6, rel_err(dw, dw_ref)
    assert rel_err(dz, dz_ref) < 1e-6, rel_err(dz, dz_ref)


def test_adjoint_scale_ring_closed_form():
    """Scale-only ring: sensitivities of L = 1/2 sum sigma_v^2 in closed form
    (residuals at the optimum all equal c/n)."""
    n = 9
    rng = np.random.default_rng(11)
    sz = rng.normal(0, 0.05, size=n)
    ei = np.arange(n, dtype=np.int32)
    ej = ((np.arange(n) + 1) % n).astype(np.int32)
    meas = np.zeros((n, 8))
    meas[:, 3] = 1.0
    meas[:, 7] = np.exp(sz)
    poses = np.zeros((n, 8))
    poses[:, 3] = 1.0
    poses[:, 7] = 1.0
    pg = PG(n, ei, ej, meas, None, None, poses, 0)
    pg.solve(**POLISH)
    p = pg.get_poses()
    sig = np.log(p[:, 7])
    c = sz.sum()
    v = np.arange(n)
    assert np.abs(sig - np.concatenate([[0.0], np.cumsum(sz[:-1] - c / n)])).max() < 1e-12
    dLdx = np.zeros((n, 7))
    dLdx[:, 6] = sig                         # L = 1/2 sum sigma^2, left tangent
    dz, dw = pg.backward(dLdx, layout="tangent")
    for m in range(n):
        ref_z = np.sum(sig * ((m < v).astype(float) - v / n))
        ref_w = np.sum(sig * (-(v * c / n ** 2 - (m < v) * c / n)))
        assert abs(dz[m, 6] - ref_z) < 1e-10
        assert np.abs(dz[m, :6]).max() < 1e-10
        assert abs(dw[m] - ref_w) < 1e-10


def _loss(pg, g):
    L, _ = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, None, None, 0).pose_loss(
        pg.get_poses(), g.poses_gt)
    return L


def test_adjoint_against_finite_differences_of_the_solve():
    g, w, _ = small(n=30, seed=5)
    pg = PG(g.n_vertices, g.edge_i, g.edge_j, g.meas, w, None, g.poses_init, 0)
    pg.solve(**POLISH)
    p_star = pg.get_poses()
    og = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, None, None, 0)
    _, dLdx = og.pose_loss(p_star, g.poses_gt)
    dz, dw = pg.backward(dLdx, layout="tangent")
    rng = np.random.default_rng(3)

    def solve_loss(meas, weight):
        pg.set_measurements(meas, weight)
        pg.set_poses(p_star)
        pg.solve(**POLISH)
        return og.pose_loss(pg.get_poses(), g.poses_gt)[0]

    for e in rng.choice(g.n_edges, 5, replace=False):
        h = 1e-5
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd_w = (solve_loss(g.meas, wp) - solve_loss(g.meas, wm)) / (2 * h)
        assert abs(fd_w - dw[e]) <= 1e-5 * max(abs(fd_w), 1e-3 * np.abs(dw).max()), (e, fd_w, dw[e])
        fd_z = np.zeros(7)
        for k in range(7):
            d = np.zeros(7)
            d[k] = h
            mp, mm = g.meas.copy(), g.meas.copy()
            mp[e] = syn.compose(O.exp(d), mp[e])
            mm[e] = syn.compose(O.exp(-d), mm[e])
            fd_z[k] = (solve_loss(mp, w) - solve_loss(mm, w)) / (2 * h)
        assert np.linalg.norm(fd_z - dz[e]) <= 1e-5 * max(np.linalg.norm(fd_z), 1e-3 * np.abs(dz).max()), \
            (e, fd_z, dz[e])


def test_autograd_function_pose8_layout():
    """Gradients w.r.t. the pose8 measurement entries and the weights through
    torch.autograd, against central differences of a torch loss."""
    from paper_2603_17201_gb300 import solve_pose_graph
    g, w, _ = small(n=24, seed=9)
    dev = torch.device("cuda", 0)
    pg = PG(g.n_vertices, g.edge_i, g.edge_j, g.meas, w, None, g.poses_init, 0)
    meas = torch.tensor(g.meas, dtype=torch.float64, device=dev, requires_grad=True)
    wt = torch.tensor(w, dtype=torch.float64, device=dev, requires_grad=True)
    p0 = torch.tensor(g.poses_init, dtype=torch.float64, device=dev)
    gt = torch.tensor(g.poses_gt, dtype=torch.float64, device=dev)

    def loss_of(poses):
        # translation and log-scale error plus a quaternion alignment term
        dq = (poses[:, :4] * gt[:, :4]).sum(1)
        return ((poses[:, 4:7] - gt[:, 4:7]) ** 2).sum() + (torch.log(poses[:, 7]) ** 2).sum() \
            + (1.0 - dq ** 2).sum()

    out = solve_pose_graph(pg, meas, wt, p0, **POLISH)
    L = loss_of(out)
    L.backward()
    gm, gw = meas.grad.cpu().numpy(), wt.grad.cpu().numpy()
    rng = np.random.default_rng(4)
    with torch.no_grad():
        def L_at(mv, wv):
            return loss_of(solve_pose_graph(pg, mv, wv, p0, **POLISH)).item()
        for e in rng.choice(g.n_edges, 3, replace=False):
            h = 1e-5
            wp, wm = wt.detach().clone(), wt.detach().clone()
            wp[e] += h
            wm[e] -= h
            fd = (L_at(meas.detach(), wp) - L_at(meas.detach(), wm)) / (2 * h)
            assert abs(fd - gw[e]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gw).max()), (fd, gw[e])
            fdm = np.zeros(8)
            for k in range(8):
                mp, mm = meas.detach().clone(), meas.detach().clone()
                mp[e, k] += h
                mm[e, k] -= h
                fdm[k] = (L_at(mp, wt.detach()) - L_at(mm, wt.detach())) / (2 * h)
            assert np.linalg.norm(fdm - gm[e]) <= 1e-5 * max(np.linalg.norm(fdm), 1e-3 * np.abs(gm).max()), \
                (fdm, gm[e])


@pytest.mark.slow
def test_c5_adjoint_4k_against_fd_and_oracle():
    """The differentiation workload: the 4,000-keyframe noisy figure-8 graph
    (67,857 edges, weights 1.0), FP64 forward to convergence, gradients of the
    final pose-error loss w.r.t. every measurement (left tangent) and weight.
    Checked against the oracle's adjoint at the same optimum (1e-6 relative to
    the largest gradient) and against central differences of the whole solve
    (step 1e-4) on 64 random edges (1e-5, per edge on vector norms, floor 1e-3
    of the largest gradient)."""
    g = syn.make_config("c5_figure8_4k_noisy")
    w = np.ones(g.n_edges)
    pg = PG(g.n_vertices, g.edge_i, g.edge_j, g.meas, w, None, g.poses_init, 0)
    rep = pg.solve(**POLISH)
    assert rep["status"] == 0 and rep["grad_inf_norm"] < 1e-9, rep
    p_star = pg.get_poses()
    og = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, None, None, 0)
    _, dLdx = og.pose_loss(p_star, g.poses_gt)
    dz, dw = pg.backward(dLdx, layout="tangent")
    dz_ref, dw_ref, _ = og.adjoint(p_star, dLdx)
    assert rel_err(dw, dw_ref) < 1e-6, rel_err(dw, dw_ref)
    assert rel_err(dz, dz_ref) < 1e-6, rel_err(dz, dz_ref)

    def solve_loss(meas, weight):
        pg.set_measurements(meas, weight)
        pg.set_poses(p_star)
        pg.solve(**POLISH)
        return og.pose_loss(pg.get_poses(), g.poses_gt)[0]

    # step 1e-4: the loss of a converged 4k-keyframe solve carries ~1e-10 of
    # rounding, which a 1e-5 step would amplify past the bar; the central
    # difference's truncation error at 1e-4 is ~1e-8 relative
    rng = np.random.default_rng(64)
    h = 1e-4
    gz, gw = np.abs(dz).max(), np.abs(dw).max()
    for e in rng.choice(g.n_edges, 64, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd_w = (solve_loss(g.meas, wp) - solve_loss(g.meas, wm)) / (2 * h)
        assert abs(fd_w - dw[e]) <= 1e-5 * max(abs(fd_w), 1e-3 * gw), (e, fd_w, dw[e])
        fd_z = np.zeros(7)
        for k in range(7):
            d = np.zeros(7)
            d[k] = h
            mp, mm = g.meas.copy(), g.meas.copy()
            mp[e] = syn.compose(O.exp(d), mp[e])
            mm[e] = syn.compose(O.exp(-d), mm[e])
            fd_z[k] = (solve_loss(mp, w) - solve_loss(mm, w)) / (2 * h)
        assert np.linalg.norm(fd_z - dz[e]) <= 1e-5 * max(np.linalg.norm(fd_z), 1e-3 * gz), (e, fd_z, dz[e])
