"""Multigrid preconditioner of the damped solve (Sec. IV-F's normal
equations): the same step as the oracle's exact sparse Cholesky at the full
sizes of the drone-flight (2k keyframes) and long handheld (8k keyframes)
graphs, far fewer PCG iterations than block-Jacobi, and correct on the
degenerate sizes of the hierarchy (one free vertex, fewer free vertices than
one aggregate, a ragged last aggregate, the gauge vertex inside an
aggregate).

Tolerance: 1e-7 relative to the largest step component, with PCG at 1e-12
(FP64) or FP32 PCG inside six FP64 refinement passes (mixed).
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


def pair(g, fixed=None):
    from paper_2603_17201_gb300 import PoseGraph
    f = g.fixed_vertex if fixed is None else fixed
    og = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, None, None, f)
    pg = PoseGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, None, None, g.poses_init, f)
    return og, pg


def exact_step(og, poses, lam_rel):
    _, Hd, Ho, b = og.linearize(poses)
    lam = lam_rel * max(np.diag(Hd[v]).max() for v in range(Hd.shape[0]))
    return og.solve_system(Hd, Ho, b, lam), lam


def rel(d, ref):
    return np.abs(d - ref).max() / max(np.abs(ref).max(), 1e-300)


def mixed_exact_step(og, pg, lam):
    """The mixed mode solves its own FP32-Jacobian normal equations: the exact
    solve of exactly that system."""
    lin = pg.linearize("mixed", jacobians=False)
    return og.solve_system(lin["h_diag"], lin["h_off"], lin["b"], lam)


@pytest.mark.parametrize("name", ["c2_figure8_2k", "c3_corridor_8k"])
def test_full_size_step_matches_exact_solve(name):
    g = syn.make_config(name)
    og, pg = pair(g)
    ref, lam = exact_step(og, g.poses_init, 1e-6)
    d, its = pg.damped_step(lam, precision="fp64", pcg_tol=1e-12, preconditioner="multigrid")
    assert rel(d, ref) <= 1e-7, rel(d, ref)
    assert its <= 80, its
    dm, _ = pg.damped_step(lam, precision="mixed", pcg_tol=1e-12, refine_steps=6, preconditioner="multigrid")
    refm = mixed_exact_step(og, pg, lam)
    assert rel(dm, refm) <= 1e-7, rel(dm, refm)
    print(f"{name}: multigrid FP64 PCG iterations {its}, rel err {rel(d, ref):.1e} (mixed {rel(dm, refm):.1e})")


def test_far_fewer_iterations_than_block_jacobi():
    g = syn.make_config("c2_figure8_2k")
    og, pg = pair(g)
    ref, lam = exact_step(og, g.poses_init, 1e-6)
    d_bj, its_bj = pg.damped_step(lam, precision="fp64", pcg_tol=1e-10, pcg_max_iters=20000,
                                  preconditioner="block_jacobi")
    d_mg, its_mg = pg.damped_step(lam, precision="fp64", pcg_tol=1e-10, preconditioner="multigrid")
    assert rel(d_bj, ref) <= 1e-6 and rel(d_mg, ref) <= 1e-6
    assert 20 * its_mg <= its_bj, (its_mg, its_bj)


@pytest.mark.parametrize("n,fixed", [(2, 0), (2, 1), (3, 1), (5, 0), (5, 4), (9, 0), (10, 3), (34, 0), (34, 17),
                                     (200, 101)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_degenerate_hierarchy_sizes(n, fixed, precision):
    g = syn.make_graph("circle", n, seed=n, window=3, n_loops=1 if n > 6 else 0, loop_min_gap=max(2, n // 2),
                       loop_max_dist=100.0, meas_noise=True)
    og, pg = pair(g, fixed)
    ref, lam = exact_step(og, g.poses_init, 1e-5)
    if precision == "mixed":
        ref = mixed_exact_step(og, pg, lam)
    d, its = pg.damped_step(lam, precision=precision, pcg_tol=1e-12, refine_steps=6, preconditioner="multigrid")
    assert rel(d, ref) <= 1e-7, (rel(d, ref), its)
    assert np.abs(d[fixed]).max() == 0.0


def test_lm_and_resolve_with_both_preconditioners_agree():
    g = syn.make_graph("figure8", 300, seed=12, window=8, n_loops=2, meas_noise=True, loop_min_gap=100,
                       loop_max_dist=3.0)
    og, pg = pair(g)
    p_ref, rep_ref = og.lm(g.poses_init, max_iters=20)
    out = {}
    for pc in ["block_jacobi", "multigrid"]:
        pg.set_poses(g.poses_init)
        # exact LM steps, so that both solves end at the same linearisation
        # for the re-solves below (the default LM tolerance of 1e-6 reaches
        # the same optimum by slightly different last iterates)
        rep = pg.solve(max_iters=20, preconditioner=pc, pcg_tol=1e-10)
        assert abs(rep["final_cost"] - rep_ref["final_cost"]) <= 1e-9 * rep_ref["final_cost"], (pc, rep, rep_ref)
        assert O.pose_error(pg.get_poses(), p_ref).max() < 1e-5
        out[pc] = rep["pcg_iterations"]
        # a re-solve at the last linearisation for another lambda
        d, _ = pg.resolve(1e-3, preconditioner=pc, pcg_tol=1e-13, pcg_max_iters=20000)
        out[pc + "_resolve"] = d
    assert rel(out["multigrid_resolve"], out["block_jacobi_resolve"]) <= 1e-6
    assert out["multigrid"] < out["block_jacobi"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lagged_coarse_levels_reach_the_same_optimum(precision):
    """multigrid_refresh > 1 keeps the coarse levels of the last complete
    set-up between rebuilds: a different (still symmetric positive definite)
    preconditioner, the same LM optimum."""
    g = syn.make_graph("figure8", 400, seed=31, window=10, n_loops=2, meas_noise=True, loop_min_gap=150,
                       loop_max_dist=3.0)
    og, pg = pair(g)
    _, ref = og.lm(g.poses_init, max_iters=20)
    for refresh in (1, 3):
        pg.set_poses(g.poses_init)
        rep = pg.solve(max_iters=20, precision=precision, multigrid_refresh=refresh)
        tol = 1e-9 if precision == "fp64" else 1e-6
        assert abs(rep["final_cost"] - ref["final_cost"]) <= tol * ref["final_cost"], (refresh, rep, ref)
