"""The direct block Cholesky solve of the damped system (Sec. IV-F: an exact
factorisation, as the paper's LDL^T; Fig. 4: the solver's cost by problem
size) against the oracle's exact sparse Cholesky, through the C ABI.

  damped step, FP64         1e-10 relative to the largest entry (both exact
                            factorisations, different elimination orders);
  damped step, mixed        the FP32 factor inside FP64 refinement (6
                            passes): 1e-7, as the mixed PCG step;
  LM solves                 final cost 1e-9 (FP64) / 1e-6 (mixed), no PCG
                            iteration at all.
Graphs: the 200-keyframe circle (pure band: its loop edge ends at the fixed
vertex), small noisy figure-8 graphs whose loop edges make separators (one
with a gauge vertex in the middle, one with 7x7 information matrices and
weights), and the crossover setting AUTO.
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


def noisy(n=61, seed=7, info=False, weights=False, fixed=0, n_loops=2):
    g = syn.make_graph("figure8", n, seed=seed, window=4, n_loops=n_loops, meas_noise=True,
                       loop_min_gap=n // 3, loop_max_dist=4.0)
    g.fixed_vertex = fixed
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 2.0, g.n_edges) if weights else None
    I = None
    if info:
        M = rng.normal(size=(g.n_edges, 7, 7)) * 0.3
        I = np.einsum("eij,ekj->eik", M, M) + np.eye(7)[None] * 0.5
    return g, w, I


def case(name):
    if name == "c1":
        return syn.make_config("c1_circle200"), None, None
    if name == "noisy":
        return noisy()
    if name == "noisy_info_w":
        return noisy(info=True, weights=True)
    if name == "fixed_mid":
        return noisy(n=45, fixed=17)
    if name == "fig8_500":
        return syn.make_graph("figure8", 500, seed=9, window=12, n_loops=4, meas_noise=True), None, None
    raise KeyError(name)


def pair(g, w, I):
    from paper_2603_17201_gb300 import PoseGraph
    og = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, w, I, g.fixed_vertex)
    pg = PoseGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, w, I, g.poses_init, g.fixed_vertex)
    return og, pg


NAMES = ["c1", "noisy", "noisy_info_w", "fixed_mid", "fig8_500"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", NAMES)
def test_direct_damped_step_matches_exact_solve(name, precision):
    g, w, I = case(name)
    og, pg = pair(g, w, I)
    _, Hd, Ho, b = og.linearize(g.poses_init)
    lam = 1e-4 * max(np.diag(Hd[v]).max() for v in range(g.n_vertices))
    if precision == "mixed":
        lin = pg.linearize("mixed", jacobians=False)
        Hd, Ho, b = lin["h_diag"], lin["h_off"], lin["b"]
    ref = og.solve_system(Hd, Ho, b, lam)
    d, its = pg.damped_step(lam, precision=precision, linear_solver="direct", refine_steps=6, pcg_tol=1e-12)
    assert its == 0
    tol = 1e-10 if precision == "fp64" else 1e-7
    assert np.abs(d - ref).max() <= tol * np.abs(ref).max(), np.abs(d - ref).max() / np.abs(ref).max()
    assert np.abs(d[g.fixed_vertex]).max() == 0.0
    # a re-solve at another lambda refactors
    d2, _ = pg.resolve(10 * lam, precision=precision, linear_solver="direct", refine_steps=6, pcg_tol=1e-12)
    ref2 = og.solve_system(Hd, Ho, b, 10 * lam)
    assert np.abs(d2 - ref2).max() <= tol * np.abs(ref2).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
@pytest.mark.parametrize("name", NAMES)
def test_direct_lm_solve_matches_oracle(name, precision, tol, parity_record):
    g, w, I = case(name)
    og, pg = pair(g, w, I)
    p_ref, ref = og.lm(g.poses_init, max_iters=20)
    rep = pg.solve(max_iters=20, precision=precision, linear_solver="direct")
    assert rep["status"] == 0 and rep["pcg_iterations"] == 0
    rel = abs(rep["final_cost"] - ref["final_cost"]) / ref["final_cost"]
    pe = O.pose_error(pg.get_poses(), p_ref)
    parity_record(f"direct {name} {precision}", rel, pe)
    assert rel <= tol, (rep, ref)


def test_auto_follows_the_measured_crossover():
    """AUTO picks DIRECT only up to PGO_DIRECT_CROSSOVER_VERTICES keyframes
    (0 on GB300, where the multigrid PCG was faster at every measured size)."""
    g, w, I = case("noisy")
    _, pg = pair(g, w, I)
    rep = pg.solve(max_iters=5, linear_solver="auto")
    assert rep["status"] == 0 and rep["pcg_iterations"] > 0
    assert pg.solve(max_iters=5, linear_solver="direct")["pcg_iterations"] == 0


def test_direct_rejects_graphs_beyond_its_limits():
    from paper_2603_17201_gb300 import PGOError, PoseGraph
    # 20 loop edges: more separators than the direct solver takes
    g = syn.make_graph("figure8", 400, seed=4, window=6, n_loops=20, loop_min_gap=60, loop_max_dist=6.0)
    assert g.n_loop_edges > 9
    pg = PoseGraph.from_synthetic(g)
    with pytest.raises(PGOError) as ei:
        pg.solve(max_iters=3, linear_solver="direct")
    assert ei.value.status == 1
    rep = pg.solve(max_iters=3, linear_solver="auto")   # falls back to PCG
    assert rep["status"] == 0 and rep["pcg_iterations"] > 0
