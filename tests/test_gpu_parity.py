"""GPU parity of every step of the hot path against the FP64 oracle, through
the C ABI (Sec. IV-F: residuals, exact Jacobians, normal equations, damped
linear solve, LM update; Sec. VI: the LM scheme).

Tolerances (stated here, derived in the design notes):
  residuals / cost      1e-12 absolute / 1e-13 relative (same FP64 formula,
                        different rounding order);
  Jacobians, H, b       1e-10 relative to the block's max (FP64 duals vs the
                        oracle's series + Gaussian elimination);
  damped step (PCG)     1e-7 relative (PCG tolerance 1e-12);
  LM final cost         1e-9 relative in FP64, 1e-6 in mixed precision;
  poses                 reported as per-vertex |log(S_gpu S_oracle^-1)|.
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
    from paper_2603_17201_gb300 import _lib
    _lib.load()
    torch.cuda.set_device(0)


def PG(*a, **k):
    from paper_2603_17201_gb300 import PoseGraph
    return PoseGraph(*a, **k)


def noisy_small(n=61, seed=7, info=False, weights=False, fixed=0):
    g = syn.make_graph("figure8", n, seed=seed, window=4, n_loops=2, meas_noise=True,
                       loop_min_gap=n // 3, loop_max_dist=4.0)
    g.fixed_vertex = fixed
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 2.0, g.n_edges) if weights else None
    I = None
    if info:
        M = rng.normal(size=(g.n_edges, 7, 7)) * 0.3
        I = np.einsum("eij,ekj->eik", M, M) + np.eye(7)[None] * 0.5
    return g, w, I


def make_pair(g, w=None, info=None, poses=None):
    p = g.poses_init if poses is None else poses
    og = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, w, info, g.fixed_vertex)
    pg = PG(g.n_vertices, g.edge_i, g.edge_j, g.meas, w, info, p, g.fixed_vertex)
    return og, pg


CASES = ["c1", "noisy", "noisy_info_w", "fixed_mid"]


def case_graph(name):
    if name == "c1":
        g = syn.make_config("c1_circle200")
        return g, None, None
    if name == "noisy":
        return noisy_small()
    if name == "noisy_info_w":
        return noisy_small(info=True, weights=True)
    if name == "fixed_mid":
        return noisy_small(n=45, fixed=17)
    raise KeyError(name)


@pytest.mark.parametrize("name", CASES)
def test_residuals_and_cost(name):
    g, w, I = case_graph(name)
    og, pg = make_pair(g, w, I)
    F_ref, r_ref = og.cost(g.poses_init, residuals=True)
    F, r = pg.cost(residuals=True)
    assert np.abs(r - r_ref).max() <= 1e-12 * max(1.0, np.abs(r_ref).max())
    assert abs(F - F_ref) <= 1e-13 * F_ref


@pytest.mark.parametrize("name", CASES)
def test_jacobians_and_normal_equations(name):
    g, w, I = case_graph(name)
    og, pg = make_pair(g, w, I)
    lin = pg.linearize("fp64")
    Ai, Aj = og.jacobians(g.poses_init)
    scale = max(np.abs(Ai).max(), np.abs(Aj).max())
    if I is None:  # the export is the unwhitened Jacobian only without info
        assert np.abs(lin["jac"][:, 0] - Ai).max() <= 1e-10 * scale
        assert np.abs(lin["jac"][:, 1] - Aj).max() <= 1e-10 * scale
    _, Hd, Ho, b = og.linearize(g.poses_init)
    for got, ref in ((lin["h_diag"], Hd), (lin["h_off"], Ho), (lin["b"], b)):
        assert np.abs(got - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("name", CASES)
def test_mixed_normal_equations(name):
    """Mixed precision: FP32 Jacobians and H products, FP64 residual and
    gradient sum; H within FP32 rounding of the FP64 oracle (1e-5 of the
    largest entry) and b likewise."""
    g, w, I = case_graph(name)
    og, pg = make_pair(g, w, I)
    lin = pg.linearize("mixed", jacobians=False)
    _, Hd, Ho, b = og.linearize(g.poses_init)
    for got, ref in ((lin["h_diag"], Hd), (lin["h_off"], Ho), (lin["b"], b)):
        err = np.abs(got - ref).max() / max(1.0, np.abs(ref).max())
        assert err <= 1e-5, err


@pytest.mark.parametrize("precond", ["block_jacobi", "multigrid"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["c1", "noisy_info_w"])
def test_damped_step(name, precision, precond):
    g, w, I = case_graph(name)
    og, pg = make_pair(g, w, I)
    _, Hd, Ho, b = og.linearize(g.poses_init)
    lam = 1e-4 * max(np.diag(Hd[v]).max() for v in range(g.n_vertices))
    if precision == "mixed":
        # the mixed mode solves its own FP32-Jacobian normal equations (bounded
        # against the FP64 ones in test_mixed_normal_equations): the exact
        # solve of exactly that system is the reference
        lin = pg.linearize("mixed", jacobians=False)
        Hd, Ho, b = lin["h_diag"], lin["h_off"], lin["b"]
    ref = og.solve_system(Hd, Ho, b, lam)
    d, its = pg.damped_step(lam, precision=precision, pcg_tol=1e-12, pcg_max_iters=20000, refine_steps=6,
                            preconditioner=precond)
    assert its > 0
    assert np.abs(d - ref).max() <= 1e-7 * np.abs(ref).max()
    assert np.abs(d[g.fixed_vertex]).max() == 0.0


def pose_err(a, b):
    return O.pose_error(a, b)


@pytest.mark.parametrize("precond", ["block_jacobi", "multigrid"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
@pytest.mark.parametrize("name", ["c1", "noisy", "noisy_info_w", "fixed_mid"])
def test_lm_solve_matches_oracle(name, precision, tol, precond):
    g, w, I = case_graph(name)
    og, pg = make_pair(g, w, I)
    p_ref, rep_ref = og.lm(g.poses_init, max_iters=20)
    rep = pg.solve(max_iters=20, precision=precision, preconditioner=precond)
    assert rep["status"] == 0
    assert abs(rep["initial_cost"] - rep_ref["initial_cost"]) <= 1e-13 * rep_ref["initial_cost"]
    rel = abs(rep["final_cost"] - rep_ref["final_cost"]) / rep_ref["final_cost"]
    assert rel <= tol, (rep, rep_ref)
    p = pg.get_poses()
    err = pose_err(p, p_ref)
    assert np.all(np.isfinite(err))
    assert err.max() < (1e-5 if precision == "fp64" else 1e-3), err.max()
    # the gauge vertex is untouched
    f = g.fixed_vertex
    q0 = g.poses_init[f, :4] / np.linalg.norm(g.poses_init[f, :4])
    assert np.abs(p[f, :4] - q0).max() < 1e-15 and np.array_equal(p[f, 4:], g.poses_init[f, 4:])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_lm_solve_c2_figure8(precision, tol):
    """The 2,000-keyframe figure-8 graph (~30k edges) at full size."""
    g = syn.make_config("c2_figure8_2k")
    og, pg = make_pair(g)
    p_ref, rep_ref = og.lm(g.poses_init, max_iters=20)
    rep = pg.solve(max_iters=20, precision=precision)
    rel = abs(rep["final_cost"] - rep_ref["final_cost"]) / rep_ref["final_cost"]
    assert rel <= tol, (rep, rep_ref)
    err = pose_err(pg.get_poses(), p_ref)
    print(f"c2 {precision}: rel cost {rel:.2e}, pose err max {err.max():.2e} rms {np.sqrt(np.mean(err**2)):.2e}, "
          f"iters {rep['iterations']} pcg {rep['pcg_iterations']} ms {rep['ms_total']:.1f}")


def test_consistent_graph_reaches_ground_truth():
    g = syn.make_config("c1_circle200")
    meas = syn.compose(g.poses_gt[g.edge_j], syn.inverse(g.poses_gt[g.edge_i]))
    pg = PG(g.n_vertices, g.edge_i, g.edge_j, meas, None, None, g.poses_init, 0)
    rep = pg.solve(max_iters=50)
    assert rep["final_cost"] < 1e-18
    assert pose_err(pg.get_poses(), g.poses_gt).max() < 1e-8


def test_edge_cases():
    # no edges: nothing to optimise, cost 0
    pg = PG(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros((0, 8)))
    assert pg.cost() == 0.0
    rep = pg.solve()
    assert rep["status"] == 0 and rep["final_cost"] == 0.0
    # single edge between the fixed vertex and one other: exact in one solve
    g = syn.make_graph("circle", 12, seed=3, meas_noise=True)
    ei, ej = np.array([0], np.int32), np.array([5], np.int32)
    pg = PG(12, ei, ej, g.meas[:1], None, None, g.poses_init, 0)
    rep = pg.solve(max_iters=30)
    assert rep["final_cost"] < 1e-20
    # duplicate edges (same pair twice, also reversed): both kept
    g = noisy_small(30)[0]
    ei = np.concatenate([g.edge_i, g.edge_i[:5], g.edge_j[5:8]])
    ej = np.concatenate([g.edge_j, g.edge_j[:5], g.edge_i[5:8]])
    meas = np.concatenate([g.meas, g.meas[:5], syn.inverse(g.meas[5:8])])
    og = O.OracleGraph(g.n_vertices, ei, ej, meas, None, None, 0)
    pg = PG(g.n_vertices, ei, ej, meas, None, None, g.poses_init, 0)
    _, ref = og.lm(g.poses_init)
    rep = pg.solve()
    assert abs(rep["final_cost"] - ref["final_cost"]) <= 1e-9 * ref["final_cost"]


def test_device_tensor_inputs_and_outputs():
    g = syn.make_config("c1_circle200")
    t = lambda a, dt=torch.float64: torch.as_tensor(a, dtype=dt, device="cuda")  # noqa: E731
    pg = PG(g.n_vertices, t(g.edge_i, torch.int32), t(g.edge_j, torch.int32), t(g.meas), None, None,
            t(g.poses_init), 0)
    out = torch.empty((g.n_vertices, 8), dtype=torch.float64, device="cuda")
    rep = pg.solve(poses_out=out)
    torch.cuda.synchronize()
    host = pg.get_poses()
    assert np.array_equal(out.cpu().numpy(), host)
    from paper_2603_17201_gb300 import evaluate_cost
    c = evaluate_cost(g.n_vertices, t(g.edge_i, torch.int32), t(g.edge_j, torch.int32), t(g.meas), None, out)
    assert abs(c.item() - rep["final_cost"]) <= 1e-12 * rep["final_cost"]


def test_repeat_solve_is_deterministic():
    g = syn.make_config("c1_circle200")
    p1 = PG(g.n_vertices, g.edge_i, g.edge_j, g.meas, None, None, g.poses_init, 0)
    p2 = PG(g.n_vertices, g.edge_i, g.edge_j, g.meas, None, None, g.poses_init, 0)
    r1 = p1.solve(precision="mixed")
    r2 = p2.solve(precision="mixed")
    assert r1["final_cost"] == r2["final_cost"]
    assert np.array_equal(p1.get_poses(), p2.get_poses())
