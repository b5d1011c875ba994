"""Batched form (Sec. IV-F solve over many graphs in one persistent launch):
every graph of an uneven batch against its own oracle solve with either
preconditioner (the multigrid hierarchy is one segment per graph), the
schedules the autotuner chooses from, and agreement with single-graph GPU
solves."""
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


def uneven_batch(n=12, seed0=50):
    rng = np.random.default_rng(seed0)
    gs = []
    for k in range(n):
        nv = int(rng.integers(20, 400))
        gs.append(syn.make_graph("figure8", nv, seed=seed0 + k, window=int(rng.integers(3, 12)),
                                 n_loops=2, meas_noise=bool(k % 2), loop_min_gap=nv // 3, loop_max_dist=3.0))
    # one graph with its gauge vertex in the middle
    gs[3].fixed_vertex = gs[3].n_vertices // 2
    return gs


@pytest.mark.parametrize("precond", ["block_jacobi", "multigrid"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_batch_matches_oracle_per_graph(precision, tol, precond):
    from paper_2603_17201_gb300 import PoseGraphBatch
    gs = uneven_batch()
    b = PoseGraphBatch(gs)
    reps, poses = b.solve(max_iters=20, precision=precision, preconditioner=precond)
    lanes, threads, bps, _ = b.schedule()
    assert lanes in (4, 8, 16) and threads in (256, 512) and bps in (1, 2)
    for g, rep, p in zip(gs, reps, poses):
        og = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, None, None, g.fixed_vertex)
        p_ref, ref = og.lm(g.poses_init, max_iters=20)
        assert rep["status"] == 0
        assert abs(rep["initial_cost"] - ref["initial_cost"]) <= 1e-13 * ref["initial_cost"]
        assert abs(rep["final_cost"] - ref["final_cost"]) <= tol * ref["final_cost"], (rep, ref)
        assert O.pose_error(p, p_ref).max() < (1e-5 if precision == "fp64" else 1e-3)
        f = g.fixed_vertex
        assert np.array_equal(p[f, 4:], g.poses_init[f, 4:])


@pytest.mark.parametrize("schedule", list(range(8)))
def test_every_fp64_schedule_agrees(schedule):
    from paper_2603_17201_gb300 import PoseGraphBatch
    gs = uneven_batch(6, seed0=80)
    b = PoseGraphBatch(gs)
    reps, _ = b.solve(max_iters=15, precision="fp64", schedule=schedule)
    b2 = PoseGraphBatch(gs)
    ref, _ = b2.solve(max_iters=15, precision="fp64", schedule=0)
    for r, q in zip(reps, ref):
        assert abs(r["final_cost"] - q["final_cost"]) <= 1e-9 * q["final_cost"]


def test_batch_agrees_with_single_graph_solver_and_resumes():
    from paper_2603_17201_gb300 import PoseGraph, PoseGraphBatch
    gs = uneven_batch(5, seed0=90)
    b = PoseGraphBatch(gs)
    reps, poses = b.solve(max_iters=6, precision="mixed")
    reps2, poses2 = b.solve(max_iters=20, precision="mixed")   # continues from the estimate
    for g, r, r2 in zip(gs, reps, reps2):
        pg = PoseGraph.from_synthetic(g)
        rs = pg.solve(max_iters=26, precision="mixed")
        assert r2["final_cost"] <= r["final_cost"] * (1 + 1e-12)
        assert abs(r2["final_cost"] - rs["final_cost"]) <= 1e-6 * rs["final_cost"]
