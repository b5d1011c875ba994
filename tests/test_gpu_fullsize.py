"""End-to-end LM parity with the FP64 oracle at the full workload sizes
(Sec. IV-F: the essential-graph solve; Sec. VI: the LM scheme), through the
C ABI, each side run to convergence with the same stop rules:

  - batched form: a seeded sample of the 256-graph workload that contains its
    largest graph (4,962 keyframes, a 6-level multigrid hierarchy) and its
    smallest, solved together in one persistent launch with the multigrid
    preconditioner, each graph against its own oracle solve;
  - the 8,000-keyframe corridor graph (151,850 edges), LM to convergence;
  - the 4,000-keyframe noisy figure-8 graph (67,857 edges), forward solve.

Bars: final cost within 1e-9 (FP64) / 1e-6 (mixed) relative of the oracle's;
poses within 1e-5 (FP64) / 1e-3 (mixed) in max |log(S_gpu S_oracle^-1)|.
Every result's relative cost error and pose error (max, RMS) is printed in
the run's summary.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_17201_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": (1e-9, 1e-5), "mixed": (1e-6, 1e-3)}
MAX_ITERS = 100


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _oracle(g):
    og = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, None, None, g.fixed_vertex)
    p, rep = og.lm(g.poses_init, max_iters=MAX_ITERS)
    assert rep["status"] == 0 and rep["stop_reason"] in (1, 2), rep   # converged, not capped
    return p, rep


def _check(name, g, rep, poses, p_ref, ref, precision, parity_record):
    ctol, ptol = TOL[precision]
    assert rep["status"] == 0
    assert abs(rep["initial_cost"] - ref["initial_cost"]) <= 1e-13 * ref["initial_cost"]
    rel = abs(rep["final_cost"] - ref["final_cost"]) / ref["final_cost"]
    pe = O.pose_error(poses, p_ref)
    parity_record(f"{name} {precision}", rel, pe)
    assert rel <= ctol, (name, precision, rep, ref)
    assert pe.max() <= ptol, (name, precision, pe.max())
    f = g.fixed_vertex   # the gauge keyframe does not move
    assert np.array_equal(poses[f, 4:], g.poses_init[f, 4:])
    assert np.abs(poses[f, :4] - g.poses_init[f, :4] / np.linalg.norm(g.poses_init[f, :4])).max() <= 1e-15


# ---------------------------------------------------------------- batched form
def _batch_sample():
    sizes = np.array(syn.batch_sizes())
    rng = np.random.default_rng(4321)
    others = [int(k) for k in rng.choice(len(sizes), 10, replace=False)
              if k not in (sizes.argmax(), sizes.argmin())][:6]
    idx = [int(sizes.argmax()), int(sizes.argmin())] + others
    return idx, syn.make_batch(only=idx)


@pytest.fixture(scope="module")
def batch_case():
    idx, gs = _batch_sample()
    refs = [_oracle(g) for g in gs]
    return idx, gs, refs


def test_largest_batch_graph_has_a_six_level_hierarchy(batch_case):
    from paper_2603_17201_gb300 import PoseGraph
    _, gs, _ = batch_case
    g = gs[0]
    assert g.n_vertices == max(syn.batch_sizes())
    info = PoseGraph.from_synthetic(g).multigrid_info()
    assert len(info) == 6, info
    assert info[-1]["nodes"] <= 8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_sample_matches_oracle_per_graph(batch_case, precision, parity_record):
    from paper_2603_17201_gb300 import PoseGraphBatch
    idx, gs, refs = batch_case
    b = PoseGraphBatch(gs)
    reps, poses = b.solve(max_iters=MAX_ITERS, precision=precision, preconditioner="multigrid")
    for k, g, rep, p, (p_ref, ref) in zip(idx, gs, reps, poses, refs):
        _check(f"batch graph {k} ({g.n_vertices} KF)", g, rep, p, p_ref, ref, precision, parity_record)


# ---------------------------------------------------------------- single graphs
@pytest.fixture(scope="module")
def c3_case():
    g = syn.make_config("c3_corridor_8k")
    return g, _oracle(g)


@pytest.fixture(scope="module")
def c5_case():
    g = syn.make_config("c5_figure8_4k_noisy")
    return g, _oracle(g)


def _single(g, precision):
    from paper_2603_17201_gb300 import PoseGraph
    pg = PoseGraph.from_synthetic(g)
    poses = np.empty((g.n_vertices, 8))
    rep = pg.solve(poses_out=poses, max_iters=MAX_ITERS, precision=precision)
    return rep, poses


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c3_corridor_8k_lm_to_convergence(c3_case, precision, parity_record):
    g, (p_ref, ref) = c3_case
    rep, poses = _single(g, precision)
    assert rep["stop_reason"] in (1, 2), rep
    _check("c3 corridor 8k", g, rep, poses, p_ref, ref, precision, parity_record)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c5_figure8_4k_forward(c5_case, precision, parity_record):
    g, (p_ref, ref) = c5_case
    rep, poses = _single(g, precision)
    _check("c5 figure-8 4k noisy", g, rep, poses, p_ref, ref, precision, parity_record)
