"""GPU parity of the loop-correction steps around the pose graph optimisation
(Sec. III-B, "Loop Correction") against the oracle, through the C ABI:

  pgo_propagate_correction  S_k' = (S_k S_c^-1) S_c' for the connected
                            keyframes, every other pose copied bit for bit;
  pgo_correct_points        x' = S_after[r]^-1 (S_before[r] x) per map point.

Tolerance 1e-12 relative to the largest value (both FP64; the kernel applies
a per-keyframe similarity table, the oracle composes per point: different
rounding order).  Copied rows and unchanged points are compared bit for bit
and skipped indices are counted exactly.  Sizes: the 200-keyframe circle (20
points per keyframe), the 2,000-keyframe figure-8 (150 per keyframe, 300,000
points, as in the benchmark) with a ragged tail, and the 8,000-keyframe
corridor (1.2 M points), plus the optimisation in between on the small graph.
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


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(1.0, np.abs(b).max())


@pytest.mark.parametrize("name,ppk,drop", [("c1_circle200", 20, 0), ("c2_figure8_2k", 150, 37),
                                           ("c3_corridor_8k", 150, 0)])
def test_propagate_and_correct_points_match_oracle(name, ppk, drop):
    from paper_2603_17201_gb300 import correct_points, propagate_correction
    g = syn.make_config(name)
    lc = syn.make_loop_correction(g, points_per_kf=ppk, seed=11)
    X, ref = lc.points[: len(lc.points) - drop], lc.ref[: len(lc.ref) - drop]   # ragged tail
    out, bad = propagate_correction(g.poses_init, lc.current, lc.corrected, lc.connected, return_bad=True)
    out_h = out.cpu().numpy()
    want = O.propagate_correction(g.poses_init, lc.current, lc.corrected, lc.connected)
    assert int(bad.item()) == 0
    assert _rel(out_h, want) <= 1e-12
    rest = np.setdiff1d(np.arange(g.n_vertices), lc.connected)
    assert np.array_equal(out_h[rest], g.poses_init[rest])
    assert np.all(out_h[lc.connected, 3] >= 0.0)
    # the connected keyframes' points follow them (others unchanged) ...
    sel = np.where(np.isin(ref, lc.connected), ref, -1).astype(np.int32)
    Xg, bad = correct_points(g.poses_init, out, X, sel, return_bad=True)
    Xw = O.correct_points(g.poses_init, want, X, sel)
    assert int(bad.item()) == 0
    assert _rel(Xg.cpu().numpy(), Xw) <= 1e-12
    assert np.array_equal(Xg.cpu().numpy()[sel < 0], X[sel < 0])
    # ... and every point follows its keyframe through a second pose change
    after = syn.compose(O.exp(np.array([0.01, -0.02, 0.03, 0.1, 0.2, -0.1, 0.05])), want)
    Xg2 = correct_points(want, after, X, ref).cpu().numpy()
    assert _rel(Xg2, O.correct_points(want, after, X, ref)) <= 1e-12


def test_edge_cases_bad_indices_in_place_and_misaligned():
    from paper_2603_17201_gb300 import correct_points, propagate_correction
    g = syn.make_config("c1_circle200")
    lc = syn.make_loop_correction(g, points_per_kf=3, seed=2)
    conn = np.concatenate([lc.connected, [-5, g.n_vertices, 10 ** 6]]).astype(np.int32)
    out, bad = propagate_correction(g.poses_init, lc.current, lc.corrected, conn, return_bad=True)
    assert int(bad.item()) == 3
    assert _rel(out.cpu().numpy(), O.propagate_correction(g.poses_init, lc.current, lc.corrected,
                                                          lc.connected)) <= 1e-12
    # no connected keyframe: a plain copy
    out0 = propagate_correction(g.poses_init, lc.current, lc.corrected, np.zeros(0, np.int32))
    assert np.array_equal(out0.cpu().numpy(), g.poses_init)
    after = out.cpu().numpy()
    ref = lc.ref.copy()
    ref[5] = g.n_vertices          # counted, unchanged
    ref[6] = -1                    # unchanged
    want = O.correct_points(g.poses_init, after, lc.points, np.where(ref >= g.n_vertices, -1, ref))
    # 8-byte-aligned (not 16) point arrays: the scalar staging path
    buf = torch.zeros(1 + lc.points.size, dtype=torch.float64, device="cuda")
    buf[1:] = torch.as_tensor(lc.points.ravel(), device="cuda")
    X = buf[1:].view(-1, 3)
    Xg, bad = correct_points(g.poses_init, after, X, ref, return_bad=True)
    assert int(bad.item()) == 1
    assert _rel(Xg.cpu().numpy(), want) <= 1e-12
    assert np.array_equal(Xg.cpu().numpy()[[5, 6]], lc.points[[5, 6]])
    # in place
    Xi = torch.as_tensor(lc.points, device="cuda").clone()
    correct_points(g.poses_init, after, Xi, ref, out=Xi)
    assert _rel(Xi.cpu().numpy(), want) <= 1e-12
    # no points
    empty = correct_points(g.poses_init, after, np.zeros((0, 3)), np.zeros(0, np.int32))
    assert empty.shape == (0, 3)


def test_loop_correction_pipeline_around_the_solve():
    """Propagate the loop correction, optimise from the propagated poses,
    then carry the optimisation to every map point: GPU against the oracle's
    same three steps (final cost 1e-9; points 1e-6 relative: the two solves
    agree to the LM stopping tolerance, not to rounding)."""
    from paper_2603_17201_gb300 import PoseGraph, correct_points, propagate_correction
    g = syn.make_config("c1_circle200")
    lc = syn.make_loop_correction(g, points_per_kf=50, seed=4)
    init = propagate_correction(g.poses_init, lc.current, lc.corrected, lc.connected).cpu().numpy()
    init_ref = O.propagate_correction(g.poses_init, lc.current, lc.corrected, lc.connected)
    pg = PoseGraph.from_synthetic(g, poses=init)
    poses = np.empty((g.n_vertices, 8))
    rep = pg.solve(poses_out=poses, max_iters=50)
    og = O.OracleGraph.from_synthetic(g)
    p_ref, ref = og.lm(init_ref, max_iters=50)
    assert abs(rep["final_cost"] - ref["final_cost"]) <= 1e-9 * ref["final_cost"]
    X = correct_points(init, poses, lc.points, lc.ref).cpu().numpy()
    Xw = O.correct_points(init_ref, p_ref, lc.points, lc.ref)
    assert _rel(X, Xw) <= 1e-6
