"""Pins of the oracle's loop-correction steps (Sec. III-B, "Loop Correction":
the connected keyframes' poses are corrected with the loop's Sim(3) before
the pose graph optimisation, and the correction is carried to the map
points), each against something other than the oracle itself:

  - a worked example computed by hand (literal numbers below);
  - the identity correction changes nothing;
  - a correction that is a change of world frame G (S_c' = S_c G) moves every
    listed keyframe to S_k G and every point to G^-1 x, a closed form
    independent of the keyframe, checked with the numpy composition of the
    input generator;
  - relative poses within the connected set are unchanged;
  - the defining property: a point's position in its reference camera is the
    same before and after (S_after x' = S_before x, numpy);
  - unlisted keyframes and points with no reference keyframe are copied
    bit for bit.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_17201_gb300 import synthetic as syn


def _apply(S, x):
    """x -> s R x + t for pose8 arrays (numpy, the generator's rotation)."""
    return S[..., 7:8] * syn.quat_rotate(S[..., 0:4], x) + S[..., 4:7]


def _canon(p):
    p = np.array(p, dtype=float)
    p[..., 0:4] /= np.linalg.norm(p[..., 0:4], axis=-1, keepdims=True)
    p[..., 0:4] *= np.where(p[..., 3:4] < 0, -1.0, 1.0)
    return p


def test_worked_example_by_hand():
    # S_c: identity rotation, t = (1, 0, 0), s = 1; corrected S_c': 90 degrees
    # about z, t = 0, s = 2; keyframe k: identity rotation, t = (0, 1, 0).
    # S_k S_c^-1 = (I, (-1, 1, 0), 1), so S_k' = (R_z(90), (-1, 1, 0), 2).
    # A point x = (1, 2, 3) of k: S_k x = (1, 3, 3); S_k'^-1 of it is
    # R_z(90)^T ((1, 3, 3) - (-1, 1, 0)) / 2 = R_z(90)^T (2, 2, 3) / 2 = (1, -1, 1.5).
    h = np.sqrt(0.5)
    poses = np.array([[0, 0, 0, 1, 1, 0, 0, 1], [0, 0, 0, 1, 0, 1, 0, 1], [0, 0, 0, 1, 5, 5, 5, 1]], float)
    corrected = np.array([0, 0, h, h, 0, 0, 0, 2.0])
    out = O.propagate_correction(poses, 0, corrected, [0, 1])
    assert np.allclose(_canon(out[0]), _canon(corrected), atol=1e-15)
    assert np.allclose(_canon(out[1]), [0, 0, h, h, -1, 1, 0, 2], atol=1e-15)
    assert np.array_equal(out[2], poses[2])
    x = O.correct_points(poses, out, np.array([[1.0, 2.0, 3.0], [7.0, 8.0, 9.0]]), [1, -1])
    assert np.allclose(x[0], [1.0, -1.0, 1.5], atol=1e-15)
    assert np.array_equal(x[1], [7.0, 8.0, 9.0])


@pytest.fixture(scope="module")
def case():
    g = syn.make_config("c1_circle200")
    lc = syn.make_loop_correction(g, points_per_kf=20, seed=3)
    return g, lc


def test_identity_correction_is_a_no_op(case):
    g, lc = case
    out = O.propagate_correction(g.poses_init, lc.current, g.poses_init[lc.current], lc.connected)
    assert O.pose_error(out, g.poses_init).max() <= 1e-13
    assert np.abs(out[:, 4:] - g.poses_init[:, 4:]).max() <= 1e-13
    X = O.correct_points(g.poses_init, out, lc.points, lc.ref)
    assert np.abs(X - lc.points).max() <= 1e-12 * max(1.0, np.abs(lc.points).max())


def test_change_of_world_frame_closed_form(case):
    g, lc = case
    G = syn.compose(O.exp(np.array([0.3, -0.2, 0.5, 1.0, -2.0, 0.5, 0.2])), np.array([0, 0, 0, 1, 0, 0, 0, 1.0]))
    corrected = syn.compose(g.poses_init[lc.current], G)
    out = O.propagate_correction(g.poses_init, lc.current, corrected, lc.connected)
    want = syn.compose(g.poses_init[lc.connected], G[None])
    assert O.pose_error(out[lc.connected], want).max() <= 1e-13
    assert np.abs(out[lc.connected, 4:] - want[:, 4:]).max() <= 1e-12
    rest = np.setdiff1d(np.arange(g.n_vertices), lc.connected)
    assert np.array_equal(out[rest], g.poses_init[rest])
    # points of connected keyframes all move by G^-1, whatever their keyframe
    sel = np.isin(lc.ref, lc.connected)
    ref = np.where(sel, lc.ref, -1)
    X = O.correct_points(g.poses_init, out, lc.points, ref)
    Gi = syn.inverse(G)
    assert np.abs(X[sel] - _apply(Gi[None], lc.points[sel])).max() <= 1e-12
    assert np.array_equal(X[~sel], lc.points[~sel])


def test_relative_poses_kept_and_points_fixed_in_their_camera(case):
    g, lc = case
    out = O.propagate_correction(g.poses_init, lc.current, lc.corrected, lc.connected)
    c = lc.connected
    rel0 = syn.compose(g.poses_init[c][:, None], syn.inverse(g.poses_init[c])[None])
    rel1 = syn.compose(out[c][:, None], syn.inverse(out[c])[None])
    assert np.abs(rel1[..., 4:] - rel0[..., 4:]).max() <= 1e-12
    assert O.pose_error(rel1.reshape(-1, 8), rel0.reshape(-1, 8)).max() <= 1e-13
    X = O.correct_points(g.poses_init, out, lc.points, lc.ref)
    before = _apply(g.poses_init[lc.ref], lc.points)
    after = _apply(out[lc.ref], X)
    assert np.abs(after - before).max() <= 1e-12 * np.abs(before).max()
