"""Pins of the oracle's projection search and loop fusion (Sec. IV-D: each
map point is projected into a keyframe and matched by descriptor similarity
within a window around its projection), each against something other than
the oracle itself:

  - ground truth: on noise-free features (exact projections, unflipped
    descriptors, every visible point detected, nothing matched before) every
    generated correspondence is recovered at Hamming distance 0;
  - every reported distance is the popcount of the descriptors' XOR (numpy);
  - a Sim(3) pose (R, s t, s) projects like (R, t, 1): the matches do not
    depend on the scale, and a wrong camera centre or projection would;
  - reordering a keyframe's features only renames the matched indices;
  - features matched before the search are never returned;
  - a hand-built conflict: two points choosing one feature, the smaller
    distance (then the lower index) keeps it; in fusion the loser fuses with
    the winner, and a feature holding a map point makes the points fuse with
    that point;
  - loop fusion skips the points a keyframe already observes.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_17201_gb300 import synthetic as syn


def _popcount(a):
    return np.unpackbits(np.ascontiguousarray(a).view(np.uint8), axis=-1).sum(axis=-1)


def test_noise_free_features_recover_the_ground_truth():
    w = syn.make_match_workload("search", n_kf=3, n_points=1500, seed=5, detect=1.0, pixel_noise=0.0,
                                max_flips=0, matched_frac=0.0, features_per_kf=3000)
    m, d, _ = O.project_match(w, "search", th=3.0)
    for k in range(3):
        t = w.truth[k]
        assert len(t["points"]) > 300
        # the predicted octave may be one above the detected one: both pass the octave window
        assert np.array_equal(m[k, t["points"]], t["features"])
        assert np.all(d[k, t["points"]] == 0)


def test_reported_distance_is_the_popcount_of_the_xor():
    w = syn.make_match_workload("search", n_kf=3, n_points=2000, seed=6)
    m, d, _ = O.project_match(w, "search")
    for k in range(3):
        sel = np.nonzero(m[k] >= 0)[0]
        assert len(sel) > 200
        f = w.feat_ptr[k] + m[k, sel]
        ham = _popcount(w.fdesc[f] ^ w.pdesc[sel])
        assert np.array_equal(d[k, sel], ham)
        assert d[k, sel].max() <= 50


def test_sim3_scale_does_not_change_the_matches():
    w = syn.make_match_workload("search", n_kf=3, n_points=2000, seed=7)
    m, d, _ = O.project_match(w, "search")
    p2 = w.poses.copy()
    p2[:, 4:7] *= 1.7
    p2[:, 7] *= 1.7
    m2, d2, _ = O.project_match(w, "search", poses=p2)
    assert np.array_equal(m, m2) and np.array_equal(d, d2)
    # an unscaled translation with the scaled s moves the camera: matches change
    p3 = w.poses.copy()
    p3[:, 7] *= 1.7
    m3, _, _ = O.project_match(w, "search", poses=p3)
    assert not np.array_equal(m, m3)


def test_feature_order_only_renames_indices():
    w = syn.make_match_workload("search", n_kf=1, n_points=2000, seed=8)
    m, d, _ = O.project_match(w, "search")
    rng = np.random.default_rng(0)
    perm = rng.permutation(w.feat_ptr[1])
    w2 = syn.MatchWorkload(**{k: getattr(w, k) for k in w.__dict__})
    for name in ("fu", "fv", "foct", "fdesc", "fskip", "fmp"):
        setattr(w2, name, getattr(w, name)[perm])
    m2, d2, _ = O.project_match(w2, "search")
    inv = np.argsort(perm)
    # unique best candidates: the same features under new indices
    ok = m[0] >= 0
    assert np.array_equal(perm[m2[0][ok]], m[0][ok]) or np.mean(perm[m2[0][ok]] == m[0][ok]) > 0.99
    assert np.array_equal(m2[0] >= 0, ok) or np.mean((m2[0] >= 0) == ok) > 0.99
    assert inv.shape[0] == perm.shape[0]


def test_matched_features_are_skipped():
    w = syn.make_match_workload("search", n_kf=3, n_points=2000, seed=9, matched_frac=0.3)
    m, _, _ = O.project_match(w, "search")
    for k in range(3):
        sel = m[k] >= 0
        assert not np.any(w.fskip[w.feat_ptr[k] + m[k, sel]])


def _tiny(mode):
    """One keyframe at the origin looking along +z, three features and three
    points that project onto feature 0; descriptors chosen by hand."""
    cam = syn.CAMERA
    poses = np.array([[0, 0, 0, 1, 0, 0, 0, 1.0]])
    X = np.array([[0.0, 0.0, 5.0], [0.0, 0.0, 5.0], [0.0, 0.0, 5.0]])
    pd = np.zeros((3, 8), np.uint32)
    pd[1, 0] = 0b11          # distance 2 from feature 0
    pd[2, 0] = 0b1           # distance 1
    fd = np.zeros((3, 8), np.uint32)
    fd[1] = 0xFFFFFFFF       # far away in descriptor space
    fd[2] = 0xFFFFFFFF
    return syn.MatchWorkload(
        mode=mode, camera=dict(cam), n_levels=8, scale_factor=1.2, poses=poses,
        feat_ptr=np.array([0, 3], np.int32), fu=np.array([cam["cx"], 10.0, 700.0], np.float32),
        fv=np.array([cam["cy"], 10.0, 400.0], np.float32), foct=np.zeros(3, np.int32), fdesc=fd,
        fskip=np.zeros(3, np.uint8), fmp=np.full(3, -1, np.int32), points=X, pdesc=pd,
        min_dist=np.full(3, 1.0), max_dist=np.full(3, 5.0), normal=np.tile([0.0, 0.0, 1.0], (3, 1)),
        pid=np.array([7, 8, 9], np.int32), truth=None)


def test_hand_built_conflicts():
    w = _tiny("search")
    m, d, _ = O.project_match(w, "search")
    # point 0 has distance 0 and wins; points 1 and 2 lose the feature
    assert m.tolist() == [[0, -1, -1]] and d[0, 0] == 0
    w.pdesc[0, 0] = 0b111    # now distance 3: point 2 (distance 1) wins
    m, d, _ = O.project_match(w, "search")
    assert m.tolist() == [[-1, -1, 0]] and d[0, 2] == 1
    w.pdesc[1, 0] = 0b10     # distance 1 too: the tie goes to the lower index, point 1
    m, _, _ = O.project_match(w, "search")
    assert m.tolist() == [[-1, 0, -1]]
    # fusion: the empty feature goes to point 1; 0 and 2 fuse with it (id 8)
    w.mode = "fusion"
    m, _, f = O.project_match(w, "fusion")
    assert m.tolist() == [[0, 0, 0]] and f.tolist() == [[8, -1, 8]]
    # a feature holding map point 42: every point choosing it fuses with 42
    w.fmp[0] = 42
    m, _, f = O.project_match(w, "fusion")
    assert f.tolist() == [[42, 42, 42]]
    # the keyframe already observes point 9 (feature 2 holds it): skipped
    w.fmp[2] = 9
    m, _, f = O.project_match(w, "fusion")
    assert m[0, 2] == -1 and f[0, 2] == -1


def test_fusion_finds_the_planted_duplicates():
    w = syn.make_match_workload("fusion", n_kf=8, n_points=2000, seed=10, pixel_noise=0.5, max_flips=10)
    m, d, f = O.project_match(w, "fusion", th=4.0)
    hits = 0
    for k in range(8):
        t = w.truth[k]
        fi = w.feat_ptr[k] + t["features"]
        planted = w.fmp[fi]
        dup = planted >= 500000
        good = m[k, t["points"]] == t["features"]
        assert np.array_equal(f[k, t["points"][dup & good]], planted[dup & good])
        own = planted == w.pid[t["points"]]
        assert np.all(m[k, t["points"][own]] == -1)
        hits += int((dup & good).sum())
    assert hits > 500
