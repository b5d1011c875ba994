"""GPU parity of the projection search (PS1, PS3a-c) and loop fusion
(Sec. IV-D) against the oracle, through the C ABI.  The matches, the Hamming
distances and the fusion targets are integers decided by single-precision
geometry that both sides evaluate with the same IEEE operations in the same
order, so they are compared bit for bit.  Cases: PS1 (one keyframe), PS3a-c
(three keyframes), loop fusion over 30 connected keyframes, ragged point
counts (1, 129, 4001), no points, features outside the image, every feature
matched before, points behind the cameras, and a call repeated on the same
frames object.
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


def _run(w, mode, th, **kw):
    from paper_2603_17201_gb300 import Frames
    fr = Frames.from_workload(w)
    m, d, f = fr.match_workload(w, mode, th=th, **kw)
    torch.cuda.synchronize()
    out = (m.cpu().numpy(), d.cpu().numpy(), None if f is None else f.cpu().numpy())
    fr.close()
    return out


def _check(w, mode, th, **kw):
    m, d, f = _run(w, mode, th, **kw)
    mr, dr, fr = O.project_match(w, mode, th=th, **kw)
    assert np.array_equal(m, mr), np.argwhere(m != mr)[:5]
    assert np.array_equal(d, dr), np.argwhere(d != dr)[:5]
    if mode == "fusion":
        assert np.array_equal(f, fr), np.argwhere(f != fr)[:5]
    return m, d, f


@pytest.mark.parametrize("n_kf,n_points,seed", [(1, 4000, 1), (3, 4000, 2), (3, 4001, 3), (3, 129, 4), (1, 1, 5)])
def test_projection_search_matches_oracle(n_kf, n_points, seed):
    w = syn.make_match_workload("search", n_kf=n_kf, n_points=n_points, seed=seed)
    m, _, _ = _check(w, "search", 10.0)
    if n_points > 1000:
        assert (m >= 0).sum() > 500 * n_kf


@pytest.mark.parametrize("n_kf,n_points,seed", [(30, 4000, 11), (8, 1500, 12)])
def test_loop_fusion_matches_oracle(n_kf, n_points, seed):
    w = syn.make_match_workload("fusion", n_kf=n_kf, n_points=n_points, seed=seed)
    m, _, f = _check(w, "fusion", 4.0)
    assert (f >= 0).sum() > 100


def test_edge_cases():
    w = syn.make_match_workload("search", n_kf=3, n_points=2000, seed=21)
    # features outside the image bounds (clamped into the border cells of the grid)
    w.fu = w.fu.copy()
    w.fu[:50] = -5.0
    w.fu[50:100] = 800.0
    _check(w, "search", 10.0)
    # every feature matched before: no match at all
    w2 = syn.MatchWorkload(**w.__dict__)
    w2.fskip = np.ones_like(w.fskip)
    m, _, _ = _check(w2, "search", 10.0)
    assert (m >= 0).sum() == 0
    # points behind the cameras
    w3 = syn.MatchWorkload(**w.__dict__)
    w3.points = -w.points
    _check(w3, "search", 10.0)
    # a wide window and a loose threshold (many candidates per point)
    _check(w, "search", 40.0, th_low=100)
    # no points
    w4 = syn.MatchWorkload(**w.__dict__)
    for k in ("points", "pdesc", "min_dist", "max_dist", "normal", "pid"):
        setattr(w4, k, getattr(w, k)[:0])
    m, d, _ = _run(w4, "search", 10.0)
    assert m.shape == (3, 0)


def test_repeated_calls_on_one_frames_object():
    from paper_2603_17201_gb300 import Frames
    w = syn.make_match_workload("fusion", n_kf=6, n_points=1000, seed=31)
    fr = Frames.from_workload(w)
    ref = O.project_match(w, "fusion", th=4.0)
    for _ in range(3):
        m, d, f = fr.match_workload(w, "fusion", th=4.0)
        assert np.array_equal(m.cpu().numpy(), ref[0]) and np.array_equal(f.cpu().numpy(), ref[2])
    ws = syn.make_match_workload("search", n_kf=6, n_points=1000, seed=31)
    ref_s = O.project_match(ws, "search", th=10.0)
    fs = Frames.from_workload(ws)
    for _ in range(2):
        m, d, _ = fs.match_workload(ws, "search", th=10.0)
        assert np.array_equal(m.cpu().numpy(), ref_s[0]) and np.array_equal(d.cpu().numpy(), ref_s[1])
