"""The seeded synthetic workloads that stand in for the paper's sequences: the
sizes, the edge structure and the measurement recipe as stated for them
(keyframes, edges, covisibility window, loop edges, drift chain), checked
without a GPU.  Every parity test and bench line reads these inputs."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2603_17201_gb300 import synthetic as syn  # noqa: E402

SIZES = {  # name: (keyframes, edges, loop edges, covisibility window)
    "c1_circle200": (200, 1850, 1, None),
    "c2_figure8_2k": (2000, 29885, 5, 15),
    "c3_corridor_8k": (8000, 151850, 40, 19),
    "c5_figure8_4k_noisy": (4000, 67857, 10, 17),
}


def centres(poses):
    """Camera centres -R^T t / s of world-to-camera Sim(3) poses (pose8)."""
    out = np.empty((len(poses), 3))
    for v, p in enumerate(poses):
        inv = O.inverse(p)
        out[v] = inv[4:7]
    return out


@pytest.mark.parametrize("name", sorted(SIZES))
def test_sizes_and_edge_structure(name):
    n, m, loops, window = SIZES[name]
    g = syn.make_config(name)
    assert (g.n_vertices, g.n_edges, g.n_loop_edges, g.fixed_vertex) == (n, m, loops, 0)
    ei, ej = g.edge_i.astype(np.int64), g.edge_j.astype(np.int64)
    assert ei.min() >= 0 and ej.max() < n and np.all(ei != ej)
    tree = m - loops
    if window is not None:
        # every forward pair within the window, the tree edges (gap 1) among them
        assert tree == sum(n - k for k in range(1, window + 1))
        gap = ej[:tree] - ei[:tree]
        assert gap.min() == 1 and gap.max() == window
    else:
        # the 200-keyframe circle: the tree plus up to 10 sampled partners per
        # keyframe within 2..15 frames, then the loop from the last to the first
        gap = np.abs(ej[:tree] - ei[:tree])
        assert gap.max() <= 15 and np.all(np.isin(np.arange(n - 1), ei[:tree][gap == 1]))
        assert (ei[-1], ej[-1]) == (n - 1, 0)
    # loop edges join keyframes more than 200 frames apart (the circle: its
    # only loop), within 1.5 m of each other on the ground-truth path
    li, lj = ei[tree:], ej[tree:]
    assert np.all(li - lj > (198 if window is None else 200))
    c = centres(g.poses_gt)
    if window is not None:
        assert np.all(np.linalg.norm(c[li] - c[lj], axis=1) <= 1.5 + 1e-9)
    assert np.allclose(np.linalg.norm(g.meas[:, :4], axis=1), 1.0, atol=1e-12)
    assert np.all(g.meas[:, 7] > 0) and np.all(g.poses_init[:, 7] > 0)


@pytest.mark.parametrize("name", ["c1_circle200", "c2_figure8_2k"])
def test_measurement_recipe(name):
    """Tree and covisibility measurements come from the drifted estimate
    (the initial guess), loop measurements from the ground truth; the first
    pose is exact.  So the initial cost lies on the loop edges alone."""
    g = syn.make_config(name)
    tree = g.n_edges - g.n_loop_edges
    og = O.OracleGraph.from_synthetic(g)
    r = og.cost(g.poses_init, residuals=True)[1]
    assert np.abs(r[:tree]).max() < 1e-9
    assert np.abs(r[tree:]).max() > 1e-3
    assert np.allclose(g.poses_init[0], g.poses_gt[0], atol=1e-15)
    rgt = og.cost(g.poses_gt, residuals=True)[1]
    assert np.abs(rgt[tree:]).max() < 1e-9


def test_seeded_and_deterministic():
    a, b = syn.make_config("c2_figure8_2k"), syn.make_config("c2_figure8_2k")
    for k in ("edge_i", "edge_j", "meas", "poses_init", "poses_gt"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    c = syn.make_config("c2_figure8_2k", seed=7)
    assert not np.array_equal(a.poses_init, c.poses_init)


def test_batch_sizes_and_edge_counts():
    """256 graphs with keyframe counts from U[100, 5000] (680,160 in total);
    graph k holds its 15-frame window pairs and one loop per 400 keyframes at
    most."""
    sizes = syn.batch_sizes()
    assert len(sizes) == 256 and min(sizes) >= 100 and max(sizes) <= 5000
    assert sum(sizes) == 680160
    for g in syn.make_batch(only=[0, 1, 58]):
        n = g.n_vertices
        assert g.n_edges - g.n_loop_edges == 15 * n - 120
        assert 1 <= g.n_loop_edges <= max(1, n // 400)
