"""Seeded synthetic Sim(3) essential graphs (the only input source shared by the
CUDA path, the oracle, the tests and the benchmark).

The paper evaluates loop closing on EuRoC and TUM-VI sequences (Sec. V-A) and
optimises the essential graph after a loop is accepted (Sec. III-B, Sec. IV-F),
but prints neither graph sizes nor graph statistics.  These generators stand in
for those essential graphs with trajectories of the same shape:

* ``circle``     200 keyframes on a 10 m circle, one loop (last -> first);
* ``figure8``    drone-flight-shaped (EuRoC-like) 3-D figure-8, two laps;
* ``corridor``   handheld-sequence-shaped (TUM-VI-like) random walk along
                 corridors of a 50 m x 50 m grid with many revisits.

Conventions (shared with the solver, stated here so the module stands alone):
a pose S = (q, t, s) maps world points to the camera frame, x_c = s R(q) x_w + t,
stored as 8 float64 values (qx, qy, qz, qw, tx, ty, tz, s).  An edge (i, j)
carries the measured relative transform Z_ij ~ S_j S_i^-1.

Drift model: the initial estimate is the chain of ground-truth relative steps,
each left-multiplied by a noise transform N = (q_n, t_n, s_n) with
q_n = normalise([n_rot / 2, 1]), t_n = n_trans, s_n = exp(n_ls) and
n ~ Normal(0, diag(sig_rot^2 I3, sig_trans^2 I3, sig_ls^2)).  Spanning-tree and
covisibility measurements come from the drifted estimate (they are consistent
with it, as after ORB-SLAM-style loop correction), loop measurements from the
ground truth; optional i.i.d. measurement noise of the same form perturbs every
edge.

Also built here: the inputs of the loop-correction steps around the
optimisation (the keyframe that closed the loop, its Sim(3) correction, its
connected keyframes and map points in front of every keyframe;
``make_loop_correction``), and keyframes with ORB-like features for the
projection search and loop fusion (a 752 x 480 camera, random 256-bit
descriptors, features at the projections of the map points plus clutter;
``make_match_workload``).

This module holds problem construction only (quaternion products to compose
poses, a pinhole projection to place features).  It contains none of the
method's arithmetic: no exp/log maps, residuals, Jacobians or normal
equations, no loop correction, no search or matching.  Randomness comes only
from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "PoseGraph", "make_graph", "make_config", "make_batch", "batch_sizes", "CONFIGS",
    "compose", "inverse", "quat_mul", "quat_rotate", "LoopCorrection", "make_loop_correction",
]


# --------------------------------------------------------------------------
# Plain quaternion / similarity-transform composition (problem construction).
# --------------------------------------------------------------------------
def quat_mul(a, b):
    """Hamilton product of (..., 4) quaternions stored (x, y, z, w)."""
    ax, ay, az, aw = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    bx, by, bz, bw = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([
        aw * bx + ax * bw + ay * bz - az * by,
        aw * by - ax * bz + ay * bw + az * bx,
        aw * bz + ax * by - ay * bx + az * bw,
        aw * bw - ax * bx - ay * by - az * bz,
    ], axis=-1)


def quat_rotate(q, v):
    """Rotate (..., 3) vectors by unit quaternions (..., 4)."""
    u = q[..., :3]
    w = q[..., 3:4]
    t = 2.0 * np.cross(u, v)
    return v + w * t + np.cross(u, t)


def compose(a, b):
    """a * b for poses stored (..., 8): (R_a R_b, s_a R_a t_b + t_a, s_a s_b)."""
    q = quat_mul(a[..., 0:4], b[..., 0:4])
    t = a[..., 7:8] * quat_rotate(a[..., 0:4], b[..., 4:7]) + a[..., 4:7]
    s = a[..., 7:8] * b[..., 7:8]
    return np.concatenate([q, t, s], axis=-1)


def inverse(a):
    """a^-1 = (R^T, -R^T t / s, 1 / s) for poses stored (..., 8)."""
    qi = a[..., 0:4] * np.array([-1.0, -1.0, -1.0, 1.0])
    t = -quat_rotate(qi, a[..., 4:7]) / a[..., 7:8]
    return np.concatenate([qi, t, 1.0 / a[..., 7:8]], axis=-1)


def _prefix_compose(steps, first):
    """P_0 = first, P_k = steps[k] * P_{k-1} for k >= 1 (steps[0] unused).

    Evaluated as a Hillis-Steele scan of the associative product so that
    large graphs are built with O(log N) vectorised passes."""
    n = steps.shape[0]
    acc = steps.copy()
    acc[0] = first
    shift = 1
    while shift < n:
        nxt = acc.copy()
        nxt[shift:] = compose(acc[shift:], acc[:-shift])
        acc = nxt
        shift *= 2
    q = acc[:, 0:4]
    acc[:, 0:4] = q / np.linalg.norm(q, axis=1, keepdims=True)
    return acc


def _noise(rng, n, sig_rot, sig_trans, sig_ls):
    """n noise transforms (q_n, t_n, s_n) as documented in the module header."""
    nr = rng.normal(0.0, sig_rot, size=(n, 3))
    nt = rng.normal(0.0, sig_trans, size=(n, 3))
    ns = rng.normal(0.0, sig_ls, size=(n, 1))
    q = np.concatenate([0.5 * nr, np.ones((n, 1))], axis=1)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return np.concatenate([q, nt, np.exp(ns)], axis=1)


def _rotmat_to_quat(R):
    """Rotation matrices (..., 3, 3) -> unit quaternions (x, y, z, w)."""
    R = np.asarray(R, dtype=np.float64)
    m00, m11, m22 = R[..., 0, 0], R[..., 1, 1], R[..., 2, 2]
    tr = m00 + m11 + m22
    out = np.empty(R.shape[:-2] + (4,))
    cand = np.stack([tr, m00, m11, m22], axis=-1)
    k = np.argmax(cand, axis=-1)
    for case in range(4):
        sel = k == case
        if not np.any(sel):
            continue
        Rs = R[sel]
        if case == 0:
            r = np.sqrt(1.0 + tr[sel]) * 2.0
            q = np.stack([(Rs[:, 2, 1] - Rs[:, 1, 2]) / r, (Rs[:, 0, 2] - Rs[:, 2, 0]) / r,
                          (Rs[:, 1, 0] - Rs[:, 0, 1]) / r, 0.25 * r], axis=-1)
        elif case == 1:
            r = np.sqrt(1.0 + Rs[:, 0, 0] - Rs[:, 1, 1] - Rs[:, 2, 2]) * 2.0
            q = np.stack([0.25 * r, (Rs[:, 0, 1] + Rs[:, 1, 0]) / r,
                          (Rs[:, 0, 2] + Rs[:, 2, 0]) / r, (Rs[:, 2, 1] - Rs[:, 1, 2]) / r], axis=-1)
        elif case == 2:
            r = np.sqrt(1.0 + Rs[:, 1, 1] - Rs[:, 0, 0] - Rs[:, 2, 2]) * 2.0
            q = np.stack([(Rs[:, 0, 1] + Rs[:, 1, 0]) / r, 0.25 * r,
                          (Rs[:, 1, 2] + Rs[:, 2, 1]) / r, (Rs[:, 0, 2] - Rs[:, 2, 0]) / r], axis=-1)
        else:
            r = np.sqrt(1.0 + Rs[:, 2, 2] - Rs[:, 0, 0] - Rs[:, 1, 1]) * 2.0
            q = np.stack([(Rs[:, 0, 2] + Rs[:, 2, 0]) / r, (Rs[:, 1, 2] + Rs[:, 2, 1]) / r,
                          0.25 * r, (Rs[:, 1, 0] - Rs[:, 0, 1]) / r], axis=-1)
        out[sel] = q
    out *= np.where(out[..., 3:4] < 0, -1.0, 1.0)
    return out / np.linalg.norm(out, axis=-1, keepdims=True)


def _poses_from_path(centres, forward):
    """World->camera poses (scale 1) of cameras at ``centres`` looking along
    ``forward`` with world +z as up."""
    f = forward / np.linalg.norm(forward, axis=1, keepdims=True)
    up = np.array([0.0, 0.0, 1.0])
    x = np.cross(f, up)
    bad = np.linalg.norm(x, axis=1) < 1e-6
    x[bad] = np.array([1.0, 0.0, 0.0])
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    y = np.cross(f, x)
    R_wc = np.stack([x, y, f], axis=-1)          # columns: camera axes in world
    R_cw = np.transpose(R_wc, (0, 2, 1))
    q = _rotmat_to_quat(R_cw)
    t = -np.einsum("nij,nj->ni", R_cw, centres)
    return np.concatenate([q, t, np.ones((len(centres), 1))], axis=1)


# --------------------------------------------------------------------------
# Trajectories
# --------------------------------------------------------------------------
def _circle(n, radius=10.0):
    phi = np.linspace(0.0, 2.0 * np.pi, n, endpoint=False)
    c = np.stack([radius * np.cos(phi), radius * np.sin(phi), np.zeros(n)], axis=1)
    f = np.stack([-np.sin(phi), np.cos(phi), np.zeros(n)], axis=1)
    return c, f


def _figure8(n, laps=2.0, half_width=10.0, height=1.5):
    phi = np.linspace(0.0, 2.0 * np.pi * laps, n, endpoint=False)
    c = np.stack([half_width * np.sin(phi), half_width * np.sin(phi) * np.cos(phi),
                  1.0 + height * np.sin(2.0 * phi)], axis=1)
    f = np.stack([half_width * np.cos(phi), half_width * np.cos(2.0 * phi),
                  2.0 * height * np.cos(2.0 * phi)], axis=1)
    return c, f


def _corridor(n, rng, size=50.0, spacing=5.0, step=1.0):
    """Random walk at ``step`` metres per keyframe along the lines of a grid
    of corridors ``spacing`` apart, turning at random at grid nodes (no
    U-turns unless at a wall)."""
    per_seg = int(round(spacing / step))
    nodes = int(round(size / spacing))
    dirs = np.array([[1, 0], [0, 1], [-1, 0], [0, -1]])
    node = np.array([nodes // 2, nodes // 2])
    d = 0
    pts, fwd = [], []
    while len(pts) < n:
        opts = []
        for k in range(4):
            if k == (d + 2) % 4:
                continue
            nxt = node + dirs[k]
            if 0 <= nxt[0] <= nodes and 0 <= nxt[1] <= nodes:
                opts.append(k)
        if not opts:
            opts = [(d + 2) % 4]
        d = int(opts[rng.integers(len(opts))])
        for s in range(per_seg):
            p = (node + dirs[d] * (s / per_seg)) * spacing
            pts.append([p[0], p[1], 1.2])
            fwd.append([dirs[d][0], dirs[d][1], 0.0])
        node = node + dirs[d]
    c = np.array(pts[:n], dtype=np.float64)
    f = np.array(fwd[:n], dtype=np.float64)
    # look slightly ahead-and-sideways so the cameras are not exactly planar
    f = f + np.array([0.0, 0.0, 0.05])
    return c, f


# --------------------------------------------------------------------------
# Graph assembly
# --------------------------------------------------------------------------
@dataclasses.dataclass
class PoseGraph:
    """A Sim(3) essential graph in the solver's input layout (all float64
    except the int32 edge endpoints)."""
    name: str
    n_vertices: int
    edge_i: np.ndarray          # (E,) int32
    edge_j: np.ndarray          # (E,) int32
    meas: np.ndarray            # (E, 8) float64, Z_ij ~ S_j S_i^-1
    weight: np.ndarray          # (E,) float64
    poses_init: np.ndarray      # (N, 8) drifted estimate (the initial guess)
    poses_gt: np.ndarray        # (N, 8) ground truth
    fixed_vertex: int = 0
    n_loop_edges: int = 0
    seed: int = 0

    @property
    def n_edges(self) -> int:
        return int(self.edge_i.shape[0])


def _window_edges(n, window):
    """All forward pairs (i, i+k), 1 <= k <= window (k = 1 is the tree edge)."""
    ii, jj = [], []
    for k in range(1, window + 1):
        i = np.arange(0, n - k)
        ii.append(i)
        jj.append(i + k)
    return np.concatenate(ii), np.concatenate(jj)


def _sampled_edges(n, rng, max_partners=10, lo=2, hi=15):
    """Tree edges plus, per keyframe, up to ``max_partners`` partners drawn
    without replacement from lo <= |i - j| <= hi; undirected duplicates are
    removed.  Pairs are stored with i < j."""
    pairs = set((k, k + 1) for k in range(n - 1))
    for k in range(n):
        cand = [j for j in range(k - hi, k + hi + 1) if 0 <= j < n and lo <= abs(j - k)]
        m = min(max_partners, len(cand))
        pick = rng.choice(len(cand), size=m, replace=False)
        for p in pick:
            j = cand[int(p)]
            pairs.add((min(k, j), max(k, j)))
    pairs = sorted(pairs)
    a = np.array(pairs, dtype=np.int64)
    return a[:, 0], a[:, 1]


def _loop_pairs(centres, n_loops, min_gap=200, max_dist=1.5):
    """``n_loops`` revisit pairs (i, j), j - i > min_gap, spatially close,
    spread evenly over the later keyframes.  Returned as (later, earlier)."""
    n = len(centres)
    out = []
    if n_loops <= 0:
        return out
    starts = np.linspace(min_gap + 1, n - 1, n_loops + 2)[1:-1].astype(int) if n_loops > 1 \
        else np.array([n - 1])
    used = set()
    for s in starts:
        found = None
        for i in list(range(s, n)) + list(range(s - 1, min_gap, -1)):
            if i in used:
                continue
            prev = centres[: i - min_gap]
            if len(prev) == 0:
                continue
            d = np.linalg.norm(prev - centres[i], axis=1)
            j = int(np.argmin(d))
            if d[j] <= max_dist:
                found = (i, j)
                break
        if found is not None:
            used.add(found[0])
            out.append(found)
    return out


def make_graph(kind, n, *, seed, window=15, n_loops=1, noise=(0.01, 0.02, 0.01),
               meas_noise=False, name=None, weight=1.0, loop_min_gap=200, loop_max_dist=1.5):
    """Build one synthetic essential graph.

    kind      'circle' | 'figure8' | 'corridor'
    n         number of keyframes
    window    covisibility window (forward pairs within ``window`` frames);
              for 'circle' the sampled scheme of the 200-keyframe case is used
    n_loops   loop edges (for 'circle': the single last -> first edge)
    loop_min_gap, loop_max_dist  a loop joins keyframes more than
              ``loop_min_gap`` frames apart within ``loop_max_dist`` metres
    noise     (sig_rot rad, sig_trans m, sig_logscale) per drift step
    meas_noise  add i.i.d. noise of the same form to every measurement
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "circle":
        c, f = _circle(n)
    elif kind == "figure8":
        c, f = _figure8(n)
    elif kind == "corridor":
        c, f = _corridor(n, rng)
    else:
        raise ValueError(f"unknown trajectory kind {kind!r}")
    gt = _poses_from_path(c, f)

    # drifted estimate: chain of noisy relative steps from the (exact) first pose
    steps = compose(gt[1:], inverse(gt[:-1]))
    steps = compose(_noise(rng, n - 1, *noise), steps)
    steps = np.concatenate([np.zeros((1, 8)), steps], axis=0)
    est = _prefix_compose(steps, gt[0])

    if kind == "circle":
        ei, ej = _sampled_edges(n, rng)
        loops = [(n - 1, 0)] if n_loops > 0 else []
    else:
        ei, ej = _window_edges(n, window)
        loops = _loop_pairs(c, n_loops, min_gap=loop_min_gap, max_dist=loop_max_dist)
    meas = compose(est[ej], inverse(est[ei]))
    if loops:
        li = np.array([p[0] for p in loops], dtype=np.int64)
        lj = np.array([p[1] for p in loops], dtype=np.int64)
        lmeas = compose(gt[lj], inverse(gt[li]))
        ei = np.concatenate([ei, li])
        ej = np.concatenate([ej, lj])
        meas = np.concatenate([meas, lmeas], axis=0)
    if meas_noise:
        meas = compose(_noise(rng, meas.shape[0], *noise), meas)
    meas[:, 0:4] /= np.linalg.norm(meas[:, 0:4], axis=1, keepdims=True)
    E = ei.shape[0]
    return PoseGraph(
        name=name or f"{kind}{n}", n_vertices=n,
        edge_i=ei.astype(np.int32), edge_j=ej.astype(np.int32),
        meas=np.ascontiguousarray(meas), weight=np.full(E, float(weight)),
        poses_init=np.ascontiguousarray(est), poses_gt=np.ascontiguousarray(gt),
        fixed_vertex=0, n_loop_edges=len(loops), seed=seed)


# The five evaluation configurations (seeded; sizes as in the workload table).
CONFIGS = {
    "c1_circle200": dict(kind="circle", n=200, seed=0, n_loops=1,
                         noise=(0.01, 0.02, 0.01)),
    "c2_figure8_2k": dict(kind="figure8", n=2000, seed=1, window=15, n_loops=5,
                          noise=(0.01, 0.02, 0.01)),
    "c3_corridor_8k": dict(kind="corridor", n=8000, seed=2, window=19, n_loops=40,
                           noise=(0.01, 0.02, 0.02)),
    "c5_figure8_4k_noisy": dict(kind="figure8", n=4000, seed=3, window=17, n_loops=10,
                                noise=(0.01, 0.02, 0.01), meas_noise=True),
}


def make_config(name, **overrides):
    """One of the named single-graph configurations."""
    kw = dict(CONFIGS[name])
    kw.update(overrides)
    return make_graph(name=name, **kw)


def batch_sizes(n_graphs=256, seed0=1000, n_min=100, n_max=5000):
    """Keyframe counts of the batched workload's graphs (graph k draws its
    size from seed ``seed0 + k``)."""
    return [int(np.random.Generator(np.random.PCG64(seed0 + k)).integers(n_min, n_max + 1))
            for k in range(n_graphs)]


def make_batch(n_graphs=256, seed0=1000, n_min=100, n_max=5000, window=15,
               kf_per_loop=400, noise=(0.01, 0.02, 0.01), only=None):
    """The batched workload: ``n_graphs`` independent figure-8 graphs with
    keyframe counts drawn uniformly from [n_min, n_max], covisibility window
    ``window`` and one loop edge per ``kf_per_loop`` keyframes.  Graph k uses
    seed ``seed0 + k`` for both its size and its noise.  ``only``: build just
    these graph indices (same graphs as in the full batch)."""
    sizes = batch_sizes(n_graphs, seed0, n_min, n_max)
    out = []
    for k in (range(n_graphs) if only is None else only):
        n = sizes[k]
        loops = max(1, n // kf_per_loop)
        out.append(make_graph("figure8", n, seed=seed0 + k, window=window,
                              n_loops=loops, noise=noise, name=f"batch{k}"))
    return out


class LoopCorrection:
    """Inputs of the loop-correction steps around the pose graph optimisation
    of one graph (see make_loop_correction)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def make_loop_correction(g, points_per_kf=150, seed=0, depth=(1.0, 8.0), half_angle=0.6):
    """Synthetic inputs of the loop-correction steps for graph ``g``:

    current    the keyframe that closed the loop: the later end of the graph's
               last loop edge (the last keyframe if it has none);
    matched    the loop edge's other end (keyframe 0 if none);
    corrected  the Sim(3) pose of ``current`` that the loop detection would
               estimate, consistent with the matched keyframe:
               S_c' = (S_c^gt (S_m^gt)^-1) S_m (exact relative pose);
    connected  ``current`` and every keyframe sharing an edge with it;
    points     ``points_per_kf`` map points per keyframe, (P, 3) world
               coordinates, created in the keyframe's camera frame at its
               drifted estimate (depth uniform in ``depth``, direction within
               ``half_angle`` rad of the optical axis z);
    ref        (P,) int32 reference keyframe of each point.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = g.n_vertices
    if g.n_loop_edges > 0:
        a, b = int(g.edge_i[-1]), int(g.edge_j[-1])
        current, matched = max(a, b), min(a, b)
    else:
        current, matched = n - 1, 0
    rel = compose(g.poses_gt[current], inverse(g.poses_gt[matched]))
    corrected = compose(rel, g.poses_init[matched])
    corrected[0:4] /= np.linalg.norm(corrected[0:4])
    nb = np.concatenate([g.edge_j[g.edge_i == current], g.edge_i[g.edge_j == current]])
    connected = np.unique(np.concatenate([[current], nb])).astype(np.int32)
    P = n * points_per_kf
    ref = np.repeat(np.arange(n, dtype=np.int32), points_per_kf)
    d = rng.uniform(depth[0], depth[1], P)
    ang = rng.uniform(0.0, half_angle, P)
    az = rng.uniform(0.0, 2.0 * np.pi, P)
    pc = np.stack([d * np.sin(ang) * np.cos(az), d * np.sin(ang) * np.sin(az), d * np.cos(ang)], axis=1)
    S = g.poses_init[ref]
    Sinv = inverse(S)
    X = Sinv[:, 7:8] * quat_rotate(Sinv[:, 0:4], pc) + Sinv[:, 4:7]
    return LoopCorrection(current=current, matched=matched, corrected=np.ascontiguousarray(corrected),
                          connected=connected, points=np.ascontiguousarray(X), ref=ref)


# --------------------------------------------------------------------------
# Projection search and loop fusion workloads (keyframe features, map points)
# --------------------------------------------------------------------------
class MatchWorkload:
    """Keyframes with ORB-like features and map points to match against them
    (see make_match_workload); arrays in the layout of pgo_frames_create and
    pgo_project_match."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


CAMERA = dict(fx=460.0, fy=460.0, cx=376.0, cy=240.0, min_x=0.0, max_x=752.0, min_y=0.0, max_y=480.0)


def _rand_desc(rng, n):
    return rng.integers(0, 2 ** 32, size=(n, 8), dtype=np.uint64).astype(np.uint32)


def _flip_bits(rng, desc, nflip):
    out = desc.copy()
    for i in range(desc.shape[0]):
        bits = rng.choice(256, int(nflip[i]), replace=False)
        for b in bits:
            out[i, b // 32] ^= np.uint32(1) << np.uint32(b % 32)
    return out


def _camera_centre(S):
    Si = inverse(S)
    return Si[..., 4:7]


def _project(S, X, cam):
    pc = S[..., 7:8] * quat_rotate(S[..., 0:4], X) + S[..., 4:7]
    u = cam["fx"] * pc[..., 0] / pc[..., 2] + cam["cx"]
    v = cam["fy"] * pc[..., 1] / pc[..., 2] + cam["cy"]
    return u, v, pc[..., 2]


def make_match_workload(mode="search", n_kf=3, n_points=4000, features_per_kf=1200, seed=0,
                        n_levels=8, scale_factor=1.2, detect=0.7, pixel_noise=1.0, max_flips=30,
                        matched_frac=0.1, duplicate_frac=0.5, observed_frac=0.02):
    """Synthetic keyframes on the figure-8 trajectory (752 x 480 camera,
    ~``features_per_kf`` features each over ``n_levels`` octaves) and
    ``n_points`` map points around them.

    Every map point has a random 256-bit descriptor, a creation distance d0
    and level l0 (max_dist = d0 scale^l0 times a factor in [1.02, 1.15], off
    the level boundaries; min_dist = max_dist / scale^(n_levels-1)) and a
    viewing direction.  A keyframe detects a fraction ``detect`` of the
    points in its view as features at the projection plus Gaussian pixel
    noise, with the point's descriptor after up to ``max_flips`` random bit
    flips and the octave its distance predicts; random clutter features fill
    the rest.  mode 'search' (projection search, PS1 with n_kf = 1, PS3a-c
    with n_kf = 3): keyframe poses are Sim(3) with a random scale, and a
    fraction ``matched_frac`` of each keyframe's features is marked as matched
    before the search.  mode 'fusion': the points are the loop side's map
    points; a fraction ``duplicate_frac`` of the detected ones are already in
    the keyframe's map under another id (the duplicates loop fusion finds),
    and a fraction ``observed_frac`` is observed by the keyframe itself.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cam = CAMERA
    c, f = _figure8(400)
    gt = _poses_from_path(c, f)
    k0 = int(rng.integers(0, 400 - n_kf * 3))
    kf_idx = k0 + 2 * np.arange(n_kf)
    S = gt[kf_idx].copy()
    # points in front of the keyframes: created from the first keyframe's view and its neighbours
    creators = kf_idx[rng.integers(0, n_kf, n_points)]
    Sc = gt[creators]
    d0 = rng.uniform(2.0, 12.0, n_points)
    ang = rng.uniform(0.0, 0.55, n_points)
    az = rng.uniform(0.0, 2.0 * np.pi, n_points)
    pc = np.stack([d0 * np.sin(ang) * np.cos(az), d0 * np.sin(ang) * np.sin(az), d0 * np.cos(ang)], axis=1)
    Sci = inverse(Sc)
    X = Sci[:, 7:8] * quat_rotate(Sci[:, 0:4], pc) + Sci[:, 4:7]
    Oc = _camera_centre(Sc)
    nrm = X - Oc
    dist0 = np.linalg.norm(nrm, axis=1)
    nrm /= dist0[:, None]
    l0 = rng.integers(0, 3, n_points)
    # a margin keeps the creating keyframe's own distance off a level boundary
    max_dist = dist0 * scale_factor ** l0 * rng.uniform(1.02, 1.15, n_points)
    min_dist = max_dist / scale_factor ** (n_levels - 1)
    pdesc = _rand_desc(rng, n_points)
    pid = np.arange(n_points, dtype=np.int32) + 100000
    feat_ptr = [0]
    fu, fv, foct, fdesc, fskip, fmp = [], [], [], [], [], []
    truth = []
    for k in range(n_kf):
        u, v, z = _project(S[k][None], X, cam)
        O = _camera_centre(S[k])
        d = np.linalg.norm(X - O, axis=1)
        inview = (z > 0) & (u >= 0) & (u < cam["max_x"]) & (v >= 0) & (v < cam["max_y"])
        inview &= (d >= min_dist) & (d <= max_dist)
        inview &= np.einsum("ij,ij->i", X - O, nrm) >= 0.5 * d     # viewing angle within 60 degrees
        det = np.nonzero(inview & (rng.random(n_points) < detect))[0][: int(features_per_kf * 0.8)]
        lev = np.zeros(len(det), dtype=np.int32)
        for i, p in enumerate(det):
            L = 0
            while L < n_levels - 1 and max_dist[p] > d[p] * scale_factor ** L:
                L += 1
            lev[i] = L
        lev = np.maximum(lev - rng.integers(0, 2, len(det)), 0).astype(np.int32)
        nu = (u[det] + rng.normal(0.0, pixel_noise, len(det))).clip(0.0, cam["max_x"] - 1e-3)
        nv = (v[det] + rng.normal(0.0, pixel_noise, len(det))).clip(0.0, cam["max_y"] - 1e-3)
        dd = _flip_bits(rng, pdesc[det], rng.integers(0, max_flips + 1, len(det)))
        ncl = max(0, features_per_kf - len(det))
        cu = rng.uniform(0.0, cam["max_x"], ncl)
        cv = rng.uniform(0.0, cam["max_y"], ncl)
        co = rng.integers(0, n_levels, ncl).astype(np.int32)
        cd = _rand_desc(rng, ncl)
        mp = np.full(len(det) + ncl, -1, dtype=np.int32)
        if mode == "fusion":
            dup = rng.random(len(det)) < duplicate_frac
            mp[: len(det)][dup] = det[dup].astype(np.int32) + 500000      # the other side's id of the same point
            own = rng.random(len(det)) < observed_frac
            mp[: len(det)][own] = pid[det[own]]
        uu = np.concatenate([nu, cu]).astype(np.float32)
        vv = np.concatenate([nv, cv]).astype(np.float32)
        oo = np.concatenate([lev, co]).astype(np.int32)
        de = np.concatenate([dd, cd]).astype(np.uint32)
        perm = rng.permutation(len(uu))
        fu.append(uu[perm]); fv.append(vv[perm]); foct.append(oo[perm]); fdesc.append(de[perm]); fmp.append(mp[perm])
        sk = (rng.random(len(uu)) < matched_frac).astype(np.uint8) if mode == "search" else np.zeros(len(uu), np.uint8)
        fskip.append(sk)
        inv = np.empty(len(uu), dtype=np.int64)
        inv[perm] = np.arange(len(uu))
        truth.append(dict(points=det, features=inv[: len(det)]))
        feat_ptr.append(feat_ptr[-1] + len(uu))
    if mode == "search":   # Sim(3) poses: same projections, scaled camera frame
        s = rng.uniform(0.8, 1.25, n_kf)
        S[:, 4:7] *= s[:, None]
        S[:, 7] = s
    return MatchWorkload(
        mode=mode, camera=dict(cam), n_levels=n_levels, scale_factor=scale_factor,
        poses=np.ascontiguousarray(S), feat_ptr=np.array(feat_ptr, dtype=np.int32),
        fu=np.concatenate(fu), fv=np.concatenate(fv), foct=np.concatenate(foct),
        fdesc=np.ascontiguousarray(np.concatenate(fdesc)), fskip=np.concatenate(fskip), fmp=np.concatenate(fmp),
        points=np.ascontiguousarray(X, dtype=np.float32), pdesc=pdesc, min_dist=min_dist.astype(np.float32),
        max_dist=max_dist.astype(np.float32), normal=np.ascontiguousarray(nrm, dtype=np.float32), pid=pid,
        truth=truth)
