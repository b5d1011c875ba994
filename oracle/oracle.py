"""ctypes wrapper of the plain FP64 C oracle (``pgo_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  The product path
(the CUDA library and its Python binding) never calls it and has no CPU
fallback.

The oracle follows the paper's problem statement (Sec. III-B and IV-F: pose
graph optimisation of the Sim(3) essential graph with Levenberg-Marquardt and
an exact sparse factorisation of the normal equations) with the readings
listed at the top of ``pgo_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

__all__ = ["build", "load", "OracleGraph", "exp", "log", "W", "left_jacobian", "adj",
           "compose", "inverse", "LMOptions", "LMReport"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pgo_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class LMOptions(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("tau", ctypes.c_double),
                ("lambda_init", ctypes.c_double), ("ftol", ctypes.c_double),
                ("gtol", ctypes.c_double), ("polish_iters", ctypes.c_int)]


class LMReport(ctypes.Structure):
    _fields_ = [("initial_cost", ctypes.c_double), ("final_cost", ctypes.c_double),
                ("final_lambda", ctypes.c_double), ("grad_inf_norm", ctypes.c_double),
                ("iterations", ctypes.c_int), ("accepted", ctypes.c_int),
                ("stop_reason", ctypes.c_int), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ProjParams(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("min_x", ctypes.c_float), ("max_x", ctypes.c_float), ("min_y", ctypes.c_float),
                ("max_y", ctypes.c_float), ("scale_factor", ctypes.c_float), ("th", ctypes.c_float),
                ("cos_min", ctypes.c_float), ("n_levels", ctypes.c_int), ("th_low", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: -O2, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                                   "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    lib.og_create.restype = ctypes.c_void_p
    lib.og_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _ip, _dp, _dp, _dp]
    lib.og_destroy.argtypes = [ctypes.c_void_p]
    lib.og_factor_nnz.restype = ctypes.c_int64
    lib.og_factor_nnz.argtypes = [ctypes.c_void_p]
    for name in ("og_exp", "og_log", "og_left_jacobian", "og_adj", "og_inverse"):
        getattr(lib, name).argtypes = [_dp, _dp]
    lib.og_W.argtypes = [_dp, ctypes.c_double, _dp]
    lib.og_compose.argtypes = [_dp, _dp, _dp]
    lib.og_cost.restype = ctypes.c_double
    lib.og_cost.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.og_jacobians.restype = ctypes.c_int
    lib.og_jacobians.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
    lib.og_linearize.restype = ctypes.c_double
    lib.og_linearize.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
    lib.og_solve_system.restype = ctypes.c_int
    lib.og_solve_system.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_double, _dp]
    lib.og_apply_update.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
    lib.og_lm.restype = ctypes.c_int
    lib.og_lm.argtypes = [ctypes.c_void_p, _dp, ctypes.POINTER(LMOptions), ctypes.POINTER(LMReport)]
    lib.og_adjoint.restype = ctypes.c_int
    lib.og_adjoint.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_double, _dp, _dp, _dp]
    lib.og_pose_loss.restype = ctypes.c_double
    lib.og_pose_loss.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
    lib.og_propagate_correction.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int, _ip, _dp]
    lib.og_correct_points.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _ip, _dp]
    vp = ctypes.c_void_p
    lib.og_project_match.argtypes = [ctypes.POINTER(ProjParams), ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp,
                                     vp, vp, vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    _lib = lib
    return lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- group ops
def exp(xi):
    """exp of xi = [omega, upsilon, sigma] -> pose (qx,qy,qz,qw,tx,ty,tz,s)."""
    xi = _f64(xi, (7,))
    out = np.zeros(8)
    load().og_exp(_d(xi), _d(out))
    return out


def log(pose):
    pose = _f64(pose, (8,))
    out = np.zeros(7)
    load().og_log(_d(pose), _d(out))
    return out


def W(omega, sigma):
    """The V matrix sum_n (omega^ + sigma I)^n / (n+1)! (3x3)."""
    omega = _f64(omega, (3,))
    out = np.zeros(9)
    load().og_W(_d(omega), float(sigma), _d(out))
    return out.reshape(3, 3)


def left_jacobian(xi):
    xi = _f64(xi, (7,))
    out = np.zeros(49)
    load().og_left_jacobian(_d(xi), _d(out))
    return out.reshape(7, 7)


def adj(pose):
    pose = _f64(pose, (8,))
    out = np.zeros(49)
    load().og_adj(_d(pose), _d(out))
    return out.reshape(7, 7)


def compose(a, b):
    a, b = _f64(a, (8,)), _f64(b, (8,))
    out = np.zeros(8)
    load().og_compose(_d(a), _d(b), _d(out))
    return out


def inverse(a):
    a = _f64(a, (8,))
    out = np.zeros(8)
    load().og_inverse(_d(a), _d(out))
    return out


# ---------------------------------------------------------------- graph
class OracleGraph:
    """An essential graph held by the oracle (edges, measurements, weights,
    optional 7x7 information matrices and the fixed gauge vertex)."""

    def __init__(self, n_vertices, edge_i, edge_j, meas, weight=None, info=None, fixed_vertex=0):
        lib = load()
        self.n = int(n_vertices)
        self.ei = np.ascontiguousarray(edge_i, dtype=np.int32)
        self.ej = np.ascontiguousarray(edge_j, dtype=np.int32)
        self.m = int(self.ei.shape[0])
        self.meas = _f64(meas, (self.m, 8))
        self.weight = None if weight is None else _f64(weight, (self.m,))
        self.info = None if info is None else _f64(info, (self.m, 49))
        self.fixed = int(fixed_vertex)
        wp = _d(self.weight) if self.weight is not None else None
        ip = _d(self.info) if self.info is not None else None
        self._h = lib.og_create(self.n, self.m, self.fixed, self.ei.ctypes.data_as(_ip),
                                self.ej.ctypes.data_as(_ip), _d(self.meas), wp, ip)
        if not self._h:
            raise ValueError("oracle rejected the graph (bad sizes, indices or a self-edge)")

    @classmethod
    def from_synthetic(cls, g, **kw):
        return cls(g.n_vertices, g.edge_i, g.edge_j, g.meas, g.weight, None, g.fixed_vertex, **kw)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.og_destroy(h)
            self._h = None

    def factor_nnz(self):
        return int(load().og_factor_nnz(self._h))

    def cost(self, poses, residuals=False):
        poses = _f64(poses, (self.n, 8))
        r = np.zeros((self.m, 7)) if residuals else None
        F = load().og_cost(self._h, _d(poses), _d(r) if residuals else None)
        return (F, r) if residuals else F

    def jacobians(self, poses):
        poses = _f64(poses, (self.n, 8))
        Ai = np.zeros((self.m, 7, 7))
        Aj = np.zeros((self.m, 7, 7))
        rc = load().og_jacobians(self._h, _d(poses), _d(Ai), _d(Aj))
        if rc:
            raise RuntimeError("singular left Jacobian")
        return Ai, Aj

    def linearize(self, poses):
        """-> (F, Hdiag (N,7,7), Hoff (E,7,7) the (i,j) block per edge, b (N,7))."""
        poses = _f64(poses, (self.n, 8))
        Hd = np.zeros((self.n, 7, 7))
        Ho = np.zeros((self.m, 7, 7))
        b = np.zeros((self.n, 7))
        F = load().og_linearize(self._h, _d(poses), _d(Hd), _d(Ho), _d(b))
        return F, Hd, Ho, b

    def solve_system(self, Hdiag, Hoff, b, lam):
        """Exact (H + lam I) delta = -b on the free vertices (delta_fixed = 0)."""
        Hd = _f64(Hdiag, (self.n, 49))
        Ho = _f64(Hoff, (self.m, 49))
        bb = _f64(b, (self.n, 7))
        d = np.zeros((self.n, 7))
        rc = load().og_solve_system(self._h, _d(Hd), _d(Ho), _d(bb), float(lam), _d(d))
        if rc:
            raise RuntimeError(f"sparse Cholesky failed ({rc})")
        return d

    def apply_update(self, poses, delta):
        poses = _f64(poses, (self.n, 8))
        delta = _f64(delta, (self.n, 7))
        out = np.zeros((self.n, 8))
        load().og_apply_update(self._h, _d(poses), _d(delta), _d(out))
        return out

    def lm(self, poses, max_iters=20, tau=1e-5, lambda_init=0.0, ftol=1e-14, gtol=1e-13,
           polish_iters=0):
        """Run LM from ``poses``; returns (optimised poses, report dict).
        ``polish_iters`` > 0 adds gradient-decreasing undamped Gauss-Newton
        steps after LM (a stationary point to full precision)."""
        p = _f64(poses, (self.n, 8)).copy()
        opt = LMOptions(int(max_iters), float(tau), float(lambda_init), float(ftol), float(gtol),
                        int(polish_iters))
        rep = LMReport()
        load().og_lm(self._h, _d(p), ctypes.byref(opt), ctypes.byref(rep))
        return p, rep.as_dict()

    def adjoint(self, poses, dL_dx, h=1e-5):
        """Implicit-adjoint gradients at an optimum: (dL/dmeas (E,7) in the
        left tangent of each measurement, dL/dweight (E,), mu (N,7))."""
        poses = _f64(poses, (self.n, 8))
        g = _f64(dL_dx, (self.n, 7))
        dz = np.zeros((self.m, 7))
        dw = np.zeros(self.m)
        mu = np.zeros((self.n, 7))
        rc = load().og_adjoint(self._h, _d(poses), _d(g), float(h), _d(dz), _d(dw), _d(mu))
        if rc:
            raise RuntimeError(f"full Hessian not positive definite ({rc})")
        return dz, dw, mu

    def pose_loss(self, poses, gt):
        """L = 1/2 sum_{v != fixed} |log(S_v G_v^-1)|^2 and dL/d(delta) (N,7)."""
        poses = _f64(poses, (self.n, 8))
        gt = _f64(gt, (self.n, 8))
        grad = np.zeros((self.n, 7))
        L = load().og_pose_loss(self._h, _d(poses), _d(gt), _d(grad))
        return L, grad


def pose_error(a, b):
    """Per-vertex |log(a_v b_v^-1)| for two (N, 8) pose arrays."""
    a = _f64(a)
    b = _f64(b)
    out = np.empty(a.shape[0])
    for v in range(a.shape[0]):
        out[v] = np.linalg.norm(log(compose(a[v], inverse(b[v]))))
    return out


__all__ += ["pose_error"]


# ---------------------------------------------------------------- loop correction
def propagate_correction(poses, current, corrected, connected):
    """Loop correction before the pose graph optimisation (Sec. III-B): the
    keyframes in ``connected`` take S_k' = (S_k S_c^-1) S_c' with S_c' =
    ``corrected`` the new pose of keyframe ``current``; others are copied.
    Returns the (N, 8) pose array."""
    poses = _f64(poses)
    n = poses.shape[0]
    conn = np.ascontiguousarray(connected, dtype=np.int32)
    corr = _f64(corrected, (8,))
    out = np.empty((n, 8))
    load().og_propagate_correction(n, _d(poses), int(current), _d(corr), int(conn.shape[0]),
                                   conn.ctypes.data_as(_ip), _d(out))
    return out


def correct_points(before, after, points, ref):
    """Map-point correction (Sec. III-B): x' = S_after[r]^-1 (S_before[r] x)
    through each point's reference keyframe r (r < 0: unchanged).  Returns
    the (P, 3) array."""
    before = _f64(before)
    after = _f64(after, before.shape)
    X = _f64(points)
    P = X.shape[0]
    X = X.reshape(P, 3)
    r = np.ascontiguousarray(ref, dtype=np.int32)
    out = np.empty((P, 3))
    load().og_correct_points(before.shape[0], _d(before), _d(after), P, _d(X), r.ctypes.data_as(_ip), _d(out))
    return out


__all__ += ["propagate_correction", "correct_points"]


# ---------------------------------------------------------------- projection search / loop fusion
def proj_params(camera, n_levels=8, scale_factor=1.2, th=10.0, cos_min=0.5, th_low=50):
    p = ProjParams()
    for k in ("fx", "fy", "cx", "cy", "min_x", "max_x", "min_y", "max_y"):
        setattr(p, k, float(camera[k]))
    p.scale_factor = float(scale_factor)
    p.th = float(th)
    p.cos_min = float(cos_min)
    p.n_levels = int(n_levels)
    p.th_low = int(th_low)
    return p


def project_match(w, mode, th=10.0, th_low=50, cos_min=0.5, poses=None):
    """Projection search (mode 'search') or loop fusion ('fusion') of the map
    points of workload ``w`` against its keyframes (Sec. IV-D), in single
    precision: returns (match, dist, fuse) as (K, P) int32 arrays (fuse None
    for the search)."""
    pp = proj_params(w.camera, w.n_levels, w.scale_factor, th, cos_min, th_low)
    K = len(w.feat_ptr) - 1
    P = w.points.shape[0]
    m = 0 if mode == "search" else 1
    poses = _f64(w.poses if poses is None else poses, (K, 8))
    arrs = dict(ptr=np.ascontiguousarray(w.feat_ptr, np.int32), fu=np.ascontiguousarray(w.fu, np.float32),
                fv=np.ascontiguousarray(w.fv, np.float32), fo=np.ascontiguousarray(w.foct, np.int32),
                fd=np.ascontiguousarray(w.fdesc, np.uint32), fs=np.ascontiguousarray(w.fskip, np.uint8),
                fm=np.ascontiguousarray(w.fmp, np.int32), X=np.ascontiguousarray(w.points, np.float32).reshape(P, 3),
                pd=np.ascontiguousarray(w.pdesc, np.uint32), mn=np.ascontiguousarray(w.min_dist, np.float32),
                mx=np.ascontiguousarray(w.max_dist, np.float32),
                nr=np.ascontiguousarray(w.normal, np.float32).reshape(P, 3), pid=np.ascontiguousarray(w.pid, np.int32))
    match = np.empty((K, P), np.int32)
    dist = np.empty((K, P), np.int32)
    fuse = np.empty((K, P), np.int32) if m == 1 else None
    a = {k: v.ctypes.data for k, v in arrs.items()}
    load().og_project_match(ctypes.byref(pp), m, K, poses.ctypes.data, a["ptr"], a["fu"], a["fv"], a["fo"], a["fd"],
                            a["fs"] if m == 0 else None, a["fm"], P, a["X"], a["pd"], a["mn"], a["mx"], a["nr"],
                            a["pid"], match.ctypes.data, dist.ctypes.data, fuse.ctypes.data if m == 1 else None)
    return match, dist, fuse


__all__ += ["ProjParams", "proj_params", "project_match"]
