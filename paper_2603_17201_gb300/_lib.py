"""ctypes declarations of the C ABI in ``include/pgo.h`` (argument marshalling
only: every step of the solve runs in the CUDA library)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_int32 = ctypes.c_int32
c_double = ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)

PGO_OK = 0
PGO_ERR_INVALID_ARG = 1
PGO_ERR_OOM = 2
PGO_ERR_CUDA = 3
PGO_ERR_NUMERICAL = 4
PGO_ERR_NOT_CONVERGED = 5
PGO_ERR_STATE = 6
STATUS_NAMES = {0: "PGO_OK", 1: "PGO_ERR_INVALID_ARG", 2: "PGO_ERR_OOM", 3: "PGO_ERR_CUDA",
                4: "PGO_ERR_NUMERICAL", 5: "PGO_ERR_NOT_CONVERGED", 6: "PGO_ERR_STATE"}

PGO_FP64 = 0
PGO_MIXED = 1
PGO_MEM_HOST = 0
PGO_MEM_DEVICE = 1
PGO_GRAD_TANGENT7 = 0
PGO_GRAD_POSE8 = 1

# Every exported symbol the header declares (checked by the CPU test-suite).
EXPORTED = [
    "pgo_last_error", "pgo_version", "pgo_default_options", "pgo_graph_create", "pgo_graph_destroy",
    "pgo_graph_set_poses", "pgo_graph_set_measurements", "pgo_graph_get_poses", "pgo_graph_cost", "pgo_graph_linearize",
    "pgo_graph_damped_step", "pgo_graph_resolve", "pgo_graph_report", "pgo_solve", "pgo_backward", "pgo_batch_create", "pgo_batch_destroy",
    "pgo_batch_solve", "pgo_batch_schedule", "pgo_evaluate_cost", "pgo_evaluate_cost_noalloc",
    "pgo_graph_multigrid_info", "pgo_graph_multigrid_export", "pgo_graph_precondition", "pgo_propagate_correction", "pgo_correct_points",
    "pgo_frames_create", "pgo_frames_destroy", "pgo_project_match",
]


class GraphDesc(ctypes.Structure):
    _fields_ = [("n_vertices", c_int32), ("n_edges", c_int32), ("fixed_vertex", c_int32),
                ("mem_space", c_int32), ("edge_i", ctypes.c_void_p), ("edge_j", ctypes.c_void_p),
                ("meas", ctypes.c_void_p), ("weight", ctypes.c_void_p), ("info", ctypes.c_void_p),
                ("poses", ctypes.c_void_p), ("stream", ctypes.c_void_p)]


class SolveOptions(ctypes.Structure):
    _fields_ = [("max_iters", c_int32), ("precision", c_int32), ("tau", c_double),
                ("lambda_init", c_double), ("ftol", c_double), ("gtol", c_double),
                ("pcg_tol", c_double), ("pcg_max_iters", c_int32), ("refine_steps", c_int32),
                ("refine_tol", c_double), ("polish_iters", c_int32), ("schedule", c_int32),
                ("preconditioner", c_int32), ("multigrid_refresh", c_int32), ("linear_solver", c_int32)]


class FramesDesc(ctypes.Structure):
    _fields_ = [("n_keyframes", c_int32), ("mem_space", c_int32), ("feat_ptr", ctypes.c_void_p),
                ("uv", ctypes.c_void_p), ("octave", ctypes.c_void_p), ("desc", ctypes.c_void_p),
                ("map_point", ctypes.c_void_p), ("min_x", ctypes.c_float), ("max_x", ctypes.c_float),
                ("min_y", ctypes.c_float), ("max_y", ctypes.c_float), ("stream", ctypes.c_void_p)]


class MatchParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("fx", "fy", "cx", "cy", "min_x", "max_x", "min_y", "max_y",
                                                "scale_factor", "th", "cos_min")] + [("n_levels", c_int32),
                                                                                     ("th_low", c_int32)]


class PointsDesc(ctypes.Structure):
    _fields_ = [("n_points", c_int32), ("xyz", ctypes.c_void_p), ("desc", ctypes.c_void_p),
                ("min_dist", ctypes.c_void_p), ("max_dist", ctypes.c_void_p), ("normal", ctypes.c_void_p),
                ("id", ctypes.c_void_p)]


PGO_MATCH_SEARCH = 0
PGO_MATCH_FUSE = 1


class Report(ctypes.Structure):
    _fields_ = [("initial_cost", c_double), ("final_cost", c_double), ("final_lambda", c_double),
                ("grad_inf_norm", c_double), ("iterations", c_int32), ("accepted", c_int32),
                ("pcg_iterations", c_int32), ("stop_reason", c_int32), ("status", c_int32),
                ("ms_total", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PGOError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it in-tree first if it is missing or
    stale).  Raises if it cannot be built or loaded: there is no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library {_build.LIB} is missing; run paper_2603_17201_gb300.build")
        lib = ctypes.CDLL(_build.LIB)
        vp = ctypes.c_void_p
        lib.pgo_last_error.restype = ctypes.c_char_p
        lib.pgo_version.restype = ctypes.c_char_p
        lib.pgo_default_options.argtypes = [ctypes.POINTER(SolveOptions)]
        lib.pgo_graph_create.argtypes = [ctypes.POINTER(GraphDesc), ctypes.POINTER(vp)]
        lib.pgo_graph_destroy.argtypes = [vp]
        lib.pgo_graph_destroy.restype = None
        lib.pgo_graph_set_poses.argtypes = [vp, vp, c_int32]
        lib.pgo_graph_get_poses.argtypes = [vp, vp, c_int32]
        lib.pgo_graph_set_measurements.argtypes = [vp, vp, vp, c_int32]
        lib.pgo_graph_cost.argtypes = [vp, _dp, vp, c_int32]
        lib.pgo_graph_linearize.argtypes = [vp, c_int32, vp, vp, vp, vp, c_int32]
        lib.pgo_graph_damped_step.argtypes = [vp, ctypes.POINTER(SolveOptions), c_double, vp,
                                              ctypes.POINTER(c_int32), c_int32]
        lib.pgo_graph_resolve.argtypes = [vp, ctypes.POINTER(SolveOptions), c_double, vp,
                                          ctypes.POINTER(c_int32), c_int32]
        lib.pgo_graph_report.argtypes = [vp, ctypes.POINTER(Report)]
        lib.pgo_propagate_correction.argtypes = [c_int32, vp, c_int32, vp, c_int32, vp, vp, vp, vp]
        lib.pgo_correct_points.argtypes = [c_int32, vp, vp, c_int32, vp, vp, vp, vp, vp]
        lib.pgo_frames_create.argtypes = [ctypes.POINTER(FramesDesc), ctypes.POINTER(vp)]
        lib.pgo_frames_destroy.argtypes = [vp]
        lib.pgo_frames_destroy.restype = None
        lib.pgo_project_match.argtypes = [vp, ctypes.POINTER(MatchParams), c_int32, vp, vp, ctypes.POINTER(PointsDesc),
                                          vp, vp, vp]
        lib.pgo_graph_precondition.argtypes = [vp, ctypes.POINTER(SolveOptions), c_double]
        lib.pgo_graph_multigrid_info.argtypes = [vp, ctypes.POINTER(c_int32), vp, vp, vp, vp]
        lib.pgo_graph_multigrid_export.argtypes = [vp, c_int32, c_int32, c_int32, vp, ctypes.c_int64,
                                                   ctypes.POINTER(ctypes.c_int64)]
        lib.pgo_solve.argtypes = [vp, ctypes.POINTER(SolveOptions), ctypes.POINTER(Report), vp, c_int32]
        lib.pgo_backward.argtypes = [vp, ctypes.POINTER(SolveOptions), vp, c_int32, vp, vp, c_int32]
        lib.pgo_batch_create.argtypes = [c_int32, ctypes.POINTER(GraphDesc), vp, ctypes.POINTER(vp)]
        lib.pgo_batch_destroy.argtypes = [vp]
        lib.pgo_batch_destroy.restype = None
        lib.pgo_batch_solve.argtypes = [vp, ctypes.POINTER(SolveOptions), ctypes.POINTER(Report), vp, c_int32]
        lib.pgo_batch_schedule.argtypes = [vp, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                           ctypes.POINTER(c_int32), ctypes.POINTER(ctypes.c_float)]
        lib.pgo_evaluate_cost.argtypes = [c_int32, c_int32, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.pgo_evaluate_cost_noalloc.argtypes = [c_int32, c_int32, vp, vp, vp, vp, vp, vp, vp, vp]
        for name in EXPORTED:
            fn = getattr(lib, name)
            if name not in ("pgo_last_error", "pgo_version", "pgo_graph_destroy", "pgo_batch_destroy",
                            "pgo_frames_destroy"):
                fn.restype = ctypes.c_int
        _lib = lib
        return lib


def check(status: int):
    if status != PGO_OK:
        msg = _lib.pgo_last_error().decode() if _lib is not None else ""
        raise PGOError(status, msg)


def default_options(**overrides) -> SolveOptions:
    lib = load()
    o = SolveOptions()
    check(lib.pgo_default_options(ctypes.byref(o)))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": PGO_FP64, "mixed": PGO_MIXED}[v.lower()]
        if k == "linear_solver" and isinstance(v, str):
            v = {"pcg": 0, "direct": 1, "auto": 2}[v.lower()]
        if k == "preconditioner" and isinstance(v, str):
            v = {"block_jacobi": 0, "jacobi": 0, "multigrid": 1, "amg": 1}[v.lower()]
        if not hasattr(o, k):
            raise TypeError(f"unknown solve option {k!r}")
        setattr(o, k, v)
    return o


# pgo_mg_array codes of pgo_graph_multigrid_export (integer arrays first)
MG_ARRAYS = {"a_ptr": 0, "a_col": 1, "a": 2, "p_ptr": 3, "p_col": 4, "p": 5, "ap_ptr": 6, "ap_col": 7, "q": 8,
             "dinv": 9, "t": 10, "agg": 11, "rho": 12, "w": 13}
MG_INT_ARRAYS = {"a_ptr", "a_col", "p_ptr", "p_col", "ap_ptr", "ap_col", "agg"}
