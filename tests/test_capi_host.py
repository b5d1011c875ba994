"""CPU-side checks of the C ABI: the library builds and loads, exports every
symbol the header declares, and rejects bad graph descriptions before any
device work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2603_17201_gb300 import _lib as L
from paper_2603_17201_gb300 import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return L.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "pgo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pgo_[a-z_0-9]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    names = header_functions()
    assert len(names) >= 16
    assert sorted(L.EXPORTED) == names
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_defaults(lib):
    assert b"sm_103a" in lib.pgo_version()
    o = L.default_options()
    assert o.max_iters == 20 and o.precision == L.PGO_FP64 and o.tau == 1e-5
    assert o.pcg_tol == 1e-6 and o.refine_steps >= 1


def _desc(n, ei, ej, meas, fixed=0, weight=None, poses=None, info=None):
    keep = []
    d = L.GraphDesc()
    d.n_vertices = n
    d.n_edges = len(ei)
    d.fixed_vertex = fixed
    d.mem_space = L.PGO_MEM_HOST
    ei = np.ascontiguousarray(ei, dtype=np.int32)
    ej = np.ascontiguousarray(ej, dtype=np.int32)
    meas = np.ascontiguousarray(meas, dtype=np.float64)
    keep += [ei, ej, meas]
    d.edge_i = ei.ctypes.data
    d.edge_j = ej.ctypes.data
    d.meas = meas.ctypes.data
    if weight is not None:
        w = np.ascontiguousarray(weight, dtype=np.float64)
        keep.append(w)
        d.weight = w.ctypes.data
    if poses is not None:
        p = np.ascontiguousarray(poses, dtype=np.float64)
        keep.append(p)
        d.poses = p.ctypes.data
    if info is not None:
        om = np.ascontiguousarray(info, dtype=np.float64)
        keep.append(om)
        d.info = om.ctypes.data
    return d, keep


@pytest.mark.parametrize("case", ["index", "self_edge", "nan_meas", "bad_scale", "zero_quat", "bad_fixed",
                                  "neg_edges", "neg_weight", "nan_pose", "info_not_spd"])
def test_create_rejects_bad_graphs(lib, case):
    g = syn.make_graph("circle", 20, seed=1)
    ei, ej, meas, fixed, n, w = g.edge_i.copy(), g.edge_j.copy(), g.meas.copy(), 0, g.n_vertices, None
    poses, info = None, None
    if case == "index":
        ej[3] = n
    elif case == "self_edge":
        ej[5] = ei[5]
    elif case == "nan_meas":
        meas[2, 5] = np.nan
    elif case == "bad_scale":
        meas[1, 7] = -1.0
    elif case == "zero_quat":
        meas[4, :4] = 0.0
    elif case == "bad_fixed":
        fixed = n
    elif case == "neg_weight":
        w = np.ones(len(ei))
        w[0] = -1.0
    elif case == "nan_pose":
        poses = g.poses_init.copy()
        poses[7, 4] = np.inf
    elif case == "info_not_spd":
        info = np.tile(np.eye(7), (len(ei), 1, 1))
        info[6, 3, 3] = -1.0
    d, keep = _desc(n, ei, ej, meas, fixed, w, poses, info)
    if case == "neg_edges":
        d.n_edges = -1
    h = ctypes.c_void_p()
    st = lib.pgo_graph_create(ctypes.byref(d), ctypes.byref(h))
    assert st == L.PGO_ERR_INVALID_ARG
    assert h.value is None
    assert len(lib.pgo_last_error()) > 0


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.pgo_graph_create(None, ctypes.byref(h)) == L.PGO_ERR_INVALID_ARG
    assert lib.pgo_default_options(None) == L.PGO_ERR_INVALID_ARG
    assert lib.pgo_solve(None, None, None, None, 0) == L.PGO_ERR_INVALID_ARG
    assert lib.pgo_evaluate_cost(-1, 0, None, None, None, None, None, None, None, None) == L.PGO_ERR_INVALID_ARG
    lib.pgo_graph_destroy(None)


def test_allocation_limit_gives_oom_and_no_handle(lib):
    """The device-allocation test hook: graph creation needs more than the
    limit, so it fails with PGO_ERR_OOM before touching the device, and the
    handle stays NULL (no GPU needed: the check precedes every CUDA call)."""
    g = syn.make_graph("circle", 40, seed=2)
    d, keep = _desc(g.n_vertices, g.edge_i, g.edge_j, g.meas)
    lib.pgo_test_set_alloc_limit.argtypes = [ctypes.c_size_t]
    lib.pgo_test_set_alloc_limit.restype = None
    lib.pgo_test_set_alloc_limit(4096)
    try:
        h = ctypes.c_void_p()
        st = lib.pgo_graph_create(ctypes.byref(d), ctypes.byref(h))
        assert st == L.PGO_ERR_OOM
        assert h.value is None
        assert b"exceeds the test limit" in lib.pgo_last_error()
    finally:
        lib.pgo_test_set_alloc_limit(0)


@pytest.mark.parametrize("case", ["no_keyframes", "bounds", "ptr_order", "nan_uv"])
def test_frames_create_rejects_bad_input(lib, case):
    """pgo_frames_create validates on the host before any device work."""
    K, F = 2, 6
    ptr = np.array([0, 3, 6], np.int32)
    uv = np.zeros((F, 2), np.float32)
    oct_ = np.zeros(F, np.int32)
    desc = np.zeros((F, 8), np.uint32)
    d = L.FramesDesc()
    d.n_keyframes = K
    d.mem_space = L.PGO_MEM_HOST
    d.min_x, d.max_x, d.min_y, d.max_y = 0.0, 752.0, 0.0, 480.0
    if case == "no_keyframes":
        d.n_keyframes = 0
    elif case == "bounds":
        d.max_x = 0.0
    elif case == "ptr_order":
        ptr[1] = 7
    elif case == "nan_uv":
        uv[4, 1] = np.nan
    d.feat_ptr = ptr.ctypes.data
    d.uv = uv.ctypes.data
    d.octave = oct_.ctypes.data
    d.desc = desc.ctypes.data
    h = ctypes.c_void_p()
    assert lib.pgo_frames_create(ctypes.byref(d), ctypes.byref(h)) == L.PGO_ERR_INVALID_ARG
    assert h.value is None
