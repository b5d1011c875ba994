"""GPU test of pgo_evaluate_cost_noalloc, the cost evaluation that allocates
no device memory.

Callers such as a real-time loop-closing thread (which must not stall on the
device allocator mid-frame) or an application that reserves its whole device
memory budget at start-up cannot let a library allocate on each call; this
entry point serves them from a fixed workspace compiled into the library.
The test calls it through the C ABI twice in a row and checks each result
against pgo_evaluate_cost, which gets its workspace from the stream-ordered
allocator, within the 1e-13 relative tolerance the cost tests use, and
against the FP64 oracle's cost of the same graph.  A second case uses about
600k edges, where the fixed-workspace launch runs more thread blocks (one per
256 edges) than the allocating one (at most 1,024, grid-stride), so the two
sum in different orders: 1e-12 relative there.  It runs last in the suite
(file name) and also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _graph_tensors(seed, n=1500, window=12):
    from paper_2603_17201_gb300 import synthetic as syn
    g = syn.make_graph("figure8", n, seed=seed, window=window, n_loops=3, meas_noise=True)
    dev = torch.device("cuda", 0)
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    w = np.random.default_rng(seed).uniform(0.5, 2.0, g.n_edges)
    return g, w, t(g.edge_i, torch.int32), t(g.edge_j, torch.int32), t(g.meas), t(w), t(g.poses_init)


def _both(lib, g, ei, ej, meas, w, poses):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda x: ctypes.c_void_p(x.data_ptr())  # noqa: E731
    ref = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    got = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    bad_ref = torch.full((), -1, dtype=torch.int32, device="cuda")
    bad_got = torch.full((), -1, dtype=torch.int32, device="cuda")
    st = lib.pgo_evaluate_cost(g.n_vertices, g.n_edges, ptr(ei), ptr(ej), ptr(meas), ptr(w), ptr(poses),
                               ptr(ref), ptr(bad_ref), stream)
    assert st == 0, lib.pgo_last_error()
    st = lib.pgo_evaluate_cost_noalloc(g.n_vertices, g.n_edges, ptr(ei), ptr(ej), ptr(meas), ptr(w),
                                       ptr(poses), ptr(got), ptr(bad_got), stream)
    assert st == 0, lib.pgo_last_error()
    torch.cuda.synchronize()
    assert int(bad_ref.item()) == 0 and int(bad_got.item()) == 0
    return ref.item(), got.item()


def test_noalloc_matches_allocating_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_17201_gb300 import _lib
    lib = _lib.load()
    torch.cuda.set_device(0)
    for seed in (5, 6):   # two calls in a row, different inputs
        g, w_h, ei, ej, meas, w, poses = _graph_tensors(seed)
        r, v = _both(lib, g, ei, ej, meas, w, poses)
        assert np.isfinite(r) and r > 0
        assert abs(v - r) <= 1e-13 * r, (v, r)
        F = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, w_h, None, 0).cost(g.poses_init)
        assert abs(v - F) <= 1e-13 * F, (v, F)


def test_noalloc_beyond_the_allocating_launch_width():
    """~600k edges: 2,300+ blocks in the fixed-workspace launch against 1,024
    in the allocating one (different summation order)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_17201_gb300 import _lib
    lib = _lib.load()
    torch.cuda.set_device(0)
    g, w_h, ei, ej, meas, w, poses = _graph_tensors(11, n=40000, window=15)
    assert 262_144 < g.n_edges <= 1_048_576
    for _ in range(2):
        r, v = _both(lib, g, ei, ej, meas, w, poses)
        assert abs(v - r) <= 1e-12 * r, (v, r)
    F = O.OracleGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, w_h, None, 0).cost(g.poses_init)
    assert abs(v - F) <= 1e-12 * F, (v, F)


def test_noalloc_rejects_sizes_beyond_its_workspace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_17201_gb300 import _lib
    lib = _lib.load()
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    st = lib.pgo_evaluate_cost_noalloc(10, 1_048_577, None, None, None, None, None,
                                       ctypes.c_void_p(out.data_ptr()), None, None)
    assert st == _lib.PGO_ERR_INVALID_ARG
    assert b"workspace limit" in lib.pgo_last_error()
