"""GPU test of pgo_evaluate_cost_noalloc, the cost evaluation that allocates
no device memory.

Callers such as a real-time loop-closing thread (which must not stall on the
device allocator mid-frame) or an application that reserves its whole device
memory budget at start-up cannot let a library allocate on each call; this
entry point serves them from a fixed workspace compiled into the library.
The test calls it through the C ABI twice in a row and checks each result
against pgo_evaluate_cost, which gets its workspace from the stream-ordered
allocator, within the 1e-13 relative tolerance the cost tests use.  It runs
last in the suite (file name) and also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _graph_tensors(seed):
    from paper_2603_17201_gb300 import synthetic as syn
    g = syn.make_graph("figure8", 1500, seed=seed, window=12, n_loops=3, meas_noise=True)
    dev = torch.device("cuda", 0)
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    w = np.random.default_rng(seed).uniform(0.5, 2.0, g.n_edges)
    return g, t(g.edge_i, torch.int32), t(g.edge_j, torch.int32), t(g.meas), t(w), t(g.poses_init)


def test_noalloc_matches_allocating_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_17201_gb300 import _lib
    lib = _lib.load()
    torch.cuda.set_device(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda x: ctypes.c_void_p(x.data_ptr())  # noqa: E731
    for seed in (5, 6):   # two calls in a row, different inputs
        g, ei, ej, meas, w, poses = _graph_tensors(seed)
        ref = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        got = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.pgo_evaluate_cost(g.n_vertices, g.n_edges, ptr(ei), ptr(ej), ptr(meas), ptr(w), ptr(poses),
                                   ptr(ref), stream)
        assert st == 0, lib.pgo_last_error()
        st = lib.pgo_evaluate_cost_noalloc(g.n_vertices, g.n_edges, ptr(ei), ptr(ej), ptr(meas), ptr(w),
                                           ptr(poses), ptr(got), stream)
        assert st == 0, lib.pgo_last_error()
        torch.cuda.synchronize()
        r, v = ref.item(), got.item()
        assert np.isfinite(r) and r > 0
        assert abs(v - r) <= 1e-13 * r, (v, r)


def test_noalloc_rejects_sizes_beyond_its_workspace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_17201_gb300 import _lib
    lib = _lib.load()
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    st = lib.pgo_evaluate_cost_noalloc(10, 1_048_577, None, None, None, None, None,
                                       ctypes.c_void_p(out.data_ptr()), None)
    assert st == _lib.PGO_ERR_INVALID_ARG
    assert b"workspace limit" in lib.pgo_last_error()
