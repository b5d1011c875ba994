"""Failure paths of the C ABI on the GPU, each made on the host side or by a
bounded wait that runs out; none faults, traps or hangs the device:

  - the device-allocation limit gives PGO_ERR_OOM and a NULL handle;
  - a PCG iteration cap gives PGO_ERR_NOT_CONVERGED (delta still written);
  - non-finite device poses make the solve stop with PGO_ERR_NUMERICAL;
  - a PCG block that never arrives at its grid barrier (test hook) makes the
    other blocks give up after the 1 ms wait limit, and the solve reports
    PGO_ERR_CUDA; a fresh graph then solves normally;
  - the stateless cost counts the edges it skips (bad index or self-edge).
"""
import ctypes
import time

import numpy as np
import pytest

from paper_2603_17201_gb300 import _lib as L
from paper_2603_17201_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    lib = L.load()
    lib.pgo_test_set_alloc_limit.argtypes = [ctypes.c_size_t]
    lib.pgo_test_set_alloc_limit.restype = None
    lib.pgo_test_set_barrier.argtypes = [ctypes.c_double, ctypes.c_int]
    lib.pgo_test_set_barrier.restype = None
    return lib


def PG(g, **kw):
    from paper_2603_17201_gb300 import PoseGraph
    return PoseGraph.from_synthetic(g, **kw)


def test_alloc_limit_gives_oom(lib):
    from paper_2603_17201_gb300 import PGOError
    g = syn.make_config("c1_circle200")
    lib.pgo_test_set_alloc_limit(1 << 16)
    try:
        with pytest.raises(PGOError) as ei:
            PG(g)
        assert ei.value.status == L.PGO_ERR_OOM
    finally:
        lib.pgo_test_set_alloc_limit(0)
    pg = PG(g)   # the limit is off again
    assert pg.solve(max_iters=3)["status"] == 0


@pytest.mark.parametrize("precond", ["block_jacobi", "multigrid"])
def test_pcg_cap_gives_not_converged(lib, precond):
    g = syn.make_config("c1_circle200")
    pg = PG(g)
    o = L.default_options(pcg_max_iters=2, preconditioner=precond)
    d = np.full((g.n_vertices, 7), np.nan)
    it = ctypes.c_int32()
    st = lib.pgo_graph_damped_step(pg._h, ctypes.byref(o), 1e-3, ctypes.c_void_p(d.ctypes.data),
                                   ctypes.byref(it), L.PGO_MEM_HOST)
    assert st == L.PGO_ERR_NOT_CONVERGED, lib.pgo_last_error()
    assert b"pcg_max_iters" in lib.pgo_last_error()
    assert it.value == 2
    assert np.all(np.isfinite(d)) and np.abs(d).max() > 0   # the capped iterate is still written


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonfinite_device_poses_give_numerical(lib, precision):
    from paper_2603_17201_gb300 import PGOError
    g = syn.make_config("c1_circle200")
    pg = PG(g)
    bad = g.poses_init.copy()
    bad[17, 5] = np.nan
    pg.set_poses(torch.as_tensor(bad, device="cuda"))   # device copy: no host validation
    with pytest.raises(PGOError) as ei:
        pg.solve(precision=precision)
    assert ei.value.status == L.PGO_ERR_NUMERICAL
    rep = L.Report()
    assert lib.pgo_graph_report(pg._h, ctypes.byref(rep)) == L.PGO_ERR_NUMERICAL
    assert rep.stop_reason == 4 and rep.iterations == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_barrier_wait_limit_reports_cuda_error(lib, precision):
    from paper_2603_17201_gb300 import PGOError
    g = syn.make_config("c1_circle200")
    pg = PG(g)
    lib.pgo_test_set_barrier(1e-3, 1)   # block 1 of every PCG launch never arrives
    try:
        t0 = time.perf_counter()
        with pytest.raises(PGOError) as ei:
            pg.solve(precision=precision, max_iters=5)
        dt = time.perf_counter() - t0
    finally:
        lib.pgo_test_set_barrier(0.0, -1)
    assert ei.value.status == L.PGO_ERR_CUDA
    assert dt < 5.0, dt   # the 1 ms limit, not the 2 s default, ended the wait
    pg.close()
    # the context stays usable: a fresh graph solves to the usual result
    pg2 = PG(g)
    rep = pg2.solve(precision=precision)
    assert rep["status"] == 0 and rep["final_cost"] < rep["initial_cost"]


def test_stateless_cost_counts_skipped_edges(lib):
    from paper_2603_17201_gb300 import evaluate_cost
    import oracle as O
    g = syn.make_config("c1_circle200")
    ei, ej = g.edge_i.copy(), g.edge_j.copy()
    ei[3] = g.n_vertices        # out of range
    ej[10] = ei[10]             # self-edge
    ei[20] = -1                 # negative
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    c, bad = evaluate_cost(g.n_vertices, t(ei, torch.int32), t(ej, torch.int32), t(g.meas), None,
                           t(g.poses_init), return_bad=True)
    assert int(bad.item()) == 3
    keep = np.ones(g.n_edges, bool)
    keep[[3, 10, 20]] = False
    og = O.OracleGraph(g.n_vertices, g.edge_i[keep], g.edge_j[keep], g.meas[keep], None, None, 0)
    ref = og.cost(g.poses_init)
    assert abs(c.item() - ref) <= 1e-13 * ref
    c2, bad2 = evaluate_cost(g.n_vertices, t(g.edge_i, torch.int32), t(g.edge_j, torch.int32), t(g.meas), None,
                             t(g.poses_init), return_bad=True)
    assert int(bad2.item()) == 0
