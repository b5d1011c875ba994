"""Host logic of graph creation and of the multigrid hierarchy, without a
GPU: the library's internal edge order, incidence lists and host analysis
(through a test hook of the C library) against a plain Python construction
of the same arrays from their definitions.

  - level 0: the vertices; aggregates of 4 consecutive free vertices (the
    gauge vertex has none); level l + 1: one node per aggregate, 4 consecutive
    nodes each, until at most 8 nodes remain;
  - P's pattern: row u holds the aggregates of u and of its neighbours;
  - A P's pattern: row u holds the union of the P rows of u and its
    neighbours;
  - the next level's operator P^T A P: row c holds every d with c in P(u)
    and d in AP(u) for some u, stored with the diagonal first, then the
    columns below it, then those above, each ascending.
"""
import ctypes
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2603_17201_gb300 import _lib as L  # noqa: E402
from paper_2603_17201_gb300 import synthetic as syn  # noqa: E402

LEVELS, AGG, P_PTR, P_COL, AP_PTR, AP_COL, A_PTR, A_COL = range(8)


@pytest.fixture(scope="module")
def lib():
    lib = L.load()
    f = lib.pgo_test_multigrid_plan
    f.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
    f.restype = ctypes.c_int
    return lib


def plan_array(lib, n, ei, ej, fixed, level, what):
    ei = np.ascontiguousarray(ei, np.int32)
    ej = np.ascontiguousarray(ej, np.int32)
    cnt = ctypes.c_int64(0)
    st = lib.pgo_test_multigrid_plan(n, len(ei), ei.ctypes.data, ej.ctypes.data, fixed, level, what, None,
                                     ctypes.byref(cnt))
    assert st == 0, lib.pgo_last_error()
    out = np.zeros(max(cnt.value, 1), np.int32)
    st = lib.pgo_test_multigrid_plan(n, len(ei), ei.ctypes.data, ej.ctypes.data, fixed, level, what,
                                     out.ctypes.data, ctypes.byref(cnt))
    assert st == 0, lib.pgo_last_error()
    return out[:cnt.value]


def csr_rows(ptr, col):
    return [list(col[ptr[u]:ptr[u + 1]]) for u in range(len(ptr) - 1)]


def reference(n, ei, ej, fixed):
    """Per level: aggregates, P rows, A P rows, and the next level's operator
    rows in the library's storage order."""
    nbrs = [{u} for u in range(n)]
    for i, j in zip(ei, ej):
        nbrs[i].add(int(j))
        nbrs[j].add(int(i))
    free = [u != fixed for u in range(n)]
    agg, k = [], 0
    for u in range(n):
        agg.append(k // 4 if free[u] else -1)
        k += free[u]
    levels = []
    while True:
        m = len(nbrs)
        P = [sorted({agg[w] for w in nbrs[u] if agg[w] >= 0}) if agg[u] >= 0 else [] for u in range(m)]
        AP = [sorted(set().union(*[set(P[w]) for w in nbrs[u] if agg[w] >= 0])) if agg[u] >= 0 else []
              for u in range(m)]
        nc = max(agg) + 1
        rows = [set() for _ in range(nc)]
        for u in range(m):
            for c in P[u]:
                rows[c].update(AP[u])
        A = [[c] + sorted(d for d in rows[c] if d < c) + sorted(d for d in rows[c] if d > c) for c in range(nc)]
        levels.append(dict(n=m, agg=agg, P=P, AP=AP, A_next=A))
        if nc <= 8:
            return levels, nc
        nbrs = [set(r) for r in rows]
        agg = [c // 4 for c in range(nc)]


def graphs():
    g1 = syn.make_config("c1_circle200")
    g2 = syn.make_graph("figure8", 300, seed=12, window=8, n_loops=2, meas_noise=True, loop_min_gap=100,
                        loop_max_dist=3.0)
    g3 = syn.make_graph("circle", 61, seed=5, window=3, n_loops=1, loop_min_gap=30, loop_max_dist=100.0)
    # duplicate edges and a gauge vertex in the middle
    ei = np.concatenate([g3.edge_i, g3.edge_i[:5]])
    ej = np.concatenate([g3.edge_j, g3.edge_j[:5]])
    return [("c1_circle200", g1.n_vertices, g1.edge_i, g1.edge_j, 0),
            ("figure8_300", g2.n_vertices, g2.edge_i, g2.edge_j, 0),
            ("circle61_duplicates_mid_gauge", g3.n_vertices, ei, ej, 30)]


@pytest.mark.parametrize("case", graphs(), ids=lambda c: c[0])
def test_analysis_matches_the_definitions(lib, case):
    _, n, ei, ej, fixed = case
    ref, n_coarsest = reference(n, ei, ej, fixed)
    sizes = list(plan_array(lib, n, ei, ej, fixed, 0, LEVELS))
    assert sizes == [lv["n"] for lv in ref] + [n_coarsest]
    for lvl, lv in enumerate(ref):
        assert list(plan_array(lib, n, ei, ej, fixed, lvl, AGG)) == lv["agg"]
        assert csr_rows(plan_array(lib, n, ei, ej, fixed, lvl, P_PTR),
                        plan_array(lib, n, ei, ej, fixed, lvl, P_COL)) == lv["P"]
        assert csr_rows(plan_array(lib, n, ei, ej, fixed, lvl, AP_PTR),
                        plan_array(lib, n, ei, ej, fixed, lvl, AP_COL)) == lv["AP"]
        assert csr_rows(plan_array(lib, n, ei, ej, fixed, lvl + 1, A_PTR),
                        plan_array(lib, n, ei, ej, fixed, lvl + 1, A_COL)) == lv["A_next"]


def test_hook_rejects_bad_input(lib):
    cnt = ctypes.c_int64(0)
    ei = np.array([0, 1], np.int32)
    ej = np.array([1, 5], np.int32)   # 5 is out of range for 4 vertices
    st = lib.pgo_test_multigrid_plan(4, 2, ei.ctypes.data, ej.ctypes.data, 0, 0, LEVELS, None, ctypes.byref(cnt))
    assert st == L.PGO_ERR_INVALID_ARG
    ej[1] = 2
    st = lib.pgo_test_multigrid_plan(4, 2, ei.ctypes.data, ej.ctypes.data, 0, 9, AGG, None, ctypes.byref(cnt))
    assert st == L.PGO_ERR_INVALID_ARG   # no level 9


PERM, INC_PTR, INC_SPLIT, INC_CODE, INC_OTHER = range(8, 13)


@pytest.mark.parametrize("case", graphs(), ids=lambda c: c[0])
def test_edge_order_and_incidence(lib, case):
    """Graph creation's internal edge order is by (min endpoint, max endpoint,
    caller index); each vertex lists the edges where it is i (side 0), then
    those where it is j (side 1), each group in internal edge order, as codes
    2 k + side with the other endpoint beside them."""
    _, n, ei, ej, fixed = case
    ei, ej = np.asarray(ei, np.int64), np.asarray(ej, np.int64)
    E = len(ei)
    order = sorted(range(E), key=lambda e: (min(ei[e], ej[e]), max(ei[e], ej[e]), e))
    assert list(plan_array(lib, n, ei, ej, fixed, 0, PERM)) == order
    rows = [([], []) for _ in range(n)]
    for k, e in enumerate(order):
        rows[ei[e]][0].append((2 * k, ej[e]))
        rows[ej[e]][1].append((2 * k + 1, ei[e]))
    ptr, split, code, other = [0], [], [], []
    for side0, side1 in rows:
        split.append(ptr[-1] + len(side0))
        for c, o in side0 + side1:
            code.append(c)
            other.append(o)
        ptr.append(len(code))
    assert list(plan_array(lib, n, ei, ej, fixed, 0, INC_PTR)) == ptr
    assert list(plan_array(lib, n, ei, ej, fixed, 0, INC_SPLIT)) == split
    assert list(plan_array(lib, n, ei, ej, fixed, 0, INC_CODE)) == code
    assert list(plan_array(lib, n, ei, ej, fixed, 0, INC_OTHER)) == other
