"""Python binding of the GB300 Sim(3) essential-graph optimiser.

Thin marshalling over the C ABI (``include/pgo.h``): arrays go in as host
numpy arrays or torch tensors (CUDA tensors are passed as device pointers on
the current torch stream), and every computation runs in the CUDA library.
The problem is the pose graph optimisation step of loop correction
(Sec. III-B, Sec. IV-F): Levenberg-Marquardt over keyframe Sim(3) poses with
one fixed gauge keyframe.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L

__all__ = ["PoseGraph", "PoseGraphBatch", "evaluate_cost", "default_options", "PGOError", "solve_pose_graph",
           "propagate_correction", "correct_points", "Frames", "match_params"]

PGOError = L.PGOError
default_options = L.default_options


def _torch():
    import torch
    return torch


def _is_cuda_tensor(x):
    try:
        torch = _torch()
    except Exception:  # pragma: no cover - torch is a hard dependency of the package
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


def _current_stream_handle():
    torch = _torch()
    if torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


class _Marshal:
    """Holds host or device copies of a set of arrays in one memory space."""

    def __init__(self, device: bool):
        self.device = device
        self.keep = []

    def put(self, x, dtype, shape=None):
        if x is None:
            return None
        if self.device:
            torch = _torch()
            tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
            t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x, dtype=dtype))
            t = t.to(device="cuda", dtype=tdt).contiguous()
            if shape is not None:
                t = t.reshape(shape)
            self.keep.append(t)
            return ctypes.c_void_p(t.data_ptr())
        if not isinstance(x, np.ndarray):
            try:
                x = x.detach().cpu().numpy()
            except AttributeError:
                x = np.asarray(x)
        a = np.ascontiguousarray(x, dtype=dtype)
        if shape is not None:
            a = a.reshape(shape)
        self.keep.append(a)
        return ctypes.c_void_p(a.ctypes.data)

    @property
    def mem_space(self):
        return L.PGO_MEM_DEVICE if self.device else L.PGO_MEM_HOST


class PoseGraph:
    """A device-resident essential graph (see ``pgo_graph_create``).

    n_vertices, edge_i, edge_j (E,), meas (E, 8) pose8 of Z_ij ~ S_j S_i^-1,
    weight (E,) or None, info (E, 7, 7) or None, poses (N, 8) or None,
    fixed_vertex (the gauge keyframe)."""

    def __init__(self, n_vertices, edge_i, edge_j, meas, weight=None, info=None, poses=None,
                 fixed_vertex=0, stream=None):
        self._lib = L.load()
        self._h = ctypes.c_void_p()
        device = any(_is_cuda_tensor(x) for x in (edge_i, edge_j, meas, weight, info, poses))
        m = _Marshal(device)
        E = int(len(edge_i))
        d = L.GraphDesc()
        d.n_vertices = int(n_vertices)
        d.n_edges = E
        d.fixed_vertex = int(fixed_vertex)
        d.mem_space = m.mem_space
        d.edge_i = m.put(edge_i, np.int32)
        d.edge_j = m.put(edge_j, np.int32)
        d.meas = m.put(meas, np.float64, (E, 8))
        d.weight = m.put(weight, np.float64, (E,))
        d.info = m.put(info, np.float64, (E, 49))
        d.poses = m.put(poses, np.float64, (int(n_vertices), 8))
        if device:
            _torch().cuda.current_stream().synchronize()
        d.stream = stream if stream is not None else _current_stream_handle()
        L.check(self._lib.pgo_graph_create(ctypes.byref(d), ctypes.byref(self._h)))
        self.n_vertices = int(n_vertices)
        self.n_edges = E
        self.fixed_vertex = int(fixed_vertex)

    @classmethod
    def from_synthetic(cls, g, poses=None, **kw):
        """From a ``synthetic.PoseGraph``; the initial estimate is its drifted
        chain unless ``poses`` is given."""
        return cls(g.n_vertices, g.edge_i, g.edge_j, g.meas, g.weight, None,
                   g.poses_init if poses is None else poses, g.fixed_vertex, **kw)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.pgo_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- state
    def set_poses(self, poses):
        """Replace the current estimate.  A CUDA tensor is copied on the
        graph's stream (it must be ready on that stream); host arrays are
        validated and copied synchronously."""
        m = _Marshal(_is_cuda_tensor(poses))
        p = m.put(poses, np.float64, (self.n_vertices, 8))
        L.check(self._lib.pgo_graph_set_poses(self._h, p, m.mem_space))
        self._keep = m.keep

    def set_measurements(self, meas, weight=None):
        """Replace the edge measurements (E, 8) and optionally the weights (E,)
        (caller's edge order).  CUDA tensors are copied on the graph's stream."""
        dev = _is_cuda_tensor(meas) or _is_cuda_tensor(weight)
        m = _Marshal(dev)
        pm = m.put(meas, np.float64, (self.n_edges, 8))
        pw = m.put(weight, np.float64, (self.n_edges,))
        L.check(self._lib.pgo_graph_set_measurements(self._h, pm, pw, m.mem_space))
        self._keep_meas = m.keep

    def backward(self, dL_dposes, layout="pose8", meas_grad=True, weight_grad=True, **opts):
        """Implicit-adjoint gradients of the last solve (see pgo_backward).
        dL_dposes: (N, 8) for layout 'pose8' or (N, 7) for 'tangent'.
        Returns (dL/dmeas (E, 8 or 7), dL/dweight (E,)) as CUDA tensors when
        dL_dposes is a CUDA tensor, else numpy arrays."""
        lay = L.PGO_GRAD_POSE8 if layout == "pose8" else L.PGO_GRAD_TANGENT7
        w = 8 if lay == L.PGO_GRAD_POSE8 else 7
        o = L.default_options(**opts)
        if _is_cuda_tensor(dL_dposes):
            torch = _torch()
            g = dL_dposes.to(torch.float64).contiguous()
            dm = torch.empty((self.n_edges, w), dtype=torch.float64, device=g.device) if meas_grad else None
            dw = torch.empty((self.n_edges,), dtype=torch.float64, device=g.device) if weight_grad else None
            ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
            L.check(self._lib.pgo_backward(self._h, ctypes.byref(o), ptr(g), lay, ptr(dm), ptr(dw),
                                           L.PGO_MEM_DEVICE))
            return dm, dw
        g = np.ascontiguousarray(dL_dposes, dtype=np.float64)
        dm = np.empty((self.n_edges, w)) if meas_grad else None
        dw = np.empty(self.n_edges) if weight_grad else None
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None  # noqa: E731
        L.check(self._lib.pgo_backward(self._h, ctypes.byref(o), ptr(g), lay, ptr(dm), ptr(dw), L.PGO_MEM_HOST))
        return dm, dw

    def get_poses(self, device=False):
        """Current estimate (N, 8): a CUDA tensor if ``device`` else numpy."""
        if device:
            torch = _torch()
            out = torch.empty((self.n_vertices, 8), dtype=torch.float64, device="cuda")
            L.check(self._lib.pgo_graph_get_poses(self._h, ctypes.c_void_p(out.data_ptr()), L.PGO_MEM_DEVICE))
            return out
        out = np.empty((self.n_vertices, 8))
        L.check(self._lib.pgo_graph_get_poses(self._h, ctypes.c_void_p(out.ctypes.data), L.PGO_MEM_HOST))
        return out

    def cost(self, residuals=False):
        """F at the current estimate (and the (E, 7) residuals)."""
        c = ctypes.c_double()
        r = np.empty((self.n_edges, 7)) if residuals else None
        L.check(self._lib.pgo_graph_cost(self._h, ctypes.byref(c),
                                         ctypes.c_void_p(r.ctypes.data) if residuals else None,
                                         L.PGO_MEM_HOST))
        return (c.value, r) if residuals else c.value

    # ---------------------------------------------------------------- steps
    def linearize(self, precision="fp64", jacobians=True):
        """Normal equations at the current estimate (FP64 copies):
        dict(jac (E,2,7,7), h_diag (N,7,7), h_off (E,7,7), b (N,7))."""
        prec = L.PGO_MIXED if str(precision).lower() == "mixed" else L.PGO_FP64
        N, E = self.n_vertices, self.n_edges
        jac = np.empty((E, 2, 7, 7)) if jacobians else None
        hd = np.empty((N, 7, 7))
        ho = np.empty((E, 7, 7))
        b = np.empty((N, 7))
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None  # noqa: E731
        L.check(self._lib.pgo_graph_linearize(self._h, prec, ptr(jac), ptr(hd), ptr(ho), ptr(b), L.PGO_MEM_HOST))
        out = dict(h_diag=hd, h_off=ho, b=b)
        if jacobians:
            out["jac"] = jac
        return out

    def damped_step(self, lam, **opts):
        """Solve (H + lam I) delta = -b at the current estimate with PCG.
        Returns (delta (N, 7), PCG iterations); raises on the iteration cap
        unless ``allow_cap=True``."""
        allow_cap = opts.pop("allow_cap", False)
        o = L.default_options(**opts)
        d = np.empty((self.n_vertices, 7))
        it = ctypes.c_int32()
        st = self._lib.pgo_graph_damped_step(self._h, ctypes.byref(o), float(lam),
                                             ctypes.c_void_p(d.ctypes.data), ctypes.byref(it), L.PGO_MEM_HOST)
        if not (allow_cap and st == L.PGO_ERR_NOT_CONVERGED):
            L.check(st)
        return d, int(it.value)

    def resolve(self, lam, **opts):
        """Re-solve the damped system at the last linearisation for a new
        lambda.  Returns (delta (N, 7), PCG iterations)."""
        allow_cap = opts.pop("allow_cap", False)
        o = L.default_options(**opts)
        d = np.empty((self.n_vertices, 7))
        it = ctypes.c_int32()
        st = self._lib.pgo_graph_resolve(self._h, ctypes.byref(o), float(lam), ctypes.c_void_p(d.ctypes.data),
                                         ctypes.byref(it), L.PGO_MEM_HOST)
        if not (allow_cap and st == L.PGO_ERR_NOT_CONVERGED):
            L.check(st)
        return d, int(it.value)

    def resolve_async(self, lam, **opts):
        """Enqueue a re-solve on the graph's stream (no synchronisation)."""
        o = L.default_options(**opts)
        L.check(self._lib.pgo_graph_resolve(self._h, ctypes.byref(o), float(lam), None, None, L.PGO_MEM_HOST))

    def precondition_async(self, lam, **opts):
        """Enqueue the preconditioner set-up at the last linearisation for
        ``lam`` on the graph's stream (no synchronisation)."""
        o = L.default_options(**opts)
        L.check(self._lib.pgo_graph_precondition(self._h, ctypes.byref(o), float(lam)))

    def multigrid_info(self):
        """Shape of the multigrid hierarchy: list of dicts (nodes, blocks of
        the operator, of P and of A P) per level, the coarsest last."""
        n = ctypes.c_int32()
        nodes = np.zeros(13, np.int32)
        a, p, ap = (np.zeros(13, np.int64) for _ in range(3))
        L.check(self._lib.pgo_graph_multigrid_info(self._h, ctypes.byref(n), ctypes.c_void_p(nodes.ctypes.data),
                                                   ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(p.ctypes.data),
                                                   ctypes.c_void_p(ap.ctypes.data)))
        return [dict(nodes=int(nodes[k]), a_blocks=int(a[k]), p_blocks=int(p[k]), ap_blocks=int(ap[k]))
                for k in range(n.value)]

    def multigrid_export(self, level, name, precision="fp64"):
        """One array of the multigrid hierarchy's last set-up in `precision`
        (pgo_graph_multigrid_export): int32 arrays for patterns and
        aggregates, float64 otherwise (7x7 blocks as (n, 7, 7))."""
        which = L.MG_ARRAYS[name]
        prec = L.PGO_MIXED if str(precision).lower() == "mixed" else L.PGO_FP64
        cnt = ctypes.c_int64()
        L.check(self._lib.pgo_graph_multigrid_export(self._h, int(level), which, prec, None, 0, ctypes.byref(cnt)))
        is_int = name in L.MG_INT_ARRAYS
        out = np.zeros(cnt.value, np.int32 if is_int else np.float64)
        L.check(self._lib.pgo_graph_multigrid_export(self._h, int(level), which, prec, ctypes.c_void_p(out.ctypes.data),
                                                     out.nbytes, ctypes.byref(cnt)))
        if not is_int and name != "rho":
            out = out.reshape(-1, 7, 7)
        return out

    def solve_report(self):
        """Report of the last solve (synchronises the graph's stream)."""
        rep = L.Report()
        L.check(self._lib.pgo_graph_report(self._h, ctypes.byref(rep)))
        return rep.as_dict()

    def solve(self, poses_out=None, **opts):
        """Levenberg-Marquardt from the current estimate; returns the report
        dict.  ``poses_out``: optional (N, 8) numpy array or CUDA tensor."""
        o = L.default_options(**opts)
        rep = L.Report()
        if poses_out is None:
            L.check(self._lib.pgo_solve(self._h, ctypes.byref(o), ctypes.byref(rep), None, L.PGO_MEM_HOST))
        elif _is_cuda_tensor(poses_out):
            L.check(self._lib.pgo_solve(self._h, ctypes.byref(o), ctypes.byref(rep),
                                        ctypes.c_void_p(poses_out.data_ptr()), L.PGO_MEM_DEVICE))
        else:
            assert poses_out.dtype == np.float64 and poses_out.flags.c_contiguous
            L.check(self._lib.pgo_solve(self._h, ctypes.byref(o), ctypes.byref(rep),
                                        ctypes.c_void_p(poses_out.ctypes.data), L.PGO_MEM_HOST))
        return rep.as_dict()

    def solve_async(self, **opts):
        """Enqueue a solve on the graph's stream without reading a report."""
        o = L.default_options(**opts)
        L.check(self._lib.pgo_solve(self._h, ctypes.byref(o), None, None, L.PGO_MEM_HOST))


class PoseGraphBatch:
    """Many independent essential graphs solved together (see
    ``pgo_batch_create`` / ``pgo_batch_solve``): one persistent launch in
    which each thread block solves whole graphs."""

    def __init__(self, graphs, stream=None):
        """graphs: sequence of synthetic.PoseGraph-like objects (n_vertices,
        edge_i, edge_j, meas, weight, poses_init, fixed_vertex)."""
        self._lib = L.load()
        self._h = ctypes.c_void_p()
        n = len(graphs)
        descs = (L.GraphDesc * n)()
        m = _Marshal(False)
        self.sizes = []
        for k, g in enumerate(graphs):
            d = descs[k]
            E = int(len(g.edge_i))
            d.n_vertices = int(g.n_vertices)
            d.n_edges = E
            d.fixed_vertex = int(getattr(g, "fixed_vertex", 0))
            d.mem_space = L.PGO_MEM_HOST
            d.edge_i = m.put(g.edge_i, np.int32)
            d.edge_j = m.put(g.edge_j, np.int32)
            d.meas = m.put(g.meas, np.float64, (E, 8))
            d.weight = m.put(getattr(g, "weight", None), np.float64, (E,))
            d.poses = m.put(getattr(g, "poses_init", None), np.float64, (int(g.n_vertices), 8))
            self.sizes.append((int(g.n_vertices), E))
        s = stream if stream is not None else _current_stream_handle()
        L.check(self._lib.pgo_batch_create(n, descs, s, ctypes.byref(self._h)))
        self.n_graphs = n

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.pgo_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, poses=True, **opts):
        """Solve every graph; returns (list of report dicts, list of (N_k, 8)
        numpy pose arrays or None)."""
        o = L.default_options(**opts)
        reps = (L.Report * self.n_graphs)()
        outs = [np.empty((nv, 8)) for nv, _ in self.sizes] if poses else None
        ptrs = (ctypes.c_void_p * self.n_graphs)(*[o_.ctypes.data for o_ in outs]) if poses else None
        L.check(self._lib.pgo_batch_solve(self._h, ctypes.byref(o), reps, ptrs, L.PGO_MEM_HOST))
        return [r.as_dict() for r in reps], outs

    def solve_async(self, **opts):
        o = L.default_options(**opts)
        L.check(self._lib.pgo_batch_solve(self._h, ctypes.byref(o), None, None, L.PGO_MEM_HOST))

    def schedule(self):
        """(lanes per block row, threads per block, blocks per SM, autotuner
        best trial ms)."""
        lanes, threads, bps, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        L.check(self._lib.pgo_batch_schedule(self._h, ctypes.byref(lanes), ctypes.byref(threads), ctypes.byref(bps),
                                             ctypes.byref(ms)))
        return lanes.value, threads.value, bps.value, ms.value


class _SolveFunction:
    """Holder for the torch.autograd.Function (built lazily so that the
    module imports without torch)."""
    fn = None

    @classmethod
    def get(cls):
        if cls.fn is not None:
            return cls.fn
        torch = _torch()

        class PoseGraphSolve(torch.autograd.Function):
            """poses* = argmin_S F(S; Z, w): forward runs the LM solve (with
            Newton polishing), backward the implicit adjoint (pgo_backward)."""

            @staticmethod
            def forward(ctx, meas, weight, graph, poses0, opts):
                graph.set_measurements(meas.detach(), weight.detach())
                graph.set_poses(poses0.detach())
                out = torch.empty((graph.n_vertices, 8), dtype=torch.float64, device=meas.device)
                ctx.report = graph.solve(poses_out=out, **opts)
                ctx.graph = graph
                ctx.opts = {k: v for k, v in opts.items() if k in ("pcg_tol", "pcg_max_iters")}
                return out

            @staticmethod
            def backward(ctx, grad_poses):
                dm, dw = ctx.graph.backward(grad_poses.contiguous(), layout="pose8", **ctx.opts)
                return dm, dw, None, None, None

        cls.fn = PoseGraphSolve
        return cls.fn


def solve_pose_graph(graph, meas, weight, poses0, **opts):
    """Differentiable solve: poses (N, 8) = argmin F over the graph's
    structure with measurements ``meas`` (E, 8) and weights ``weight`` (E,),
    starting from ``poses0``.  Gradients flow back to meas and weight through
    the implicit adjoint.  ``opts`` are solve options (polish_iters defaults
    to 8 so that the optimum is a stationary point to full precision)."""
    opts = dict(opts)
    opts.setdefault("polish_iters", 8)
    opts.setdefault("max_iters", 50)
    return _SolveFunction.get().apply(meas, weight, graph, poses0, opts)


def evaluate_cost(n_vertices, edge_i, edge_j, meas, weight, poses, return_bad=False):
    """Stateless F over CUDA tensors (int32 edges, float64 pose8 arrays);
    returns a 0-d CUDA tensor written on the current stream (and, with
    ``return_bad``, a 0-d int32 CUDA tensor counting the skipped edges whose
    endpoints are out of range or equal)."""
    torch = _torch()
    lib = L.load()
    out = torch.empty((), dtype=torch.float64, device="cuda")
    bad = torch.zeros((), dtype=torch.int32, device="cuda")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    L.check(lib.pgo_evaluate_cost(int(n_vertices), int(edge_i.numel()), ptr(edge_i), ptr(edge_j), ptr(meas),
                                  ptr(weight), ptr(poses), ptr(out), ptr(bad), _current_stream_handle()))
    return (out, bad) if return_bad else out


def _dev_f64(x, shape):
    torch = _torch()
    t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    return t.to(device="cuda", dtype=torch.float64).reshape(shape).contiguous()


def _dev_i32(x):
    torch = _torch()
    t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32))
    return t.to(device="cuda", dtype=torch.int32).reshape(-1).contiguous()


def propagate_correction(poses, current, corrected, connected, return_bad=False):
    """Loop correction before the optimisation (pgo_propagate_correction):
    S_k' = (S_k S_c^-1) S_c' for the keyframes in ``connected``, the others
    copied.  Inputs are host arrays or CUDA tensors; returns an (N, 8) CUDA
    tensor written on the current stream (and the count of skipped indices
    as a 0-d int32 CUDA tensor with ``return_bad``)."""
    torch = _torch()
    lib = L.load()
    p = _dev_f64(poses, (-1, 8))
    n = p.shape[0]
    c = _dev_f64(corrected, (8,))
    k = _dev_i32(connected)
    out = torch.empty((n, 8), dtype=torch.float64, device="cuda")
    bad = torch.zeros((), dtype=torch.int32, device="cuda")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    L.check(lib.pgo_propagate_correction(n, ptr(p), int(current), ptr(c), int(k.numel()), ptr(k), ptr(out), ptr(bad),
                                         _current_stream_handle()))
    return (out, bad) if return_bad else out


def correct_points(poses_before, poses_after, points, ref, out=None, return_bad=False):
    """Map-point correction (pgo_correct_points): x' = S_after[r]^-1
    (S_before[r] x) through each point's reference keyframe r (r < 0:
    unchanged).  Returns a (P, 3) CUDA tensor (``out`` if given, which may be
    ``points`` itself) written on the current stream."""
    torch = _torch()
    lib = L.load()
    b = _dev_f64(poses_before, (-1, 8))
    a = _dev_f64(poses_after, (-1, 8))
    X = _dev_f64(points, (-1, 3))
    r = _dev_i32(ref)
    if out is None:
        out = torch.empty_like(X)
    bad = torch.zeros((), dtype=torch.int32, device="cuda")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    L.check(lib.pgo_correct_points(b.shape[0], ptr(b), ptr(a), X.shape[0], ptr(X), ptr(r), ptr(out), ptr(bad),
                                   _current_stream_handle()))
    return (out, bad) if return_bad else out


def _dev(x, dtype):
    torch = _torch()
    tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8,
           np.uint32: torch.int32}[dtype]
    if isinstance(x, torch.Tensor):
        return x.to(device="cuda").contiguous()
    a = np.ascontiguousarray(x, dtype=dtype)
    if dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(device="cuda").contiguous()


def match_params(camera, n_levels=8, scale_factor=1.2, th=10.0, cos_min=0.5, th_low=50):
    """pgo_match_params from a camera dict (fx, fy, cx, cy, min_x, max_x,
    min_y, max_y) and the search settings."""
    p = L.MatchParams()
    for k in ("fx", "fy", "cx", "cy", "min_x", "max_x", "min_y", "max_y"):
        setattr(p, k, float(camera[k]))
    p.scale_factor, p.th, p.cos_min = float(scale_factor), float(th), float(cos_min)
    p.n_levels, p.th_low = int(n_levels), int(th_low)
    return p


class Frames:
    """Keyframe features resident on the device (pgo_frames_create):
    feat_ptr (K + 1,), uv (F, 2) float32, octave (F,), desc (F, 8) uint32,
    map_point (F,) or None, image bounds (min_x, max_x, min_y, max_y)."""

    def __init__(self, feat_ptr, uv, octave, desc, map_point=None, bounds=(0.0, 752.0, 0.0, 480.0), stream=None):
        self._lib = L.load()
        self._h = ctypes.c_void_p()
        ptr = np.ascontiguousarray(feat_ptr, dtype=np.int32)
        self.K = int(ptr.shape[0] - 1)
        self.n_features = int(ptr[-1])
        m = _Marshal(False)
        d = L.FramesDesc()
        d.n_keyframes = self.K
        d.mem_space = L.PGO_MEM_HOST
        d.feat_ptr = m.put(ptr, np.int32)
        d.uv = self._put_f32(m, uv)
        d.octave = m.put(octave, np.int32)
        dd = np.ascontiguousarray(desc, dtype=np.uint32).reshape(-1)
        m.keep.append(dd)
        d.desc = ctypes.c_void_p(dd.ctypes.data)
        d.map_point = m.put(map_point, np.int32)
        d.min_x, d.max_x, d.min_y, d.max_y = (float(b) for b in bounds)
        d.stream = stream if stream is not None else _current_stream_handle()
        L.check(self._lib.pgo_frames_create(ctypes.byref(d), ctypes.byref(self._h)))
        self.bounds = tuple(float(b) for b in bounds)

    @staticmethod
    def _put_f32(m, x):
        a = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
        m.keep.append(a)
        return ctypes.c_void_p(a.ctypes.data)

    @classmethod
    def from_workload(cls, w):
        cam = w.camera
        return cls(w.feat_ptr, np.stack([w.fu, w.fv], axis=1), w.foct, w.fdesc, w.fmp,
                   (cam["min_x"], cam["max_x"], cam["min_y"], cam["max_y"]))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.pgo_frames_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def project_match(self, params, mode, poses, xyz, desc, min_dist, max_dist, normal, ids=None, matched=None):
        """pgo_project_match over every (keyframe, point) pair; returns CUDA
        tensors (match, dist, fuse) of shape (K, P) (fuse None for the
        search).  Inputs are host arrays or CUDA tensors."""
        torch = _torch()
        mode_i = L.PGO_MATCH_SEARCH if mode == "search" else L.PGO_MATCH_FUSE
        X = _dev(xyz, np.float32).reshape(-1)
        P = X.numel() // 3
        D = _dev(desc, np.uint32).reshape(-1)
        mn, mx = _dev(min_dist, np.float32), _dev(max_dist, np.float32)
        nr = _dev(normal, np.float32).reshape(-1)
        idt = _dev(ids, np.int32) if ids is not None else None
        pz = _dev(poses, np.float64).reshape(-1)
        mt = _dev(matched, np.uint8) if (matched is not None and mode_i == L.PGO_MATCH_SEARCH) else None
        match = torch.empty((self.K, P), dtype=torch.int32, device="cuda")
        dist = torch.empty((self.K, P), dtype=torch.int32, device="cuda")
        fuse = torch.empty((self.K, P), dtype=torch.int32, device="cuda") if mode_i == L.PGO_MATCH_FUSE else None
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        pd = L.PointsDesc()
        pd.n_points = P
        pd.xyz, pd.desc, pd.min_dist, pd.max_dist, pd.normal, pd.id = (ptr(X), ptr(D), ptr(mn), ptr(mx), ptr(nr),
                                                                       ptr(idt))
        L.check(self._lib.pgo_project_match(self._h, ctypes.byref(params), mode_i, ptr(pz), ptr(mt), ctypes.byref(pd),
                                            ptr(match), ptr(dist), ptr(fuse)))
        self._keep = (X, D, mn, mx, nr, idt, pz, mt)
        return match, dist, fuse

    def match_workload(self, w, mode, th=10.0, th_low=50, cos_min=0.5, poses=None):
        """project_match with the arrays of a synthetic MatchWorkload."""
        p = match_params(w.camera, w.n_levels, w.scale_factor, th, cos_min, th_low)
        return self.project_match(p, mode, w.poses if poses is None else poses, w.points, w.pdesc, w.min_dist,
                                  w.max_dist, w.normal, w.pid, w.fskip if mode == "search" else None)
