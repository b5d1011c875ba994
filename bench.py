"""Benchmark: Sim(3) essential-graph Levenberg-Marquardt on one GB300.

Metric: edges/s = E x LM iterations executed / solve time, and ms per solve,
for the mixed-precision solve (FP32 Jacobians/PCG inside FP64 refinement,
FP64 cost and acceptance) beside the plain FP64 solve, each checked to reach
a final cost within 1e-6 relative of the FP64 oracle.  A step is one full LM
solve (at most 20 iterations) of the 2,000-keyframe figure-8 graph (~30k
edges) from its drifted initial estimate; the graph is resident on the
device and the L2 cache is flushed (256 MB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the repository's reference
implementation of the same method) on the host cores.  Under torchrun with
N > 1 every rank solves its own copy of the graph (replicas: the single-graph
solve does not shard) and rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c2_figure8_2k"
SCHED = {"graph": -1, "eager": 1}
MAX_ITERS = 20
METRIC = "Sim(3) PGO ms/solve & edges/s at rel cost <=1e-6: mixed vs plain FP64, one GB300"
UNIT = "edges/s"
# DRAM bytes (read + write) of one PCG iteration of the roofline kernel,
# k_pcg<float,float,32> on the bench graph: one ncu capture of the 9-iteration
# launch of `bench.py --roofline-only` read 21,231,104 B and wrote 22,272 B
# (profiles/k_pcg_float_c2_figure8_2k.md), amortised over its 9 iterations.
# Set to None whenever the kernel changes until it is captured again.
TRAFFIC_PER_ITERATION = (21231104 + 22272) / 9
# DRAM bytes of one warm FP32 multigrid set-up (k_amg_setup<float>, with the
# level-0 block-Jacobi blocks), the third set-up of the same command: 19,938,304 B
# read, 300,544 B written (profiles/k_amg_setup_float_c2_figure8_2k.md).
TRAFFIC_PER_SETUP = 19938304 + 300544


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the extra workloads of the default run (8k corridor, 4k adjoint, 256-graph batch)")
    ap.add_argument("--roofline-only", action="store_true",
                    help="only the roofline leg: linearise once, then the capped FP32 PCG re-solves "
                         "(an ncu capture of k_pcg should skip 2 launches: the third runs 9 iterations)")
    ap.add_argument("--solver-sweep", action="store_true",
                    help="only the direct-versus-PCG size sweep (one JSON line)")
    ap.add_argument("--profile-solve", action="store_true",
                    help="only one FP64 and one mixed solve of the workload with host-issued launches "
                         "(every kernel a launch of its own), for per-kernel ncu captures")
    ap.add_argument("--batch", action="store_true",
                    help="the batched form instead: 256 uneven graphs (100..5,000 keyframes) in one persistent "
                         "launch per solve, beside sequential single-graph solves of a sample of them")
    ap.add_argument("--schedule", default="graph", choices=["graph", "eager"],
                    help="graph: one CUDA graph per solve (default); eager: host-driven launches "
                         "(for profilers that cannot see inside conditional graph nodes)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------- helpers
def max_over_ranks(value, world, device):
    """The largest value over the ranks (the job's time is its slowest rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_replicas(world, n_edges, lm_iters, total_ms, steps):
    """Whole-job throughput of `world` replicas, each solving its own copy of
    the graph `steps` times (LM iterations per solve in `lm_iters`) in at most
    `total_ms` (the maximum over ranks)."""
    return {"ms_per_solve": total_ms / steps,
            "edges_per_s": world * n_edges * sum(lm_iters) / (total_ms / 1e3)}


def launches_per_solve(precision, lm_iters, refine_steps=2):
    """Kernel launches of one solve through the CUDA graph: set_poses, the LM
    state reset and the first cost; per LM iteration linearise, assemble,
    multigrid set-up (which forms the level-0 block-Jacobi blocks too), PCG
    (mixed: refinement residual, PCG, accumulate per refinement pass), update
    and cost."""
    per_iter = 6 if precision == "fp64" else 5 + 3 * refine_steps
    return 3 + lm_iters * per_iter


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def vcycle_pcg_bytes_per_iter(info, n_vertices, n_edges, value_bytes):
    """Algorithmic bytes of one PCG iteration preconditioned by the V(1,1)
    multigrid cycle (see the design notes).  The cycle applies, per level l,
    the smoothed prolongation Q_l = (I - w D^-1 A) P_l (stored in the pattern
    of A P) on the way down (restriction) and up, and on level L - 1 the dense
    W = Q C^-1 Q^T.  Level 0: the stored operator (one block per edge plus the
    diagonal blocks) read twice (the CG product and the cycle's residual),
    D^-1 twice (pre- and post-smoothing), Q twice, and 18 passes over
    7-vectors (11 of the CG, 7 of the cycle).  Each further sparse level: its
    operator once, Q twice, D^-1 twice and 8 vector passes.  Level L - 1: its
    operator once, D^-1 twice, W once and 6 vector passes."""
    blk, vec = 49 * value_bytes, 7 * value_bytes
    N, E, L = n_vertices, n_edges, len(info) - 1
    d = L - 1
    if d == 0:
        return (2 * (E + N) + 2 * N + N * N) * blk + 18 * N * vec
    b = (2 * (E + N) + 2 * N + 2 * info[0]["ap_blocks"]) * blk + 18 * N * vec
    for lv in info[1:d]:
        b += (lv["a_blocks"] + 2 * lv["ap_blocks"] + 2 * lv["nodes"]) * blk + 8 * lv["nodes"] * vec
    nd = info[d]["nodes"]
    b += (info[d]["a_blocks"] + 2 * nd + nd * nd) * blk + 6 * nd * vec
    return b


def workload_config(name, g, world=1):
    """The `config` object of the bench line, identical in both arms."""
    return {"workload": name, "n_vertices": g.n_vertices, "n_edges": g.n_edges, "max_lm_iters": MAX_ITERS,
            "graph": "figure-8 3-D trajectory, 2 laps, covisibility window 15, 5 loop edges"
            if name == WORKLOAD else name,
            "l2": "flushed before every timed step (256 MB write)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def oracle_reference(g, max_iters, poses=False):
    import oracle
    og = oracle.OracleGraph.from_synthetic(g)
    t = time.perf_counter()
    p, rep = og.lm(g.poses_init, max_iters=max_iters)
    dt = time.perf_counter() - t
    return (dt, rep, p) if poses else (dt, rep)


def pose_error_summary(poses, ref):
    """Max and RMS over vertices of |log(S_gpu S_oracle^-1)|."""
    import numpy as np
    import oracle
    e = oracle.pose_error(poses, ref)
    return {"max": float(e.max()), "rms": float(np.sqrt(np.mean(e * e)))}


def roofline_leg(pg, N, E, stream, flush, torch, reps=5):
    """Per-iteration duration of the dominant kernel, the FP32 PCG of the
    mixed solve with its multigrid V-cycle: re-solve the damped system at the
    current linearisation twice per repetition, with PCG caps of 2 and 9
    iterations (tolerance 0, one refinement pass; both caps below the ~10
    iterations in which the cycle reaches FP32 rounding), each a single k_pcg
    launch after the same preconditioner set-up; CUDA events on the graph's
    stream time both, and the difference divided by the difference in
    iterations is the time of one PCG iteration.  achieved = algorithmic bytes
    per iteration / that time."""
    peaks, peak_kind = measured_peaks()
    lam = 1e-3
    info = pg.multigrid_info()
    def timed(cap):
        kw = dict(precision="mixed", pcg_tol=1e-30, refine_tol=1e-30, refine_steps=1, pcg_max_iters=cap)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pg.resolve_async(lam, **kw)
        e1.record(stream)
        e1.synchronize()
        its = pg.resolve(lam, allow_cap=True, **kw)[1]
        return e0.elapsed_time(e1), its
    timed(2)   # untimed: builds and instantiates both re-solve graphs
    timed(9)
    per_it = []
    for _ in range(reps):
        t_lo, i_lo = timed(2)
        t_hi, i_hi = timed(9)
        if i_hi > i_lo:
            per_it.append((t_hi - t_lo) / (i_hi - i_lo))
    it_ms = statistics.median(per_it) if per_it else float("nan")
    bytes_it = vcycle_pcg_bytes_per_iter(info, N, E, 4)
    achieved = bytes_it / (it_ms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    bj = block_jacobi_pcg_bytes_per_iter(N, E, 4)
    kernel = ("k_pcg<float,float,32> (mixed inner PCG with the V(1,1) multigrid cycle, a warp per block row)"
              if pcg_rows_per_block(N, torch.cuda.get_device_properties(0).multi_processor_count) * 32 <= 512 else
              "k_pcg<float,float,16> (mixed inner PCG with the V(1,1) multigrid cycle, 16 lanes per block row)")
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": TRAFFIC_PER_ITERATION,
            "kernel": kernel + ", per iteration",
            "achieved_kind": "algorithmic bytes (V-cycle operators and vectors) / CUDA-event time per iteration",
            "limiter": "latency: 9 dependent phases behind grid barriers per iteration; the marginal iteration "
                       "runs from L2 and shared memory",
            "frac_block_jacobi_bytes": bj / (it_ms * 1e-3) / 1e9 / peak,
            "block_jacobi_bytes_per_iteration": bj,
            "peak_kind": peak_kind, "us_per_pcg_iteration": 1e3 * it_ms,
            "algorithmic_bytes_per_iteration": bytes_it, "multigrid_levels": [lv["nodes"] for lv in info],
            "iterations_timed": [i_lo, i_hi]}


def pcg_rows_per_block(N, sms):
    """Rows per thread block of the persistent PCG (one block per SM)."""
    return max(1, -(-N // sms))


def block_jacobi_pcg_bytes_per_iter(n_vertices, n_edges, value_bytes):
    """The plain block-Jacobi PCG iteration's algorithmic bytes: every
    off-diagonal block read once (used for both directions), the diagonal and
    preconditioner blocks once, and six passes over the 7-vectors."""
    blk, vec = 49 * value_bytes, 7 * value_bytes
    return n_edges * blk + n_vertices * (2 * blk + 6 * vec)


def setup_bytes(info, n_vertices, n_edges, value_bytes):
    """Compulsory bytes of one multigrid set-up: read each level's operator
    once (level 0: one block per edge plus the diagonal blocks) and the poses,
    write each product once -- tentative prolongations (one block per node),
    P, A P and Q = (I - w D^-1 A) P (both in the pattern of A P), the next
    level's operator and D^-1 -- and, on the level next to the coarsest, the
    dense W = Q C^-1 Q^T and H = Q C^-1."""
    blk = 49 * value_bytes
    L = len(info) - 1
    b = n_vertices * 64
    for l in range(L):
        a = n_edges + n_vertices if l == 0 else info[l]["a_blocks"]
        b += (a + info[l]["nodes"] + info[l]["p_blocks"] + 2 * info[l]["ap_blocks"]) * blk
        b += (info[l + 1]["a_blocks"] + info[l + 1]["nodes"]) * blk
    if L >= 1:
        b += (info[L - 1]["nodes"] ** 2 + info[L - 1]["nodes"] * info[L]["nodes"]) * blk
    return b


def setup_leg(pg, N, E, stream, flush, torch, reps=7):
    """Duration of the FP32 multigrid set-up of the mixed solve at the
    current linearisation (pgo_graph_precondition: block-Jacobi blocks plus
    the numeric hierarchy), CUDA events on the graph's stream, L2 flushed
    before each repetition; achieved = compulsory bytes / duration."""
    peaks, peak_kind = measured_peaks()
    info = pg.multigrid_info()
    lam = 1e-3
    pg.precondition_async(lam, precision="mixed")
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pg.precondition_async(lam, precision="mixed")
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms)
    b = setup_bytes(info, N, E, 4)
    peak = peaks.get("hbm_gbs", 6800.0)
    return {"bound": "hbm", "achieved": b / (t * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
            "frac": b / (t * 1e-3) / 1e9 / peak, "traffic": TRAFFIC_PER_SETUP,
            "kernel": "k_amg_setup<float> (FP32 multigrid set-up with the level-0 block-Jacobi blocks, once per LM linearisation)",
            "achieved_kind": "compulsory bytes of the set-up / CUDA-event time",
            "limiter": "latency and instruction issue: grid-barrier phases of 7x7 block products",
            "ms_per_setup": t, "algorithmic_bytes_per_setup": b, "peak_kind": peak_kind}


def run_profile_solve(args):
    """One host-scheduled FP64 and one mixed solve of the workload (every
    kernel of the solve a launch of its own), then one call of each other
    kernel family: the loop-correction steps (150 map points per keyframe),
    the projection search PS3a-c and loop fusion (4,000 map points), a
    direct-solver solve of the 200-keyframe circle and the stateless cost."""
    import numpy as np
    import torch
    from paper_2603_17201_gb300 import (Frames, PoseGraph, correct_points, evaluate_cost, match_params,
                                        propagate_correction)
    from paper_2603_17201_gb300 import synthetic as syn
    torch.cuda.set_device(0)
    g = syn.make_config(args.workload)
    for precision in ("fp64", "mixed"):
        pg = PoseGraph.from_synthetic(g)
        rep = pg.solve(max_iters=MAX_ITERS, precision=precision, schedule=SCHED["eager"])
        print(json.dumps({"precision": precision, "final_cost": rep["final_cost"], "iterations": rep["iterations"],
                          "pcg_iterations": rep["pcg_iterations"]}), flush=True)
        pg.close()
    lc = syn.make_loop_correction(g, points_per_kf=150, seed=1)
    out = propagate_correction(g.poses_init, lc.current, lc.corrected, lc.connected)
    correct_points(g.poses_init, out, lc.points, lc.ref)
    for mode, K, th in (("search", 3, 10.0), ("fusion", 30, 4.0)):
        w = syn.make_match_workload(mode, n_kf=K, n_points=4000, seed=7)
        fr = Frames.from_workload(w)
        fr.match_workload(w, mode, th=th)
        torch.cuda.synchronize()
        fr.close()
    c1 = syn.make_config("c1_circle200")
    pd = PoseGraph.from_synthetic(c1)
    rep = pd.solve(max_iters=MAX_ITERS, precision="mixed", linear_solver="direct", schedule=SCHED["eager"])
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    evaluate_cost(g.n_vertices, t(g.edge_i, torch.int32), t(g.edge_j, torch.int32), t(g.meas), None,
                  t(g.poses_init))
    torch.cuda.synchronize()
    print(json.dumps({"direct_c1_mixed_final_cost": rep["final_cost"]}), flush=True)


def run_roofline_only(args):
    import torch
    from paper_2603_17201_gb300 import PoseGraph
    from paper_2603_17201_gb300 import synthetic as syn
    torch.cuda.set_device(0)
    g = syn.make_config(args.workload)
    pg = PoseGraph.from_synthetic(g)
    pg.linearize("mixed", jacobians=False)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    r = roofline_leg(pg, g.n_vertices, g.n_edges, torch.cuda.current_stream(), flush, torch, reps=1)
    print(json.dumps({"roofline": r}), flush=True)


# --------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2603_17201_gb300 import synthetic as syn
    g = syn.make_config(args.workload)
    for _ in range(args.warmup):
        oracle_reference(g, MAX_ITERS)
    times, iters = [], []
    for _ in range(args.steps):
        dt, rep = oracle_reference(g, MAX_ITERS)
        times.append(dt)
        iters.append(rep["iterations"])
    total = sum(times)
    value = g.n_edges * sum(iters) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args.workload, g, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": host_cores(), "kind": "oracle",
                         "sample": f"{args.steps} full LM solves of {args.workload}, single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- batched form
BATCH_SCHEDULES = [(4, 256, 1), (8, 256, 1), (16, 256, 1), (8, 512, 1), (16, 512, 1),
                   (4, 256, 2), (8, 256, 2), (16, 256, 2)]


def batch_leg(steps, sample=32):
    """256 graphs with N ~ U[100, 5000] (window 15, one loop per 400 keyframes):
    each step solves all of them (20 LM iterations at most) in one persistent
    launch from their initial estimates, timed by the library's CUDA events
    around the launch (a fresh batch per step, created outside the timing, the
    schedule autotuned once in the warm-up).  Beside it, sequential
    single-graph solves of the first `sample` graphs, scaled to 256."""
    import torch
    from paper_2603_17201_gb300 import PoseGraph, PoseGraphBatch
    from paper_2603_17201_gb300 import synthetic as syn
    gs = syn.make_batch()
    V = sum(g.n_vertices for g in gs)
    E = sum(g.n_edges for g in gs)
    out = {}
    for precision in ("fp64", "mixed"):
        t0 = time.perf_counter()
        b = PoseGraphBatch(gs)
        t_create = time.perf_counter() - t0
        b.solve(poses=False, max_iters=MAX_ITERS, precision=precision)   # warm-up + autotune
        lanes, threads, bps, _ = b.schedule()
        sched = BATCH_SCHEDULES.index((lanes, threads, bps)) + (len(BATCH_SCHEDULES) if precision == "mixed" else 0)
        ms, its = [], []
        for _ in range(max(1, steps)):
            b.close()
            b = PoseGraphBatch(gs)
            reps, _ = b.solve(poses=False, max_iters=MAX_ITERS, precision=precision, schedule=sched)
            assert max(r["status"] for r in reps) == 0
            ms.append(reps[0]["ms_total"])
            its.append(sum(r["iterations"] for r in reps))
        b.close()
        seq = 0.0
        for g in gs[:sample]:
            pg = PoseGraph.from_synthetic(g)
            pg.solve(max_iters=MAX_ITERS, precision=precision)
            pg.set_poses(g.poses_init)
            seq += pg.solve(max_iters=MAX_ITERS, precision=precision)["ms_total"]
            pg.close()
        t = statistics.median(ms)
        out[precision] = {"ms_per_batch": t, "ms_per_graph": t / len(gs), "lm_iterations": statistics.median(its),
                          "graph_edges_per_s": E / (t * 1e-3),
                          "schedule": {"lanes": lanes, "threads": threads, "blocks_per_sm": bps},
                          "create_ms": 1e3 * t_create,
                          "sequential_single_ms_scaled": seq * len(gs) / sample,
                          "sequential_sample": f"first {sample} graphs, single-graph multigrid solves"}
    torch.cuda.synchronize()
    return {"workload": "c4_batch256", "graphs": len(gs), "vertices": V, "edges": E,
            "mixed": out["mixed"], "fp64": out["fp64"],
            "speedup_batched_mixed_vs_sequential_fp64": out["fp64"]["sequential_single_ms_scaled"] /
            out["mixed"]["ms_per_batch"],
            "speedup_batched_mixed_vs_batched_fp64": out["fp64"]["ms_per_batch"] / out["mixed"]["ms_per_batch"]}


def run_batch(args):
    import torch
    torch.cuda.set_device(0)
    r = batch_leg(args.steps)
    line = {"metric": "batched Sim(3) PGO: ms per batch of 256 graphs (one persistent launch)", "unit": "ms",
            "value": r["mixed"]["ms_per_batch"], "higher_is_better": False, "dtype": "f32+f64",
            "data": "synthetic", "steps": args.steps,
            "config": {"workload": "c4_batch256", "graphs": r["graphs"], "vertices": r["vertices"],
                       "edges": r["edges"], "max_lm_iters": MAX_ITERS}}
    line.update({k: v for k, v in r.items() if k not in ("graphs", "vertices", "edges", "workload")})
    print(json.dumps(line), flush=True)


def single_leg(name, steps, flush, torch, max_iters=MAX_ITERS):
    """One named single-graph workload: `steps` timed LM solves per precision
    (one warm-up each) from the drifted estimate, device-resident inputs, L2
    flushed before each, CUDA events on the graph's stream."""
    from paper_2603_17201_gb300 import PoseGraph
    from paper_2603_17201_gb300 import synthetic as syn
    g = syn.make_config(name)
    dev = torch.device("cuda", torch.cuda.current_device())
    t = lambda a, dt=torch.float64: torch.as_tensor(a, dtype=dt, device=dev)  # noqa: E731
    init = t(g.poses_init)
    pg = PoseGraph(g.n_vertices, t(g.edge_i, torch.int32), t(g.edge_j, torch.int32), t(g.meas), None, None, init, 0)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": name, "n_vertices": g.n_vertices, "n_edges": g.n_edges, "max_lm_iters": max_iters}
    for precision in ("fp64", "mixed"):
        ms, rep = [], None
        for k in range(steps + 1):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pg.set_poses(init)
            pg.solve_async(max_iters=max_iters, precision=precision)
            e1.record(stream)
            e1.synchronize()
            rep = pg.solve_report()
            if k > 0:
                ms.append(e0.elapsed_time(e1))
        m = statistics.median(ms)
        out[precision] = {"ms_per_solve": m, "edges_per_s": g.n_edges * rep["iterations"] / (m * 1e-3),
                          "lm_iterations": rep["iterations"], "pcg_iterations": rep["pcg_iterations"],
                          "final_cost": rep["final_cost"], "stop_reason": rep["stop_reason"]}
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_solve"] / out["mixed"]["ms_per_solve"]
    out["rel_cost_mixed_vs_fp64"] = abs(out["mixed"]["final_cost"] - out["fp64"]["final_cost"]) / out["fp64"]["final_cost"]
    pg.close()
    return out


def correction_leg(torch, flush, name="c3_corridor_8k", points_per_kf=150, reps=50):
    """Loop-correction steps on a graph's keyframes and map points
    (`points_per_kf` per keyframe): pgo_propagate_correction of the connected
    keyframes and pgo_correct_points of every map point (the post-optimisation
    pass), device-resident arrays, L2 flushed before the timed calls, CUDA
    events on the current stream around `reps` back-to-back C ABI calls
    (mean per call).  Roofline of the point
    pass: 52 bytes (point read and write, reference index) and 9 FP64 fused
    multiply-adds (18 flops) per point; the FP64 rate bounds it."""
    import numpy as np
    from paper_2603_17201_gb300 import correct_points, propagate_correction
    from paper_2603_17201_gb300 import synthetic as syn
    g = syn.make_config(name)
    lc = syn.make_loop_correction(g, points_per_kf=points_per_kf, seed=1)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    poses, corr, conn = t(g.poses_init), t(lc.corrected), t(lc.connected, torch.int32)
    X, ref = t(lc.points), t(lc.ref, torch.int32)
    out_p = propagate_correction(poses, lc.current, corr, conn)
    out_x = correct_points(poses, out_p, X, ref)
    # the C ABI calls with their device pointers marshalled once, `reps` calls
    # back to back between the events: the device time, not Python's
    import ctypes
    from paper_2603_17201_gb300 import _lib
    lib = _lib.load()
    ptr = lambda x: ctypes.c_void_p(x.data_ptr())  # noqa: E731
    h_stream = ctypes.c_void_p(stream.cuda_stream)
    P, N = X.shape[0], g.n_vertices
    prop_args = (N, ptr(poses), int(lc.current), ptr(corr), int(conn.numel()), ptr(conn), ptr(out_p), None, h_stream)
    pts_args = (N, ptr(poses), ptr(out_p), P, ptr(X), ptr(ref), ptr(out_x), None, h_stream)

    def timed(fn, args):
        torch.cuda.synchronize()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn(*args)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_prop = timed(lib.pgo_propagate_correction, prop_args)
    ms_pts = timed(lib.pgo_correct_points, pts_args)
    bytes_ = 52 * P + N * (2 * 64 + 2 * 128)
    flops = 18 * P
    peaks, peak_kind = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    fp64_tflops = 1.25   # nominal GB300 FP64 rate (no FP64 figure is measured)
    f_hbm = bytes_ / (ms_pts * 1e-3) / 1e9 / hbm
    f_alu = flops / (ms_pts * 1e-3) / 1e12 / fp64_tflops
    return {"workload": f"{name} keyframes, {points_per_kf} map points each", "n_vertices": N, "n_points": P,
            "n_connected": int(len(lc.connected)),
            "propagate_us": 1e3 * ms_prop, "correct_points_us": 1e3 * ms_pts,
            "points_per_s": P / (ms_pts * 1e-3),
            "roofline": {"bound": "alu" if f_alu > f_hbm else "hbm",
                         "achieved": flops / (ms_pts * 1e-3) / 1e12, "peak": fp64_tflops, "unit": "TFLOP/s (FP64)",
                         "frac": f_alu, "peak_kind": "nominal FP64 rate",
                         "achieved_hbm_gbs": bytes_ / (ms_pts * 1e-3) / 1e9, "frac_hbm": f_hbm,
                         "hbm_peak_kind": peak_kind, "traffic": None,
                         "kernel": "k_point_table + k_apply_points (pgo_correct_points, one call)"}}


def matching_leg(torch, flush, reps=20):
    """Projection search PS3a-c (3 keyframes, 4,000 map points) and loop
    fusion (30 connected keyframes, 4,000 loop map points): pgo_project_match
    on device-resident features (a frames object) and points, L2 flushed
    before the timed calls, CUDA events on the current stream around `reps`
    back-to-back C ABI calls (mean per call).  Throughput in (keyframe, point)
    pairs per second; the compulsory traffic (points, features and outputs
    once) is a few MB, so the call is bound by latency and the integer
    popcount work of the candidate comparisons, not by HBM."""
    import numpy as np
    from paper_2603_17201_gb300 import Frames, match_params
    from paper_2603_17201_gb300 import synthetic as syn
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name, mode, K, th in (("ps3_search", "search", 3, 10.0), ("loop_fusion", "fusion", 30, 4.0)):
        w = syn.make_match_workload(mode, n_kf=K, n_points=4000, seed=7)
        fr = Frames.from_workload(w)
        prm = match_params(w.camera, w.n_levels, w.scale_factor, th)
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
        args = (t(w.poses, torch.float64), t(w.points, torch.float32), t(w.pdesc.view(np.int32), torch.int32),
                t(w.min_dist, torch.float32), t(w.max_dist, torch.float32), t(w.normal, torch.float32),
                t(w.pid, torch.int32), t(w.fskip, torch.uint8) if mode == "search" else None)
        m, _, f = fr.project_match(prm, mode, *args[:7], matched=args[7])
        # the C ABI call with its arguments marshalled once, `reps` calls back
        # to back between the events
        import ctypes
        from paper_2603_17201_gb300 import _lib
        lib = _lib.load()
        ptr = lambda x: ctypes.c_void_p(x.data_ptr()) if x is not None else None  # noqa: E731
        pdsc = _lib.PointsDesc()
        pdsc.n_points = int(w.points.shape[0])
        pdsc.xyz, pdsc.desc, pdsc.min_dist, pdsc.max_dist, pdsc.normal, pdsc.id = (
            ptr(args[1]), ptr(args[2]), ptr(args[3]), ptr(args[4]), ptr(args[5]), ptr(args[6]))
        dist = torch.empty_like(m)
        cargs = (fr._h, ctypes.byref(prm), 0 if mode == "search" else 1, ptr(args[0]), ptr(args[7]),
                 ctypes.byref(pdsc), ptr(m), ptr(dist), ptr(f))
        torch.cuda.synchronize()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            lib.pgo_project_match(*cargs)
        e1.record(stream)
        e1.synchronize()
        ms = [e0.elapsed_time(e1) / reps]
        tm = statistics.median(ms)
        P = w.points.shape[0]
        out[name] = {"keyframes": K, "points": P, "features": int(w.feat_ptr[-1]), "us_per_call": 1e3 * tm,
                     "pairs_per_s": K * P / (tm * 1e-3), "matches": int((m >= 0).sum().item())}
        fr.close()
    return out


def solver_sweep_leg(torch, flush, sizes=(100, 200, 300, 400, 600, 800, 1000, 1500, 2000), steps=3):
    """Direct block Cholesky against the multigrid PCG by graph size (the
    shape of the paper's Fig. 4 size sweep): figure-8 graphs of N keyframes
    (window 15, one loop per 400 keyframes), full LM solves from the drifted
    estimate in each precision, device-resident, L2 flushed before each,
    CUDA events on the graph's stream, median of `steps`."""
    from paper_2603_17201_gb300 import PGOError, PoseGraph
    from paper_2603_17201_gb300 import synthetic as syn
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    rows = []
    for n in sizes:
        g = syn.make_graph("figure8", n, seed=100 + n, window=15, n_loops=max(1, n // 400))
        init = torch.as_tensor(g.poses_init, device=dev)
        pg = PoseGraph(g.n_vertices, g.edge_i, g.edge_j, g.meas, None, None, g.poses_init, 0)
        row = {"n_vertices": n, "n_edges": g.n_edges}
        for precision in ("fp64", "mixed"):
            for solver in ("pcg", "direct"):
                ms = []
                try:
                    for k in range(steps + 1):
                        flush.fill_(1.0)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        pg.set_poses(init)
                        pg.solve_async(max_iters=MAX_ITERS, precision=precision, linear_solver=solver)
                        e1.record(stream)
                        e1.synchronize()
                        if k > 0:
                            ms.append(e0.elapsed_time(e1))
                    rep = pg.solve_report()
                    row[f"{precision}_{solver}_ms"] = statistics.median(ms)
                    row[f"{precision}_{solver}_cost"] = rep["final_cost"]
                except PGOError as e:
                    row[f"{precision}_{solver}_ms"] = None
                    row[f"{precision}_{solver}_why"] = str(e)[:80]
        pg.close()
        rows.append(row)
    cross = {}
    for precision in ("fp64", "mixed"):
        faster = [r["n_vertices"] for r in rows if r.get(f"{precision}_direct_ms") is not None
                  and r[f"{precision}_direct_ms"] < r[f"{precision}_pcg_ms"]]
        cross[precision] = max(faster) if faster else 0
    return {"rows": rows, "direct_faster_up_to_vertices": cross}


def adjoint_leg(steps, torch):
    """The differentiation workload (4,000-keyframe noisy figure-8, 67,857
    edges, weights 1): FP64 forward solve to a stationary point (LM plus
    Newton polish), then pgo_backward for a seeded loss gradient dL/dx (N x 7
    on the device): gradients w.r.t. every measurement and weight.  Wall time
    of each call (both synchronise), median over `steps`."""
    import numpy as np
    from paper_2603_17201_gb300 import PoseGraph
    from paper_2603_17201_gb300 import synthetic as syn
    g = syn.make_config("c5_figure8_4k_noisy")
    dev = torch.device("cuda", torch.cuda.current_device())
    t = lambda a, dt=torch.float64: torch.as_tensor(a, dtype=dt, device=dev)  # noqa: E731
    init = t(g.poses_init)
    pg = PoseGraph(g.n_vertices, t(g.edge_i, torch.int32), t(g.edge_j, torch.int32), t(g.meas),
                   t(np.ones(g.n_edges)), None, init, 0)
    dl = t(np.random.default_rng(5).normal(size=(g.n_vertices, 7)))
    opts = dict(max_iters=60, polish_iters=10, gtol=1e-15, pcg_tol=1e-12, pcg_max_iters=20000)
    fwd, bwd, rep = [], [], None
    for k in range(steps + 1):
        pg.set_poses(init)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = pg.solve(**opts)
        t1 = time.perf_counter()
        pg.backward(dl, layout="tangent", pcg_tol=1e-12, pcg_max_iters=20000)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if k > 0:
            fwd.append(1e3 * (t1 - t0))
            bwd.append(1e3 * (t2 - t1))
    pg.close()
    return {"workload": "c5_figure8_4k_noisy", "n_vertices": g.n_vertices, "n_edges": g.n_edges,
            "forward_ms": statistics.median(fwd), "backward_ms": statistics.median(bwd),
            "forward_lm_iterations": rep["iterations"], "grad_inf_norm": rep["grad_inf_norm"],
            "precision": "fp64"}


# --------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2603_17201_gb300 import PoseGraph
    from paper_2603_17201_gb300 import synthetic as syn
    from paper_2603_17201_gb300 import _lib

    g = syn.make_config(args.workload)
    E, N = g.n_edges, g.n_vertices
    stream = torch.cuda.current_stream(dev)
    t = lambda a, dt=torch.float64: torch.as_tensor(a, dtype=dt, device=dev)  # noqa: E731
    dev_init = t(g.poses_init)
    pg = PoseGraph(N, t(g.edge_i, torch.int32), t(g.edge_j, torch.int32), t(g.meas), None, None, dev_init, 0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def solve_steps(precision, steps, timed):
        ms, its, reps = [], [], []
        for _ in range(steps):
            flush.fill_(1.0)   # L2 flush, outside the timed interval
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pg.set_poses(dev_init)
            pg.solve_async(max_iters=MAX_ITERS, precision=precision, schedule=SCHED[args.schedule])
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            rep = pg.solve_report()
            its.append(rep["iterations"])
            reps.append(rep)
        return ms, its, reps

    results = {}
    final_poses = {}
    clocks = None
    launches = 0
    for precision in ("fp64", "mixed"):
        solve_steps(precision, args.warmup, False)
        barrier()
        with ClockSampler(local) as cs:
            ms, its, reps = solve_steps(precision, args.steps, True)
            barrier()
        if precision == "mixed":
            clocks = cs.summary()
        final_poses[precision] = pg.get_poses()   # the last timed solve's result (host copy, untimed)
        tot_ms = max_over_ranks(sum(ms), world, dev)
        rep = reps[-1]
        results[precision] = dict(aggregate_replicas(world, E, its, tot_ms, args.steps),
                                  lm_iterations=its[-1], pcg_iterations=rep["pcg_iterations"],
                                  final_cost=rep["final_cost"], initial_cost=rep["initial_cost"])
        if precision == "mixed":
            launches = sum(launches_per_solve(precision, k) for k in its)

    roofline = roofline_leg(pg, N, E, stream, flush, torch)
    roofline_setup = setup_leg(pg, N, E, stream, flush, torch)
    extra = {}
    if not args.no_extra and world == 1:
        extra["c3"] = single_leg("c3_corridor_8k", 3, flush, torch)
        extra["c5_adjoint"] = adjoint_leg(2, torch)
        extra["c4_batch"] = batch_leg(1, sample=16)
    if not args.no_extra:
        extra["loop_correction"] = correction_leg(torch, flush)
        extra["matching"] = matching_leg(torch, flush)
        extra["solver_sweep"] = solver_sweep_leg(torch, flush)

    # ---- correctness gate: final cost vs the FP64 oracle ----
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        dt, orep, opos = oracle_reference(g, MAX_ITERS, poses=True)
        for precision in ("fp64", "mixed"):
            rel = abs(results[precision]["final_cost"] - orep["final_cost"]) / orep["final_cost"]
            results[precision]["rel_cost_err_vs_oracle"] = rel
            results[precision]["pose_err_vs_oracle"] = pose_error_summary(final_poses[precision], opos)
        cpu = {"value": E * orep["iterations"] / dt, "unit": UNIT, "cores": 1, "host_cores": host_cores(),
               "kind": "oracle",
               "sample": f"one full LM solve of {args.workload} ({orep['iterations']} iterations, "
                         f"{dt:.1f} s, single thread)"}

    # ---- end to end through the C ABI with host buffers: create the graph
    # from pinned host arrays, solve, read the poses back, destroy ----
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    h_ei, h_ej, h_meas, h_init = pin(g.edge_i), pin(g.edge_j), pin(g.meas), pin(g.poses_init)
    h_out = torch.empty((N, 8), dtype=torch.float64).pin_memory()
    e2e_ms, e2e_its = [], []
    for k in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        pe = PoseGraph(N, h_ei.numpy(), h_ej.numpy(), h_meas.numpy(), None, None, h_init.numpy(), 0)
        rep = pe.solve(poses_out=h_out.numpy(), max_iters=MAX_ITERS, precision="mixed",
                       schedule=SCHED[args.schedule])
        pe.close()
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
            e2e_its.append(rep["iterations"])
    e2e_total = max_over_ranks(sum(e2e_ms), world, dev)
    e2e = {"value": world * E * sum(e2e_its) / (e2e_total / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(E * (4 + 4 + 64) + N * 64), "d2h_bytes_per_step": int(N * 64),
           "ms_per_step": e2e_total / len(e2e_ms)}

    if rank == 0:
        mixed = results["mixed"]
        line = {
            "metric": METRIC, "value": mixed["edges_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mixed["ms_per_solve"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": workload_config(args.workload, g, world),
            "mixed": mixed, "fp64": results["fp64"],
            "speedup_mixed_vs_fp64": results["fp64"]["ms_per_solve"] / mixed["ms_per_solve"],
            "roofline": roofline, "roofline_setup": roofline_setup,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.batch:
        run_batch(args)
        return
    if args.solver_sweep:
        import torch
        torch.cuda.set_device(0)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        print(json.dumps({"solver_sweep": solver_sweep_leg(torch, flush)}), flush=True)
    elif args.profile_solve:
        run_profile_solve(args)
    elif args.roofline_only:
        run_roofline_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
