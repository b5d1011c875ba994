"""Host logic of bench.py without a GPU: the job time as the maximum over
ranks with two gloo processes on the CPU (the N > 1 replicas path), the
whole-job aggregation of replicas, the kernel-launch count of a solve, the
algorithmic bytes of one multigrid PCG iteration and the pose-error summary
against the oracle."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=2)
    out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank, 2, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(_free_port(), out), nprocs=2, join=True)
        assert out[0] == 15.0 and out[1] == 15.0


def test_aggregate_replicas_and_launch_count():
    import bench
    one = bench.aggregate_replicas(1, 1000, [10, 10], 200.0, 2)
    two = bench.aggregate_replicas(2, 1000, [10, 10], 200.0, 2)
    assert one["ms_per_solve"] == 100.0 and one["edges_per_s"] == 1000 * 20 / 0.2
    assert two["edges_per_s"] == 2 * one["edges_per_s"]   # weak scaling: twice the work in the same time
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.launches_per_solve("fp64", 11) == 3 + 11 * 6
    assert bench.launches_per_solve("mixed", 11) == 3 + 11 * 11


def test_vcycle_bytes_per_iteration_counts_each_operator_read():
    """The roofline's algorithmic bytes of one multigrid PCG iteration, on a
    hand-sized hierarchy (FP32 blocks of 49 x 4 B, vectors of 7 x 4 B):
    level 0 reads its operator twice, D^-1 twice and Q twice; a further
    sparse level its operator once, Q twice and D^-1 twice; the level next to
    the coarsest its operator once, D^-1 twice and the dense W once."""
    import bench
    blk, vec = 196, 28
    N, E = 10, 20
    lv0 = {"nodes": N, "a_blocks": 0, "p_blocks": 5, "ap_blocks": 12}
    lv1 = {"nodes": 5, "a_blocks": 13, "p_blocks": 5, "ap_blocks": 8}
    lv2 = {"nodes": 3, "a_blocks": 7, "p_blocks": 3, "ap_blocks": 3}
    crs = {"nodes": 1, "a_blocks": 1, "p_blocks": 0, "ap_blocks": 0}
    # three levels above the coarsest: level 1 sparse, level 2 dense (W: 3 x 3 blocks)
    want = ((2 * (E + N) + 2 * N + 2 * 12) * blk + 18 * N * vec
            + (13 + 2 * 8 + 2 * 5) * blk + 8 * 5 * vec
            + (7 + 2 * 3 + 3 * 3) * blk + 6 * 3 * vec)
    assert bench.vcycle_pcg_bytes_per_iter([lv0, lv1, lv2, crs], N, E, 4) == want
    # one level above the coarsest: level 0 itself is the dense level (W: N x N blocks)
    assert bench.vcycle_pcg_bytes_per_iter([lv0, crs], N, E, 4) == (2 * (E + N) + 2 * N + N * N) * blk + 18 * N * vec
    # FP64 doubles every byte
    assert bench.vcycle_pcg_bytes_per_iter([lv0, lv1, lv2, crs], N, E, 8) == 2 * want


def test_pose_error_summary_is_the_rotation_angle():
    """The bench's pose error per vertex is |log(S_gpu S_oracle^-1)|: a pose
    against itself gives 0, a pose turned by a known angle about an axis gives
    that angle (the rotation part of the Sim(3) log), a scale change s gives
    |ln s|."""
    import numpy as np

    import bench

    ref = np.array([[0.0, 0.0, 0.0, 1.0, 1.0, 2.0, 3.0, 1.0]] * 3)
    assert bench.pose_error_summary(ref, ref)["max"] < 1e-15
    turned = ref.copy()
    ang = [0.0, 0.1, 0.3]
    for v, a in enumerate(ang):
        # left-multiply by a rotation of angle a about z: q = (0, 0, sin(a/2), cos(a/2))
        qz = np.array([0.0, 0.0, np.sin(a / 2), np.cos(a / 2)])
        turned[v, :4] = qz
        turned[v, 4:7] = [np.cos(a) * 1.0 - np.sin(a) * 2.0, np.sin(a) * 1.0 + np.cos(a) * 2.0, 3.0]
    e = bench.pose_error_summary(turned, ref)
    assert abs(e["max"] - 0.3) < 1e-12
    assert abs(e["rms"] - np.sqrt((0.1 ** 2 + 0.3 ** 2) / 3)) < 1e-12
    scaled = ref.copy()
    scaled[:, 4:7] *= 2.0
    scaled[:, 7] = 2.0
    assert abs(bench.pose_error_summary(scaled, ref)["max"] - np.log(2.0)) < 1e-12
