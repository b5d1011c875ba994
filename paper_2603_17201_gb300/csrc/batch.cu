// Batched form: many independent essential graphs of uneven size solved by
// one persistent kernel launch, replayed as a one-node CUDA graph.
//
// This file holds the schedule table, the launch dispatch and the small
// per-graph pose kernels.  The persistent kernel itself (batch_impl.cuh) is
// compiled once per schedule in the batch_part*.cu translation units.
#include "batch_sched.cuh"
#include "common.cuh"

namespace pgo {

// Poses of every graph from its own current buffer into dst (pose8, global
// vertex order): one block per graph.
__global__ void k_batch_get_poses(DevGraph g, BatchArgs a, double* dst) {
  const int gi = blockIdx.x;
  const int cur = a.gst[gi].cur;
  const int v0 = a.v0[gi], v1 = v0 + a.nv[gi];
  for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    Sim3T<double> P = load_pose(g, cur, v);
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[(size_t)v * 8 + k] = P.q[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) dst[(size_t)v * 8 + 4 + k] = P.t[k];
    dst[(size_t)v * 8 + 7] = P.s;
  }
}

// Reset every graph to pose buffer 0 (poses copied from its current buffer).
__global__ void k_batch_reset(DevGraph g, BatchArgs a) {
  const int gi = blockIdx.x;
  const int cur = a.gst[gi].cur;
  const int v0 = a.v0[gi], v1 = v0 + a.nv[gi];
  if (cur != 0)
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) store_pose(g, 0, v, load_pose(g, cur, v));
  __syncthreads();
  if (threadIdx.x == 0) a.gst[gi].cur = 0;
}

struct BatchSchedule {
  int mixed, lanes, threads, blocks_per_sm;
};

static const BatchSchedule kSchedules[] = {
#define PGO_S(M, G, NT, B) {M, G, NT, B},
    PGO_BATCH_SCHEDULES(PGO_S)
#undef PGO_S
};

int batch_schedule_count() { return (int)(sizeof(kSchedules) / sizeof(kSchedules[0])); }
int batch_schedule_mixed(int s) { return kSchedules[s].mixed; }
int batch_schedule_lanes(int s) { return kSchedules[s].lanes; }
int batch_schedule_threads(int s) { return kSchedules[s].threads; }
int batch_schedule_blocks_per_sm(int s) { return kSchedules[s].blocks_per_sm; }

cudaError_t launch_batch_lm(const DevGraph& g, const BatchArgs& a, int schedule, cudaStream_t s) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (schedule < 0 || schedule >= batch_schedule_count()) return cudaErrorInvalidValue;
  const int slots = sms * kSchedules[schedule].blocks_per_sm;
  const int blocks = a.n_graphs < slots ? a.n_graphs : slots;
  const size_t n7 = 7 * AMG_CMAX;
  const size_t smem = a.amg ? (n7 * n7 + n7) * sizeof(double) : 0;
  // explicit dispatch in list order
  int idx = 0;
#define PGO_D(M, G, NT, B)                                   \
  if (schedule == idx) {                                     \
    return launch_batch_instance<M, G, NT, B>(g, a, blocks, smem, s); \
  }                                                          \
  ++idx;
  PGO_BATCH_SCHEDULES(PGO_D)
#undef PGO_D
  return cudaErrorInvalidValue;
}

void launch_batch_get_poses(const DevGraph& g, const BatchArgs& a, double* dst, cudaStream_t s) {
  k_batch_get_poses<<<a.n_graphs, 256, 0, s>>>(g, a, dst);
}

void launch_batch_reset(const DevGraph& g, const BatchArgs& a, cudaStream_t s) {
  k_batch_reset<<<a.n_graphs, 256, 0, s>>>(g, a);
}


}  // namespace pgo
