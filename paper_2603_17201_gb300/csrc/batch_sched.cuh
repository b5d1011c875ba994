// Launch schedules of the persistent batch kernel (picked by the autotuner in
// the host runtime) and the per-schedule launcher, which the batch_part*.cu
// translation units instantiate.
#pragma once
#include "internal.cuh"

namespace pgo {

// (mixed, lanes per block row, threads per block, blocks per SM): two blocks
// per SM solve two graphs side by side on one SM (more warps to hide the
// latency of the block-level phases, half the registers per thread).
#define PGO_BATCH_SCHEDULES(X) \
  X(0, 4, 256, 1) X(0, 8, 256, 1) X(0, 16, 256, 1) X(0, 8, 512, 1) X(0, 16, 512, 1) \
  X(0, 4, 256, 2) X(0, 8, 256, 2) X(0, 16, 256, 2) \
  X(1, 4, 256, 1) X(1, 8, 256, 1) X(1, 16, 256, 1) X(1, 8, 512, 1) X(1, 16, 512, 1) \
  X(1, 4, 256, 2) X(1, 8, 256, 2) X(1, 16, 256, 2)

template <int MIXED, int G, int NT, int BPS>
cudaError_t launch_batch_instance(const DevGraph& g, const BatchArgs& a, int blocks, size_t smem, cudaStream_t s);

}  // namespace pgo
