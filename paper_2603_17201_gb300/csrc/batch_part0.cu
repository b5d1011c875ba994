// Persistent batch kernel, compiled for two of its launch schedules (the
// schedules are split over eight translation units that compile in parallel).
#include "batch_impl.cuh"

namespace pgo {

template cudaError_t launch_batch_instance<0, 4, 256, 1>(const DevGraph&, const BatchArgs&, int, size_t,
                                                            cudaStream_t);
template cudaError_t launch_batch_instance<0, 8, 256, 1>(const DevGraph&, const BatchArgs&, int, size_t,
                                                            cudaStream_t);

}  // namespace pgo
