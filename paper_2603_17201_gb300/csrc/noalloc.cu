// pgo_evaluate_cost_noalloc: the stateless cost evaluation without any
// device allocation.
//
// pgo_evaluate_cost obtains its small reduction workspace from the
// stream-ordered allocator on every call.  Some callers cannot allow that: a
// real-time tracking or loop-closing thread that must not risk the latency
// of growing the allocator's pool in the middle of a frame, and applications
// that reserve the whole device memory budget up front (typical on embedded
// GPUs) so that any later allocation may fail.  This variant uses a fixed
// workspace that lives in the library's own device image instead.
//
// The workspace is a file-scope device array.  Host code cannot use the
// array's name as a device address, so the first call on each device, with
// that device current, looks its address up with cudaGetSymbolAddress and
// keeps it; later calls on that device reuse the cached address.  That first
// call should therefore come before any stream capture.
//
// Every call shares the one workspace and it keeps the previous call's
// contents, so each call clears the counters it needs before launching.  Calls
// that overlap on the GPU (on different streams, or from several threads)
// race on the workspace and must not be issued.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "internal.cuh"

namespace {

// One thread per edge, 256 threads per block, one double partial per block:
// up to kNoAllocMaxBlocks blocks, i.e. up to kNoAllocMaxEdges edges.
constexpr int kNoAllocMaxBlocks = 4096;
constexpr int kNoAllocMaxEdges = kNoAllocMaxBlocks * 256;
constexpr size_t kCounterBytes = 256;
constexpr size_t kNoAllocScratchBytes = kNoAllocMaxBlocks * sizeof(double) + kCounterBytes;   // 33,024 B

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" pgo_status pgo_evaluate_cost_noalloc(int32_t n_vertices, int32_t n_edges, const int32_t* edge_i,
                                                const int32_t* edge_j, const double* meas, const double* weight,
                                                const double* poses, double* cost_out, void* stream) {
  auto fail = [](pgo_status st, const char* msg) {
    pgo::set_last_error(msg);
    return st;
  };
  if (n_vertices < 0 || n_edges < 0) return fail(PGO_ERR_INVALID_ARG, "pgo_evaluate_cost_noalloc: negative size");
  if (n_edges > kNoAllocMaxEdges) {
    char buf[160];
    snprintf(buf, sizeof(buf),
             "pgo_evaluate_cost_noalloc: n_edges %d exceeds the fixed workspace limit of %d edges; "
             "use pgo_evaluate_cost", n_edges, kNoAllocMaxEdges);
    return fail(PGO_ERR_INVALID_ARG, buf);
  }
  if (!cost_out) return fail(PGO_ERR_INVALID_ARG, "pgo_evaluate_cost_noalloc: cost_out is NULL");
  if (n_edges > 0 && (!edge_i || !edge_j || !meas || !poses))
    return fail(PGO_ERR_INVALID_ARG, "pgo_evaluate_cost_noalloc: NULL input array");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(PGO_ERR_CUDA, "pgo_evaluate_cost_noalloc: no usable current device");
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(PGO_ERR_CUDA, "pgo_evaluate_cost_noalloc: cudaGetSymbolAddress of the workspace failed");
      }
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* partial = reinterpret_cast<double*>(base);
  unsigned* ticket = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(base) + kNoAllocMaxBlocks * sizeof(double));
  int* bad = reinterpret_cast<int*>(ticket + 4);
  // the workspace keeps the previous call's contents: zero the counters
  if (cudaMemsetAsync(ticket, 0, kCounterBytes, s) != cudaSuccess) {
    cudaGetLastError();
    return fail(PGO_ERR_CUDA, "pgo_evaluate_cost_noalloc: clearing the workspace counters failed");
  }
  const int blocks = n_edges > 0 ? (n_edges + 255) / 256 : 1;
  pgo::launch_eval_cost_raw_blocks(n_vertices, n_edges, edge_i, edge_j, meas, weight, poses, partial, ticket, bad,
                                   cost_out, blocks, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PGO_ERR_CUDA, cudaGetErrorString(e));
  return PGO_OK;
}
