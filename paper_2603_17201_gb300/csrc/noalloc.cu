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
// array's name as a device address, so the first call in each CUDA context
// (with that context's device current) looks its address up with
// cudaGetSymbolAddress and keeps it with the context's unique id; later calls
// in the same context reuse the cached address, and a call in a new context
// (after cudaDeviceReset, say) looks it up again.  That first call should
// therefore come before any stream capture.
//
// Every call shares the one workspace and it keeps the previous call's
// contents, so each call clears the counters it needs before launching.  Calls
// that overlap on the GPU (on different streams, or from several threads)
// race on the workspace and must not be issued.
#include <cuda.h>
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
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // unique id of the context of the cached address

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current CUDA context (0: none, or the
// driver entry points are unavailable, which forces a fresh look-up).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();
    resolved = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

}  // namespace

extern "C" pgo_status pgo_evaluate_cost_noalloc(int32_t n_vertices, int32_t n_edges, const int32_t* edge_i,
                                                const int32_t* edge_j, const double* meas, const double* weight,
                                                const double* poses, double* cost_out, int32_t* bad_edges_out,
                                                void* stream) {
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
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(PGO_ERR_CUDA, "pgo_evaluate_cost_noalloc: cudaGetSymbolAddress of the workspace failed");
      }
      g_scratch_addr[dev] = p;
      g_scratch_ctx[dev] = current_context_id();   // the look-up made the device's context current
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
                                   cost_out, bad_edges_out, blocks, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PGO_ERR_CUDA, cudaGetErrorString(e));
  return PGO_OK;
}
