// rd_noalloc.cu -- rd_evaluate_batch_noalloc: the batched forward solve with
// its work-queue scratch in a fixed, file-scope device array instead of the
// problem's growable workspace, so that the call itself never allocates.
//
// Who needs it: callers that cannot call cudaMalloc/cudaFree while they run,
// for example a host application whose device memory is entirely reserved by
// another allocator (so a new cudaMalloc would fail or fragment its pool), or
// a time-critical loop that must not stall on the device-wide
// synchronisation that cudaFree and a workspace re-allocation imply.
// rd_evaluate_batch grows the problem's workspace when a batch is larger than
// any seen before; this entry point never does.
//
// The scratch array below is part of the library's device image: every GPU
// that loads the library holds it (about 1 MiB) until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "rd_common.cuh"
#include "rd_internal.h"

namespace rd {

// Work lists of the persistent solve kernels: RD_MAX_SIZES lists of up to
// RD_NOALLOC_MAX_BATCH proposal indices, then the per-size append and pop
// counters.
static __device__ __align__(256) int
    g_noalloc_queue[RD_MAX_SIZES * RD_NOALLOC_MAX_BATCH + 2 * RD_MAX_SIZES];

// Device address of g_noalloc_queue on each device (in host code the symbol
// is only a host-side stand-in, never an address the GPU can use).  Looked up
// by rd_problem_create, once per device with that device current: the lookup
// loads this file's module, and with it the array, onto the device, so it
// belongs in a call that allocates anyway; rd_evaluate_batch_noalloc then
// only reads the cached address.
constexpr int kMaxDevices = 64;
static int* g_noalloc_addr[kMaxDevices] = {};
static std::mutex g_noalloc_mutex;

rd_status noalloc_prepare(int device) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("device index out of range for the allocation-free scratch");
    return RD_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[device]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_queue);
    if (e != cudaSuccess || !ptr) {
      set_error(std::string("cudaGetSymbolAddress of the allocation-free scratch failed: ") +
                cudaGetErrorString(e));
      return RD_ECUDA;
    }
    g_noalloc_addr[device] = static_cast<int*>(ptr);
  }
  return RD_OK;
}

static int* noalloc_scratch(int device) {
  if (device < 0 || device >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  return g_noalloc_addr[device];
}

}  // namespace rd

using namespace rd;

extern "C" rd_status rd_evaluate_batch_noalloc(rd_problem* p, int B, const double* theta,
                                               const int* size_idx, double* loglik,
                                               uint32_t* status, void* fields) {
  if (!p) {
    set_error("rd_evaluate_batch_noalloc: problem is NULL");
    return RD_EINVAL;
  }
  if (B < 0 || B > RD_NOALLOC_MAX_BATCH) {
    set_error("rd_evaluate_batch_noalloc: B must be in 0.." +
              std::to_string(RD_NOALLOC_MAX_BATCH) +
              " (the size of its fixed scratch); use rd_evaluate_batch for larger batches");
    return RD_EINVAL;
  }
  if (B == 0) return RD_OK;
  if (!theta || !loglik || !status) {
    set_error("rd_evaluate_batch_noalloc: NULL argument");
    return RD_EINVAL;
  }
  for (int s = 0; s < p->desc.n_sizes; ++s) {
    if (!p->ic_set[s] || !p->obs_set[s]) {
      set_error("initial state and observations must be set for every grid size");
      return RD_ESTATE;
    }
  }
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess || device != p->device) {
    set_error("rd_evaluate_batch_noalloc: the problem's device must be the current device");
    return RD_EINVAL;
  }
  int* scratch = noalloc_scratch(device);  // looked up by rd_problem_create
  if (!scratch) {
    set_error("rd_evaluate_batch_noalloc: scratch address not prepared for this device");
    return RD_ESTATE;
  }
  WorkQueue q = make_queue(p);  // sizes and their order; storage replaced below
  q.items = scratch;
  q.capacity = RD_NOALLOC_MAX_BATCH;
  q.counts = scratch + RD_MAX_SIZES * RD_NOALLOC_MAX_BATCH;
  q.pops = q.counts + RD_MAX_SIZES;
  // launch_fill_queue zeroes the counters left by the previous call first
  cudaError_t e = launch_fill_queue(q, B, size_idx, loglik, status, p->stream);
  if (e == cudaSuccess) {
    e = launch_solve_queue(p, q, theta, loglik, status, fields, p->stream);
  }
  if (e != cudaSuccess) {
    set_error(std::string("rd_evaluate_batch_noalloc: launch failed: ") + cudaGetErrorString(e));
    return RD_ECUDA;
  }
  return RD_OK;
}
