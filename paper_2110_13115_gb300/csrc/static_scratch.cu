// rb_filter_static: the hierarchical filter of rb_filter with its scratch held in a file-scope
// static device array instead of a caller-provided workspace, for callers that cannot allocate
// device memory. The array is part of the library's device image, so every GPU that loads the
// library holds RB_STATIC_SCRATCH_BYTES of it until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[RB_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_static_scratch, per device

}  // namespace

extern "C" int rb_filter_static(const rb_filter_desc* desc, const rb_basis* basis, const float* strain,
                                const double* psd, rb_trigger* trig, int64_t capacity, int64_t* n_trig,
                                void* stream) {
  rb_filter_sizes sizes;
  int rc = rb_filter_plan(desc, &sizes);
  if (rc) return rc;
  if (sizes.workspace_bytes > (size_t)RB_STATIC_SCRATCH_BYTES) {
    rb::set_detail("this problem needs %zu bytes of scratch; the static scratch holds %zu bytes "
                   "(use rb_filter with a caller-provided workspace)",
                   sizes.workspace_bytes, (size_t)RB_STATIC_SCRATCH_BYTES);
    return RB_ERR_UNSUPPORTED;
  }
  int dev = 0;
  RB_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    rb::set_detail("device ordinal %d out of range", dev);
    return RB_ERR_UNSUPPORTED;
  }
  void* scratch = nullptr;
  {
    // one-time set-up per device, with that device current: the host-side name of the array is
    // not a device address, so ask the runtime for the device address once and keep it
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      RB_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  return rb_filter(desc, basis, strain, psd, trig, capacity, n_trig, scratch, (size_t)RB_STATIC_SCRATCH_BYTES, stream);
}
