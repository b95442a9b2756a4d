// rb_filter_static: the hierarchical filter of rb_filter with its scratch held in a file-scope
// static device array instead of a caller-provided workspace, for callers that cannot allocate
// device memory. The array is part of the library's device image, so every GPU that loads the
// library holds RB_STATIC_SCRATCH_BYTES of it until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[RB_STATIC_SCRATCH_BYTES];

// The host-side name of the array is a stand-in, not a device address: the device address is
// asked of the runtime (cudaGetSymbolAddress) with the device current. It belongs to the CUDA
// context that loaded the module, so it is kept per context id (unique for the life of the
// process): after cudaDeviceReset the device gets a new primary context, the module is loaded
// again, possibly elsewhere, and the next call looks the address up afresh.
using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

std::mutex g_mu;
std::map<unsigned long long, void*> g_scratch_by_ctx;

template <class F>
F driver_entry(const char* name) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<F>(p);
}

// Id of the calling thread's current context; false when there is none yet or the driver lacks
// the query.
bool current_ctx_id(unsigned long long* id) {
  static const PfnCtxGetCurrent get_current = driver_entry<PfnCtxGetCurrent>("cuCtxGetCurrent");
  static const PfnCtxGetId get_id = driver_entry<PfnCtxGetId>("cuCtxGetId");
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

int scratch_address(void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  if (current_ctx_id(&id)) {
    auto it = g_scratch_by_ctx.find(id);
    if (it != g_scratch_by_ctx.end()) {
      *out = it->second;
      return RB_OK;
    }
  }
  // set-up, once per context: this query also binds the device's primary context if the thread
  // had none, so the id is read again afterwards
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || p == nullptr) {
    rb::set_detail("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    return RB_ERR_CUDA;
  }
  if (current_ctx_id(&id)) g_scratch_by_ctx[id] = p;
  *out = p;
  return RB_OK;
}

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
  void* scratch = nullptr;
  if ((rc = scratch_address(&scratch))) return rc;
  return rb_filter(desc, basis, strain, psd, trig, capacity, n_trig, scratch, (size_t)RB_STATIC_SCRATCH_BYTES, stream);
}
