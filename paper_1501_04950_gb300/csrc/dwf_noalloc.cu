// dwf_noalloc.cu -- dwf_apply_Dbb_noalloc: the D_bb apply for callers that
// cannot allocate device memory.
//
// dwf_apply_Dbb keeps its red intermediate field in handle workspace that it
// allocates with cudaMalloc on first use.  Some callers cannot allow that:
// frameworks whose pool allocator owns the device memory, or latency-critical
// loops where the implicit device synchronisation of cudaMalloc/cudaFree is
// not acceptable.  This entry point instead uses the file-scope device array
// g_noalloc_scratch below, of DWF_NOALLOC_SCRATCH_BYTES, which every GPU that
// loads the library holds until the process exits.
#include <mutex>

#include "../../include/dwf.h"
#include "dwf_internal.cuh"

namespace {

// The red intermediate field of the two-pass apply.  It is fully overwritten
// by the first pass of every call, so nothing needs clearing; all calls share
// it, so calls that overlap on the GPU (different streams, different handles)
// race on its contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DWF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a stand-in, so the address is looked up once per device
// (with that device current) and cached.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int dwf_apply_Dbb_noalloc(dwf_handle h, void* out, const void* in, int prec, int nrhs,
                                     dwf_stream s) {
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess)
    return dwf::set_error(h, DWF_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
  return dwf::apply_dbb_with_scratch(h, out, in, prec, nrhs, scratch, DWF_NOALLOC_SCRATCH_BYTES,
                                     reinterpret_cast<cudaStream_t>(s));
}
