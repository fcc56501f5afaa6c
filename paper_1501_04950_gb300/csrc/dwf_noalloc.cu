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
#include "../../include/dwf.h"
#include "dwf_internal.cuh"

namespace {

// The red intermediate field of the two-pass apply.  It is fully overwritten
// by the first pass of every call, so nothing needs clearing; all calls share
// it, so calls that overlap on the GPU (different streams, different handles)
// race on its contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DWF_NOALLOC_SCRATCH_BYTES];

}  // namespace

namespace dwf {
// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a stand-in, so dwf_create looks the address up once,
// with the handle's device current, and keeps it in the handle.
cudaError_t noalloc_scratch_address(void** out) {
  return cudaGetSymbolAddress(out, g_noalloc_scratch);
}
}  // namespace dwf

extern "C" int dwf_apply_Dbb_noalloc(dwf_handle h, void* out, const void* in, int prec, int nrhs,
                                     dwf_stream s) {
  return dwf::apply_dbb_noalloc(h, out, in, prec, nrhs, DWF_NOALLOC_SCRATCH_BYTES,
                                reinterpret_cast<cudaStream_t>(s));
}
