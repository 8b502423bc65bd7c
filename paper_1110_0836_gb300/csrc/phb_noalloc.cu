// phb_mhd_rhs_noalloc: neighbour build + fused RHS for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the right-
// hand side: code running inside a memory pool that forbids new device
// allocations, a host framework that owns every device buffer and hands out
// only the arrays of a computation, or a real-time loop that must not block
// on the allocator.  They can still supply the inputs and outputs; this entry
// point takes every byte of scratch (cell lists, neighbour lists, slot-order
// copies, FP32 records) from one fixed array that the library declares at file
// scope in device memory.  It runs the same kernels as phb_build_neighbors
// followed by phb_mhd_rhs, with that array as the workspace.
#include "phb_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB on every device that loads the library

// The scratch itself.  In host code `g_static_scratch` is only a host-side
// stand-in for the symbol, not a device address: the device address comes from
// cudaGetSymbolAddress in the context that is current when the call is made.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of the scratch array in the current context.  It is looked
// up on every call rather than cached per device ordinal: after
// cudaDeviceReset, or under another context on the same device, the array
// lives at another address, and a cached one would send the kernels to memory
// that is no longer (or not) theirs.  The lookup is a host-side query; the
// first one in a context also loads the library's device code there.
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace

using namespace phb;

extern "C" size_t phb_noalloc_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" phb_status phb_mhd_rhs_noalloc(const phb_plan* plan, const phb_params* params,
                                          const double* pos, const double* lambda, const double* U,
                                          double* dudt, int32_t* fit_status, int32_t* status_word,
                                          phb_stream_t stream) {
  if (!plan || plan->ws_bytes == 0 || plan->n <= 0) return PHB_ERR_INVALID_ARG;
  // the build and the fused fit need only the common part of the workspace
  if (plan->ws_off[R_END_COMMON] > kStaticScratchBytes) return PHB_ERR_WORKSPACE;
  void* ws = nullptr;
  if (scratch_address(&ws) != cudaSuccess) return PHB_ERR_CUDA;
  const size_t bytes = plan->ws_off[R_END_COMMON];
  phb_status s = phb_build_neighbors(plan, pos, lambda, ws, bytes, status_word, stream);
  if (s != PHB_OK) return s;
  return phb_mhd_rhs(plan, params, pos, lambda, U, ws, bytes, dudt, fit_status, status_word, stream);
}
