// Driver-API functions reached through the runtime's entry-point query, so that the library
// links against the CUDA runtime only: the id of the current context (unique for the life of
// the process, also across a context destroyed and created again) and the encoder of TMA
// tensor maps.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace unocg {

template <typename F>
inline F driver_fn(const char* name) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion(name, &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<F>(fn);
}

// Id of the context current on this host thread (the runtime's primary context of the current
// device once any runtime call has initialised it).
inline cudaError_t current_context_id(unsigned long long* id) {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = driver_fn<GetCurrent>("cuCtxGetCurrent");
  static GetId get_id = driver_fn<GetId>("cuCtxGetId");
  if (!get_current || !get_id) return cudaErrorNotSupported;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || !c) return cudaErrorDeviceUninitialized;
  return get_id(c, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

using TensorMapEncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                          const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                          CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                          CUtensorMapFloatOOBfill);
inline TensorMapEncodeTiled tensor_map_encoder() {
  static TensorMapEncodeTiled fn = driver_fn<TensorMapEncodeTiled>("cuTensorMapEncodeTiled");
  return fn;
}

}  // namespace unocg
