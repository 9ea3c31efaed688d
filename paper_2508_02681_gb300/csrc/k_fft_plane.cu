// Plane passes (forward r2c + axis 2, inverse axis 2 + c2r) of the transform, FP64 and FP32.
#define UNOCG_FFT_HOST_DEFS
#include "fft_kernels.cuh"

namespace unocg {
template cudaError_t launch_plane_fwd<double>(const PlaneFwdArgs<double>&, cudaStream_t);
template cudaError_t launch_plane_fwd<float>(const PlaneFwdArgs<float>&, cudaStream_t);
template cudaError_t launch_plane_inv<double>(const PlaneInvArgs<double>&, cudaStream_t);
template cudaError_t launch_plane_inv<float>(const PlaneInvArgs<float>&, cudaStream_t);
}  // namespace unocg
