// Axis-1 pass with the block multiply, FP32 fields with BF16 weights (mixed-precision CG) and
// FP32 weights (training operator: apply and backward).
#include "fft_kernels.cuh"

namespace unocg {
template cudaError_t launch_line<float, __nv_bfloat16>(const LineArgs<float, __nv_bfloat16>&, int, cudaStream_t);
template cudaError_t launch_line<float, float>(const LineArgs<float, float>&, int, cudaStream_t);
}  // namespace unocg
