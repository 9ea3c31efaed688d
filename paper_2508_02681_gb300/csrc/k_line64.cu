// Axis-1 pass with the block multiply, FP64 fields and FP64 weights.
#include "fft_kernels.cuh"

namespace unocg {
template cudaError_t launch_line<double, double>(const LineArgs<double, double>&, int, cudaStream_t);
}  // namespace unocg
