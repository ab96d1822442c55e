// Single-precision z pass for lines of 256 and 384 points (see kernels_f32_z.cu).
#include "step_kernels.cuh"

namespace pstd {
template cudaError_t zpass_n<float, 256>(const StepArgs<float>&, const DftArgs<float>*, int, int, cudaStream_t);
template cudaError_t zpass_n<float, 384>(const StepArgs<float>&, const DftArgs<float>*, int, int, cudaStream_t);
}  // namespace pstd
