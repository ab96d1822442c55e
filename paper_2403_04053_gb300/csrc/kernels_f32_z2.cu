// Single-precision z pass for lines of 128 and 192 points (see kernels_f32_z.cu).
#include "step_kernels.cuh"

namespace pstd {
template cudaError_t zpass_n<float, 128>(const StepArgs<float>&, const DftArgs<float>*, int, int, cudaStream_t);
template cudaError_t zpass_n<float, 192>(const StepArgs<float>&, const DftArgs<float>*, int, int, cudaStream_t);
}  // namespace pstd
