// Double-precision z pass for lines of 256 and 384 points (see kernels_f64_z.cu).
#include "step_kernels.cuh"

namespace pstd {
template cudaError_t zpass_n<double, 256>(const StepArgs<double>&, const DftArgs<double>*, int, int, cudaStream_t);
template cudaError_t zpass_n<double, 384>(const StepArgs<double>&, const DftArgs<double>*, int, int, cudaStream_t);
}  // namespace pstd
