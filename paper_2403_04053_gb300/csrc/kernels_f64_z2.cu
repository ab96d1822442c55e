// Double-precision z pass for lines of 128 and 192 points (see kernels_f64_z.cu).
#include "step_kernels.cuh"

namespace pstd {
template cudaError_t zpass_n<double, 128>(const StepArgs<double>&, const DftArgs<double>*, int, int, cudaStream_t);
template cudaError_t zpass_n<double, 192>(const StepArgs<double>&, const DftArgs<double>*, int, int, cudaStream_t);
}  // namespace pstd
