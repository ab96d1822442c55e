// Double-precision instantiations of the z pass (its DFT and source-epilogue variants), in
// translation units of their own so that the build compiles them in parallel with the other
// kernels: lines of up to 96 points and the size dispatch here, 128 and 192 points in
// kernels_f64_z2.cu, 256 and 384 points in kernels_f64_z3.cu.
#include "step_kernels.cuh"

namespace pstd {
extern template cudaError_t zpass_n<double, 128>(const StepArgs<double>&, const DftArgs<double>*, int, int, cudaStream_t);
extern template cudaError_t zpass_n<double, 192>(const StepArgs<double>&, const DftArgs<double>*, int, int, cudaStream_t);
extern template cudaError_t zpass_n<double, 256>(const StepArgs<double>&, const DftArgs<double>*, int, int, cudaStream_t);
extern template cudaError_t zpass_n<double, 384>(const StepArgs<double>&, const DftArgs<double>*, int, int, cudaStream_t);
template cudaError_t launch_zpass<double>(const StepArgs<double>&, const DftArgs<double>*, int, int, cudaStream_t);
}  // namespace pstd
