// Single-precision instantiations of the z pass (its DFT and source-epilogue variants), in
// translation units of their own so that the build compiles them in parallel with the other
// kernels: lines of up to 96 points and the size dispatch here, 128 and 192 points in
// kernels_f32_z2.cu, 256 and 384 points in kernels_f32_z3.cu.
#include "step_kernels.cuh"

namespace pstd {
extern template cudaError_t zpass_n<float, 128>(const StepArgs<float>&, const DftArgs<float>*, int, int, cudaStream_t);
extern template cudaError_t zpass_n<float, 192>(const StepArgs<float>&, const DftArgs<float>*, int, int, cudaStream_t);
extern template cudaError_t zpass_n<float, 256>(const StepArgs<float>&, const DftArgs<float>*, int, int, cudaStream_t);
extern template cudaError_t zpass_n<float, 384>(const StepArgs<float>&, const DftArgs<float>*, int, int, cudaStream_t);
template cudaError_t launch_zpass<float>(const StepArgs<float>&, const DftArgs<float>*, int, int, cudaStream_t);
}  // namespace pstd
