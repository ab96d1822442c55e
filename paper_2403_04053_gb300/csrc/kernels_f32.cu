// Single-precision instantiations of the step (with the fused running DFT) and transform kernels.
#include "ntdf_kernels.cuh"
#include "step_kernels.cuh"

namespace pstd {
template cudaError_t launch_xpass<float>(const StepArgs<float>&, const DftArgs<float>*, int, cudaStream_t);
template cudaError_t launch_ypass<float>(const StepArgs<float>&, const DftArgs<float>*, int, cudaStream_t);
template cudaError_t launch_source<float>(const StepArgs<float>&, int, cudaStream_t);
template cudaError_t launch_aux_table<float>(const double2*, const double*, const double*, int, int, long long, long, bool,
                                           float2*, float2*, cudaStream_t);
template cudaError_t launch_aux_eval<float>(const AuxEvalArgs<float>&, cudaStream_t);
template bool xypass_available<float>(int, int, int);
template bool pipe_y_available<float>(int);
template bool tma_pass_available<float>(int);
template cudaError_t launch_xypass<float>(const StepArgs<float>&, const DftArgs<float>*, const DftArgs<float>*, int, cudaStream_t,
                                           int);
template cudaError_t launch_transform<float>(const TransformArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_farfield<float>(const FarArgs<float>&, cudaStream_t);
template cudaError_t launch_spectrum_pack<float>(const float2*, const float2*, int, int, double, float2*, cudaStream_t);
template cudaError_t launch_pack_records<float>(const float2*, const float2*, int, int, int, const double*, double,
                                                long long, float2*, cudaStream_t);
}  // namespace pstd
