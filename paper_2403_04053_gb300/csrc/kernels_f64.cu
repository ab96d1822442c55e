// Double-precision instantiations of the step (with the fused running DFT) and transform kernels.
#include "ntdf_kernels.cuh"
#include "step_kernels.cuh"

namespace pstd {
template cudaError_t launch_xpass<double>(const StepArgs<double>&, const DftArgs<double>*, int, cudaStream_t);
template cudaError_t launch_ypass<double>(const StepArgs<double>&, const DftArgs<double>*, int, cudaStream_t);
template cudaError_t launch_source<double>(const StepArgs<double>&, int, cudaStream_t);
template cudaError_t launch_aux_table<double>(const double2*, const double*, const double*, int, int, long long, long, bool,
                                           double2*, double2*, cudaStream_t);
template cudaError_t launch_aux_eval<double>(const AuxEvalArgs<double>&, cudaStream_t);
template bool xypass_available<double>(int, int, int);
template bool pipe_y_available<double>(int);
template bool tma_pass_available<double>(int);
template cudaError_t launch_xypass<double>(const StepArgs<double>&, const DftArgs<double>*, const DftArgs<double>*, int, cudaStream_t,
                                           int);
template cudaError_t launch_transform<double>(const TransformArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_farfield<double>(const FarArgs<double>&, cudaStream_t);
template cudaError_t launch_spectrum_pack<double>(const double2*, const double2*, int, int, double, double2*, cudaStream_t);
template cudaError_t launch_pack_records<double>(const double2*, const double2*, int, int, int, const double*, double,
                                                long long, double2*, cudaStream_t);
}  // namespace pstd
