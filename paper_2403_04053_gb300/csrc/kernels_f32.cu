// Single-precision instantiations of the step, plane-DFT and transform kernels.
#include "ntdf_kernels.cuh"
#include "step_kernels.cuh"

namespace pstd {
template cudaError_t launch_xpass<float>(const StepArgs<float>&, int, cudaStream_t);
template cudaError_t launch_ypass<float>(const StepArgs<float>&, int, cudaStream_t);
template cudaError_t launch_zpass<float>(const StepArgs<float>&, int, cudaStream_t);
template cudaError_t launch_plane_dft<float>(const DftArgs<float>&, int, cudaStream_t);
template cudaError_t launch_transform<float>(const TransformArgs<float>&, int, int, bool, cudaStream_t);
template cudaError_t launch_pack_records<float>(const double2*, const double2*, int, int, int, const double*, double,
                                                long long, float2*, cudaStream_t);
}  // namespace pstd
