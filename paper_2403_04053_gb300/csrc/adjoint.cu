// Instantiations of the adjoint kernels (single and double precision).
#include "adjoint_kernels.cuh"

namespace pstd {
#define PSTD_ADJOINT_INSTANTIATE(R, C)                                                                          \
    template cudaError_t launch_injection<R>(const InjectionArgs<R>&, cudaStream_t);                             \
    template cudaError_t launch_inject<R>(C*, const C*, C, long long, cudaStream_t);                              \
    template cudaError_t launch_grad<R>(const GradArgs<R>&, cudaStream_t);                                        \
    template cudaError_t launch_adj_points<R>(const AdjointTransformArgs<R>&, cudaStream_t);                      \
    template cudaError_t launch_transform_adjoint<R>(const AdjointTransformArgs<R>&, int, int, cudaStream_t);     \
    template cudaError_t launch_sum_splits<R>(const C*, int, long long, C*, cudaStream_t);                        \
    template cudaError_t launch_unpack_records<R>(const C*, int, int, int, const double*, double, long long, C*,   \
                                                  C*, cudaStream_t);                                             \
    template cudaError_t launch_widen<R>(const C*, double2*, long long, cudaStream_t);
PSTD_ADJOINT_INSTANTIATE(float, float2)
PSTD_ADJOINT_INSTANTIATE(double, double2)
#undef PSTD_ADJOINT_INSTANTIATE
}  // namespace pstd
