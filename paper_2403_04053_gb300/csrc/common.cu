// Precision-independent helper kernels: a tiled complex-double GEMM used to evaluate the
// trigonometric interpolant at the Gauss-Legendre nodes of every surface cell, and the
// fixed-order reduction of per-split partial sums of the surface transform.
#include "pstd_internal.h"

namespace pstd {

namespace {
constexpr int kTile = 16;

__global__ void zgemm_kernel(int M, int N, int K, const double2* __restrict__ A, int lda, const double2* __restrict__ B,
                             int ldb, double2* __restrict__ C, int ldc, double2 alpha)
{
    __shared__ double2 As[kTile][kTile];
    __shared__ double2 Bs[kTile][kTile + 1];
    const int row = blockIdx.y * kTile + threadIdx.y;
    const int col = blockIdx.x * kTile + threadIdx.x;
    double sx = 0.0, sy = 0.0;
    for (int k0 = 0; k0 < K; k0 += kTile) {
        const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
        As[threadIdx.y][threadIdx.x] = (row < M && ka < K) ? A[(long long)row * lda + ka] : make_double2(0.0, 0.0);
        Bs[threadIdx.y][threadIdx.x] = (kb < K && col < N) ? B[(long long)kb * ldb + col] : make_double2(0.0, 0.0);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTile; ++kk) {
            const double2 a = As[threadIdx.y][kk], b = Bs[kk][threadIdx.x];
            sx += a.x * b.x - a.y * b.y;
            sy += a.x * b.y + a.y * b.x;
        }
        __syncthreads();
    }
    if (row < M && col < N)
        C[(long long)row * ldc + col] = make_double2(alpha.x * sx - alpha.y * sy, alpha.x * sy + alpha.y * sx);
}

__global__ void reduce_partials_kernel(const double2* __restrict__ partial, int splits, long long M, double2* __restrict__ out,
                                       double* __restrict__ dsdo)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < splits; ++s) {
        const double2 v = partial[(long long)s * M + p];
        sx += v.x;
        sy += v.y;
    }
    if (out) out[p] = make_double2(sx, sy);
    if (dsdo) dsdo[p] = sx * sx + sy * sy;
}
}  // namespace

cudaError_t launch_zgemm(int M, int N, int K, const double2* A, int lda, const double2* B, int ldb, double2* C, int ldc,
                         double2 alpha, cudaStream_t s)
{
    dim3 block(kTile, kTile), grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
    zgemm_kernel<<<grid, block, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double2* partial, int splits, long long M, double2* out, double* dsdo,
                                   cudaStream_t s)
{
    reduce_partials_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(partial, splits, M, out, dsdo);
    return cudaGetLastError();
}

}  // namespace pstd
