// Helper kernels: a tiled complex GEMM (single or double precision) used to evaluate the
// trigonometric interpolant at the Gauss-Legendre nodes of every surface cell and the plane
// spectra of the far field, an FP64 -> working-precision conversion, and the fixed-order
// reduction of per-split partial sums of the surface transform.
#include "pstd_internal.h"

namespace pstd {

namespace {
constexpr int kTile = 16;

template <typename C>
__global__ void cgemm_kernel(int M, int N, int K, const C* __restrict__ A, int lda, const C* __restrict__ B, int ldb,
                             C* __restrict__ Cm, int ldc, double2 alpha)
{
    using R = decltype(C::x);
    __shared__ C As[kTile][kTile];
    __shared__ C Bs[kTile][kTile + 1];
    const int row = blockIdx.y * kTile + threadIdx.y;
    const int col = blockIdx.x * kTile + threadIdx.x;
    R sx = 0, sy = 0;
    C zero;
    zero.x = 0;
    zero.y = 0;
    for (int k0 = 0; k0 < K; k0 += kTile) {
        const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
        As[threadIdx.y][threadIdx.x] = (row < M && ka < K) ? A[(long long)row * lda + ka] : zero;
        Bs[threadIdx.y][threadIdx.x] = (kb < K && col < N) ? B[(long long)kb * ldb + col] : zero;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTile; ++kk) {
            const C a = As[threadIdx.y][kk], b = Bs[kk][threadIdx.x];
            sx += a.x * b.x - a.y * b.y;
            sy += a.x * b.y + a.y * b.x;
        }
        __syncthreads();
    }
    if (row < M && col < N) {
        C out;
        out.x = R(alpha.x) * sx - R(alpha.y) * sy;
        out.y = R(alpha.x) * sy + R(alpha.y) * sx;
        Cm[(long long)row * ldc + col] = out;
    }
}

template <typename C>
__global__ void convert_kernel(const double2* __restrict__ in, C* __restrict__ out, long long n)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    C v;
    v.x = decltype(C::x)(in[e].x);
    v.y = decltype(C::x)(in[e].y);
    out[e] = v;
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

template <typename C>
cudaError_t launch_cgemm(int M, int N, int K, const C* A, int lda, const C* B, int ldb, C* Cm, int ldc, double2 alpha,
                         cudaStream_t s)
{
    dim3 block(kTile, kTile), grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
    cgemm_kernel<C><<<grid, block, 0, s>>>(M, N, K, A, lda, B, ldb, Cm, ldc, alpha);
    return cudaGetLastError();
}
template cudaError_t launch_cgemm<float2>(int, int, int, const float2*, int, const float2*, int, float2*, int, double2,
                                          cudaStream_t);
template cudaError_t launch_cgemm<double2>(int, int, int, const double2*, int, const double2*, int, double2*, int, double2,
                                           cudaStream_t);

template <typename C> cudaError_t launch_convert(const double2* in, C* out, long long n, cudaStream_t s)
{
    convert_kernel<C><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}
template cudaError_t launch_convert<float2>(const double2*, float2*, long long, cudaStream_t);
template cudaError_t launch_convert<double2>(const double2*, double2*, long long, cudaStream_t);

cudaError_t launch_reduce_partials(const double2* partial, int splits, long long M, double2* out, double* dsdo,
                                   cudaStream_t s)
{
    reduce_partials_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(partial, splits, M, out, dsdo);
    return cudaGetLastError();
}

}  // namespace pstd
