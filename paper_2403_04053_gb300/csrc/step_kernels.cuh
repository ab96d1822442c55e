// Leapfrog PSTD step (Eq. PSTDupdating with the mask of Eqs. expmask, Gamma), split into
// three line passes that each apply one axis of the spectral kinetic operator
// K = sum_a F_a^-1[k_a^2 F_a] (Eq. spatialFFTeigen) to psi^n:
//
//   x pass:  prev <- psi^{n-1} - i (dt hbar eta / m) K_x psi^n
//   y pass:  prev <- prev       - i (dt hbar eta / m) K_y psi^n
//   z pass:  prev <- Gamma * [prev - i (dt hbar eta / m) K_z psi^n - (2 i dt / hbar) (V-term + source)]
//
// so the buffer that held psi^{n-1} ends up holding psi^{n+1}.  The V-term and the
// source are evaluated in registers from 1-D tables (no extra HBM traffic outside
// the potential's support):
//   EXACT form : V (psi^n + psi_inc^n)                       (state = scattered field)
//   PAPER form : V psi~^n + hbar^2/2m psi_inc^n [lap zeta + 2 i k . grad zeta]  (Eq. tildeSchrodinger)
// with psi_inc^n(r) = a(t_n) e^{-i w0 t_n} prod_a e^{i k_a (x_a - r_O,a)}; the time factor
// is evaluated in double precision from n on the device.
#pragma once

#include <type_traits>

#include "fft_line.cuh"
#include "pstd_internal.h"

namespace pstd {

__device__ __forceinline__ double envelope_dev(double t, double ramp)
{
    if (ramp <= 0.0 || t >= ramp) return 1.0;
    if (t <= 0.0) return 0.0;
    return 0.5 * (1.0 - cos(3.14159265358979323846 * t / ramp));
}

template <typename R, typename C> __device__ __forceinline__ C zero_c() { return mk<C>(R(0), R(0)); }

template <typename R> __device__ __forceinline__ bool finite_c(R a, R b) { return isfinite(a) && isfinite(b); }

// ---------------------------------------------------------------------------------
// x pass: 32 consecutive rows per CTA, staged through shared memory (rows are
// contiguous, so the tile is one contiguous block of 32 * nx values)
// ---------------------------------------------------------------------------------
template <typename R, int N>
__global__ void __launch_bounds__(kLanes * Plan<N>::T) xpass_kernel(StepArgs<R> a)
{
    using C = typename StepArgs<R>::C;
    constexpr int T = Plan<N>::T, E = N / T, R0 = Plan<N>::R[0];
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int lane = threadIdx.x & 31, j = threadIdx.x >> 5;
    const int b = blockIdx.y;
    const int rows = a.ny * a.nz;
    const int row0 = blockIdx.x * kLanes;
    const int nrows = min(kLanes, rows - row0);
    const long long tile0 = (long long)b * a.ncell + (long long)row0 * N;
    for (int e = threadIdx.x; e < kLanes * N; e += blockDim.x) {
        const int r = e / N, x = e - r * N;
        sm[x * kPitch + r] = r < nrows ? a.cur[tile0 + e] : zero_c<R, C>();
    }
    __syncthreads();
    C v[E];
    const R eta = R(a.mem[b].eta);
    kinetic_line<N, true>(v, sm, lane, j, a.tw[0], a.kin[0], eta);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < E; ++q) sm[slot_pos<N, T, R0>(q, j) * kPitch + lane] = v[q];
    __syncthreads();
    for (int e = threadIdx.x; e < nrows * N; e += blockDim.x) {
        const int r = e / N, x = e - r * N;
        const C w = sm[x * kPitch + r];
        const C p = a.prev[tile0 + e];
        a.prev[tile0 + e] = mk<C>(p.x + w.y, p.y - w.x);   // p - i w
    }
}

// ---------------------------------------------------------------------------------
// y pass: lines along y, 32 consecutive x per CTA (lane = x), coalesced in place
// ---------------------------------------------------------------------------------
template <typename R, int N>
__global__ void __launch_bounds__(kLanes * Plan<N>::T) ypass_kernel(StepArgs<R> a)
{
    using C = typename StepArgs<R>::C;
    constexpr int T = Plan<N>::T, E = N / T, R0 = Plan<N>::R[0];
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int lane = threadIdx.x & 31, j = threadIdx.x >> 5;
    const int x = blockIdx.x * kLanes + lane;
    const int z = blockIdx.y, b = blockIdx.z;
    const bool act = x < a.nx;
    const long long stride = a.nx;
    const long long base = (long long)b * a.ncell + (long long)z * a.nx * a.ny + x;
    C v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = act ? a.cur[base + slot_pos<N, T, R0>(q, j) * stride] : zero_c<R, C>();
    const R eta = R(a.mem[b].eta);
    kinetic_line<N, false>(v, sm, lane, j, a.tw[1], a.kin[1], eta);
    if (!act) return;
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const long long idx = base + slot_pos<N, T, R0>(q, j) * stride;
        const C p = a.prev[idx];
        a.prev[idx] = mk<C>(p.x + v[q].y, p.y - v[q].x);
    }
}

// ---------------------------------------------------------------------------------
// z pass: lines along z, lane = x; completes psi^{n+1} with V, source and mask
// ---------------------------------------------------------------------------------
template <typename R, int N>
__global__ void __launch_bounds__(kLanes * Plan<N>::T) zpass_kernel(StepArgs<R> a)
{
    using C = typename StepArgs<R>::C;
    constexpr int T = Plan<N>::T, E = N / T, R0 = Plan<N>::R[0];
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int lane = threadIdx.x & 31, j = threadIdx.x >> 5;
    const int x = blockIdx.x * kLanes + lane;
    const int y = blockIdx.y, b = blockIdx.z;
    const bool act = x < a.nx;
    const long long stride = (long long)a.nx * a.ny;
    const long long base = (long long)b * a.ncell + (long long)y * a.nx + x;
    C v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = act ? a.cur[base + slot_pos<N, T, R0>(q, j) * stride] : zero_c<R, C>();
    const MemberDev md = a.mem[b];
    kinetic_line<N, false>(v, sm, lane, j, a.tw[2], a.kin[2], R(md.eta));
    if (!act) return;

    // incident wave at (x, y, .): a(t_n) e^{-i w0 t_n} e^{i k_x (x - O_x)} e^{i k_y (y - O_y)}
    const double t = (double)a.step * a.dt;
    const double env = envelope_dev(t, md.ramp);
    double sw, cw;
    sincos(md.w0 * t, &sw, &cw);
    const C s = mk<C>(R(env * cw), R(-env * sw));
    const C pxy = cmul(cmul(s, a.phase[0][b * a.nx + x]), a.phase[1][b * a.ny + y]);
    const R gxy = a.mask[0][x] * a.mask[1][y];
    const R c2 = R(2.0 * a.dt / a.hbar);
    const bool in_vxy = x >= a.vlo[0] && x < a.vhi[0] && y >= a.vlo[1] && y < a.vhi[1];
    const int vnx = a.vhi[0] - a.vlo[0], vny = a.vhi[1] - a.vlo[1];
    const bool paper = a.mode == PSTD_TFSF_PAPER;
    const bool in_tfxy = paper && x > a.tf_lo[0] && x < a.tf_hi[0] && y > a.tf_lo[1] && y < a.tf_hi[1];
    R zx = 0, zx1 = 0, zx2 = 0, zy = 0, zy1 = 0, zy2 = 0;
    if (in_tfxy) {
        zx = a.zeta[0][x]; zx1 = a.zeta1[0][x]; zx2 = a.zeta2[0][x];
        zy = a.zeta[1][y]; zy1 = a.zeta1[1][y]; zy2 = a.zeta2[1][y];
    }
    bool ok = true;
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int z = slot_pos<N, T, R0>(q, j);
        const long long idx = base + z * stride;
        const C p = a.prev[idx];
        C acc = mk<C>(p.x + v[q].y, p.y - v[q].x);
        if (in_vxy && z >= a.vlo[2] && z < a.vhi[2]) {
            const R Vv = a.V[((long long)(z - a.vlo[2]) * vny + (y - a.vlo[1])) * vnx + (x - a.vlo[0])];
            C src = a.cur[idx];
            if (!paper) src = cadd(src, cmul(pxy, a.phase[2][b * a.nz + z]));
            const R cv = c2 * Vv;
            acc.x += cv * src.y;
            acc.y -= cv * src.x;
        }
        if (in_tfxy && z > a.tf_lo[2] && z < a.tf_hi[2]) {
            const R zz = a.zeta[2][z], zz1 = a.zeta1[2][z], zz2 = a.zeta2[2][z];
            const R lap = zx2 * zy * zz + zx * zy2 * zz + zx * zy * zz2;
            const R kg = R(md.k[0]) * zx1 * zy * zz + R(md.k[1]) * zx * zy1 * zz + R(md.k[2]) * zx * zy * zz1;
            const C pinc = cmul(pxy, a.phase[2][b * a.nz + z]);
            // hbar^2/2m psi_inc (lap + 2 i kg), times -(2 i dt / hbar)
            const R h2m = R(a.hbar * a.hbar / (2.0 * a.mass));
            const C S = cscale(cmul(pinc, mk<C>(lap, R(2) * kg)), h2m);
            acc.x += c2 * S.y;
            acc.y -= c2 * S.x;
        }
        const R g = gxy * a.mask[2][z];
        acc = cscale(acc, g);
        ok = ok && finite_c<R>(acc.x, acc.y);
        a.prev[idx] = acc;
    }
    if (!ok) atomicOr(a.flag, 1);
}

// ---------------------------------------------------------------------------------
// running DFT on the two virtual planes normal to one axis (Eqs. psiphasor, dpsiphasor):
// one thread per line along the axis; d psi / d a at the plane node h is the spectral
// derivative sum_q D_h(q) psi(q) with D_h(q) = (1/N) sum_m i k_m e^{2 pi i m (h - q)/N}
// ---------------------------------------------------------------------------------
template <typename R>
__global__ void plane_dft_kernel(DftArgs<R> a)
{
    using C = typename DftArgs<R>::C;
    const int b = blockIdx.y;
    if (!((a.member_mask >> b) & 1ull)) return;
    const long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int n, u, w;          // line length, fast and slow line coordinates
    long long stride, base;
    int nu;               // extent of the fast line coordinate (pixel = w * nu + u)
    if (a.axis == 0) {            // lines along x; lines indexed (y, z); plane [z][y]
        n = a.nx; nu = a.ny;
        if (line >= (long long)a.ny * a.nz) return;
        u = (int)(line % a.ny); w = (int)(line / a.ny);
        stride = 1;
        base = ((long long)w * a.ny + u) * a.nx;
    } else if (a.axis == 1) {     // lines along y; lines (x, z); plane [z][x]
        n = a.ny; nu = a.nx;
        if (line >= (long long)a.nx * a.nz) return;
        u = (int)(line % a.nx); w = (int)(line / a.nx);
        stride = a.nx;
        base = (long long)w * a.nx * a.ny + u;
    } else {                      // lines along z; lines (x, y); plane [y][x]
        n = a.nz; nu = a.nx;
        if (line >= (long long)a.nx * a.ny) return;
        u = (int)(line % a.nx); w = (int)(line / a.nx);
        stride = (long long)a.nx * a.ny;
        base = (long long)w * a.nx + u;
    }
    base += (long long)b * a.ncell;
    double d0x = 0, d0y = 0, d1x = 0, d1y = 0;
    for (int q = 0; q < n; ++q) {
        const C val = a.cur[base + q * stride];
        const C w0 = a.dw[q], w1 = a.dw[n + q];
        d0x += double(val.x * w0.x - val.y * w0.y);
        d0y += double(val.x * w0.y + val.y * w0.x);
        d1x += double(val.x * w1.x - val.y * w1.y);
        d1y += double(val.x * w1.y + val.y * w1.x);
    }
    const C p0 = a.cur[base + a.h[0] * stride];
    const C p1 = a.cur[base + a.h[1] * stride];
    const long long pix = (long long)w * nu + u;
    const MemberDev& md = a.mem[b];
    const double t = (double)a.step * a.dt;
    for (int f = 0; f < md.nfreq; ++f) {
        double sf, cf;
        sincos(md.omega[f] * t, &sf, &cf);       // e^{+i omega t_n}
        double2* accf = a.acc + (long long)b * a.acc_member_stride + (long long)f * a.acc_freq_stride;
        const int f0 = 2 * a.axis, f1 = 2 * a.axis + 1;
        double2* ps0 = accf + a.face_off[f0] + pix;
        double2* dp0 = accf + a.face_off[f0] + a.face_size[f0] + pix;
        double2* ps1 = accf + a.face_off[f1] + pix;
        double2* dp1 = accf + a.face_off[f1] + a.face_size[f1] + pix;
        const double q0x = p0.x, q0y = p0.y, q1x = p1.x, q1y = p1.y;
        ps0->x += q0x * cf - q0y * sf;  ps0->y += q0x * sf + q0y * cf;
        ps1->x += q1x * cf - q1y * sf;  ps1->y += q1x * sf + q1y * cf;
        dp0->x += d0x * cf - d0y * sf;  dp0->y += d0x * sf + d0y * cf;
        dp1->x += d1x * cf - d1y * sf;  dp1->y += d1x * sf + d1y * cf;
    }
}

// ---------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------
template <typename R, int N> size_t pass_smem() { return sizeof(typename StepArgs<R>::C) * (size_t)N * kPitch; }

template <typename R, int N> cudaError_t xpass_n(const StepArgs<R>& a, int batch, cudaStream_t s)
{
    const size_t sm = pass_smem<R, N>();
    cudaError_t e = cudaFuncSetAttribute(xpass_kernel<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.ny * a.nz + kLanes - 1) / kLanes, batch);
    xpass_kernel<R, N><<<grid, kLanes * Plan<N>::T, sm, s>>>(a);
    return cudaGetLastError();
}
template <typename R, int N> cudaError_t ypass_n(const StepArgs<R>& a, int batch, cudaStream_t s)
{
    const size_t sm = pass_smem<R, N>();
    cudaError_t e = cudaFuncSetAttribute(ypass_kernel<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.nx + kLanes - 1) / kLanes, a.nz, batch);
    ypass_kernel<R, N><<<grid, kLanes * Plan<N>::T, sm, s>>>(a);
    return cudaGetLastError();
}
template <typename R, int N> cudaError_t zpass_n(const StepArgs<R>& a, int batch, cudaStream_t s)
{
    const size_t sm = pass_smem<R, N>();
    cudaError_t e = cudaFuncSetAttribute(zpass_kernel<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.nx + kLanes - 1) / kLanes, a.ny, batch);
    zpass_kernel<R, N><<<grid, kLanes * Plan<N>::T, sm, s>>>(a);
    return cudaGetLastError();
}

#define PSTD_SIZE_DISPATCH(FN, n, ...)                 \
    switch (n) {                                        \
    case 8: return FN<R, 8>(__VA_ARGS__);               \
    case 12: return FN<R, 12>(__VA_ARGS__);             \
    case 16: return FN<R, 16>(__VA_ARGS__);             \
    case 24: return FN<R, 24>(__VA_ARGS__);             \
    case 32: return FN<R, 32>(__VA_ARGS__);             \
    case 48: return FN<R, 48>(__VA_ARGS__);             \
    case 64: return FN<R, 64>(__VA_ARGS__);             \
    case 96: return FN<R, 96>(__VA_ARGS__);             \
    case 128: return FN<R, 128>(__VA_ARGS__);           \
    case 192: return FN<R, 192>(__VA_ARGS__);           \
    case 256: return FN<R, 256>(__VA_ARGS__);           \
    case 384: return FN<R, 384>(__VA_ARGS__);           \
    default: return cudaErrorInvalidValue;              \
    }

template <typename R> cudaError_t launch_xpass(const StepArgs<R>& a, int batch, cudaStream_t s)
{
    PSTD_SIZE_DISPATCH(xpass_n, a.nx, a, batch, s)
}
template <typename R> cudaError_t launch_ypass(const StepArgs<R>& a, int batch, cudaStream_t s)
{
    PSTD_SIZE_DISPATCH(ypass_n, a.ny, a, batch, s)
}
template <typename R> cudaError_t launch_zpass(const StepArgs<R>& a, int batch, cudaStream_t s)
{
    PSTD_SIZE_DISPATCH(zpass_n, a.nz, a, batch, s)
}
template <typename R> cudaError_t launch_plane_dft(const DftArgs<R>& a, int batch, cudaStream_t s)
{
    long long lines = a.axis == 0 ? (long long)a.ny * a.nz : a.axis == 1 ? (long long)a.nx * a.nz : (long long)a.nx * a.ny;
    dim3 grid((unsigned)((lines + 127) / 128), batch);
    plane_dft_kernel<R><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pstd
