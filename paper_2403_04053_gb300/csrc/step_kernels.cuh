// Leapfrog PSTD step (Eq. PSTDupdating with the mask of Eqs. expmask, Gamma), split into
// three line passes that each apply one axis of the spectral kinetic operator
// K = sum_a F_a^-1[k_a^2 F_a] (Eq. spatialFFTeigen) to psi^n:
//
//   x pass:  prev <- psi^{n-1} - i (dt hbar eta / m) K_x psi^n - (2 i dt / hbar) (V-term + source)
//   y pass:  prev <- prev       - i (dt hbar eta / m) K_y psi^n
//   z pass:  prev <- Gamma * [prev - i (dt hbar eta / m) K_z psi^n]
//
// so the buffer that held psi^{n-1} ends up holding psi^{n+1}.  The V-term and the
// source sit in the x pass, whose epilogue walks the tile in memory order: its extra
// reads of psi^n inside the potential's support are coalesced and independent.  They
// are evaluated in registers from 1-D tables (no extra HBM traffic outside the
// potential's support):
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

// With PSTD_PREFETCH_PREV the y and z passes load the read-modify-write operand together
// with psi^n, so its latency overlaps the FFT instead of following it (more registers).
#ifndef PSTD_PREFETCH_PREV
#define PSTD_PREFETCH_PREV 0
#endif

// Minimum resident CTAs per SM requested from the register allocator: 4 CTAs of 256
// threads (64 registers each) let the 512 CTAs of a 128^3 pass run in one wave on 152 SMs.
template <typename R, int N> constexpr int pass_min_blocks()
{
    return (sizeof(R) == 4 && Plan<N>::T <= 8) ? (PSTD_PREFETCH_PREV ? 2 : 4) : 1;
}

template <typename R> __device__ __forceinline__ bool finite_c(R a, R b) { return isfinite(a) && isfinite(b); }

// psi_inc^n at node (x, y, z) of member b: s e^{i k_x (x - O_x)} e^{i k_y (y - O_y)} e^{i k_z (z - O_z)}
template <typename R, typename C>
__device__ __forceinline__ C incident_at(const StepArgs<R>& a, int b, C s, int x, int y, int z)
{
    return cmul(cmul(cmul(s, a.phase[0][b * a.nx + x]), a.phase[1][b * a.ny + y]), a.phase[2][b * a.nz + z]);
}

// ---------------------------------------------------------------------------------
// x pass: 32 consecutive rows per CTA, staged through shared memory (rows are
// contiguous, so the tile is one contiguous block of 32 * nx values)
// ---------------------------------------------------------------------------------
template <typename R, int N>
__global__ void __launch_bounds__(kLanes * Plan<N>::T, (pass_min_blocks<R, N>())) xpass_kernel(StepArgs<R> a)
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
    const C s = mk<C>(R(a.tfac[b].x), R(a.tfac[b].y));   // a(t_n) e^{-i w0 t_n}
    const R c2 = R(2.0 * a.dt / a.hbar);
    const bool paper = a.mode == PSTD_TFSF_PAPER;
    const int vnx = a.vhi[0] - a.vlo[0], vny = a.vhi[1] - a.vlo[1];
    for (int e = threadIdx.x; e < nrows * N; e += blockDim.x) {
        const int r = e / N, x = e - r * N;
        const C w = sm[x * kPitch + r];
        const C p = a.prev[tile0 + e];
        C acc = mk<C>(p.x + w.y, p.y - w.x);   // p - i w
        const int row = row0 + r, y = row % a.ny, z = row / a.ny;
        if (x >= a.vlo[0] && x < a.vhi[0] && y >= a.vlo[1] && y < a.vhi[1] && z >= a.vlo[2] && z < a.vhi[2]) {
            const R Vv = a.V[((long long)(z - a.vlo[2]) * vny + (y - a.vlo[1])) * vnx + (x - a.vlo[0])];
            C src = a.cur[tile0 + e];
            if (!paper) src = cadd(src, incident_at<R, C>(a, b, s, x, y, z));
            const R cv = c2 * Vv;
            acc.x += cv * src.y;
            acc.y -= cv * src.x;
        }
        if (paper && x > a.tf_lo[0] && x < a.tf_hi[0] && y > a.tf_lo[1] && y < a.tf_hi[1] && z > a.tf_lo[2] &&
            z < a.tf_hi[2]) {
            const R zx = a.zeta[0][x], zx1 = a.zeta1[0][x], zx2 = a.zeta2[0][x];
            const R zy = a.zeta[1][y], zy1 = a.zeta1[1][y], zy2 = a.zeta2[1][y];
            const R zz = a.zeta[2][z], zz1 = a.zeta1[2][z], zz2 = a.zeta2[2][z];
            const R lap = zx2 * zy * zz + zx * zy2 * zz + zx * zy * zz2;
            const MemberDev& md = a.mem[b];
            const R kg = R(md.k[0]) * zx1 * zy * zz + R(md.k[1]) * zx * zy1 * zz + R(md.k[2]) * zx * zy * zz1;
            // hbar^2/2m psi_inc (lap + 2 i kg), times -(2 i dt / hbar)
            const R h2m = R(a.hbar * a.hbar / (2.0 * a.mass));
            const C S = cscale(cmul(incident_at<R, C>(a, b, s, x, y, z), mk<C>(lap, R(2) * kg)), h2m);
            acc.x += c2 * S.y;
            acc.y -= c2 * S.x;
        }
        a.prev[tile0 + e] = acc;
    }
}

// ---------------------------------------------------------------------------------
// y pass: lines along y, 32 consecutive x per CTA (lane = x), coalesced in place
// ---------------------------------------------------------------------------------
template <typename R, int N>
__global__ void __launch_bounds__(kLanes * Plan<N>::T, (pass_min_blocks<R, N>())) ypass_kernel(StepArgs<R> a)
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
#if PSTD_PREFETCH_PREV
    C pv[E];
#pragma unroll
    for (int q = 0; q < E; ++q) pv[q] = act ? a.prev[base + slot_pos<N, T, R0>(q, j) * stride] : zero_c<R, C>();
#endif
    const R eta = R(a.mem[b].eta);
    kinetic_line<N, false>(v, sm, lane, j, a.tw[1], a.kin[1], eta);
    if (!act) return;
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const long long idx = base + slot_pos<N, T, R0>(q, j) * stride;
#if PSTD_PREFETCH_PREV
        const C p = pv[q];
#else
        const C p = a.prev[idx];
#endif
        a.prev[idx] = mk<C>(p.x + v[q].y, p.y - v[q].x);
    }
}

// ---------------------------------------------------------------------------------
// z pass: lines along z, lane = x; completes psi^{n+1} with the mask
// ---------------------------------------------------------------------------------
template <typename R, int N>
__global__ void __launch_bounds__(kLanes * Plan<N>::T, (pass_min_blocks<R, N>())) zpass_kernel(StepArgs<R> a)
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
#if PSTD_PREFETCH_PREV
    C pv[E];
#pragma unroll
    for (int q = 0; q < E; ++q) pv[q] = act ? a.prev[base + slot_pos<N, T, R0>(q, j) * stride] : zero_c<R, C>();
#endif
    kinetic_line<N, false>(v, sm, lane, j, a.tw[2], a.kin[2], R(a.mem[b].eta));
    if (!act) return;
    const R gxy = a.mask[0][x] * a.mask[1][y];
    bool ok = true;
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int z = slot_pos<N, T, R0>(q, j);
        const long long idx = base + z * stride;
#if PSTD_PREFETCH_PREV
        const C p = pv[q];
#else
        const C p = a.prev[idx];
#endif
        const R g = gxy * a.mask[2][z];
        const C acc = mk<C>(g * (p.x + v[q].y), g * (p.y - v[q].x));
        ok = ok && finite_c<R>(acc.x, acc.y);
        a.prev[idx] = acc;
    }
    if (!ok) atomicOr(a.flag, 1);
}

// ---------------------------------------------------------------------------------
// running DFT on the two virtual planes normal to one axis (Eqs. psiphasor, dpsiphasor).
// d psi / d a at the plane node h is the spectral derivative sum_q D_h(q) psi(q) with
// D_h(q) = (1/N) sum_m i k_m e^{2 pi i m (h - q)/N}, formed in the working precision; the
// products with e^{i omega t_n} are accumulated in double precision.  Lines along y and z:
// one thread per line, lanes over x (coalesced).  Lines along x: one warp per line, lanes
// over x, reduced with shuffles.
// ---------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void dft_accumulate(const DftArgs<R>& a, int b, long long pix, const double2* __restrict__ ef, int nfreq,
                                               typename DftArgs<R>::C p0, typename DftArgs<R>::C p1,
                                               typename DftArgs<R>::C d0, typename DftArgs<R>::C d1)
{
    const int f0 = 2 * a.axis, f1 = 2 * a.axis + 1;
    for (int f = 0; f < nfreq; ++f) {
        const double2 e = ef[(long long)f * a.phase_len];
        const double cf = e.x, sf = e.y;
        double2* accf = a.acc + (long long)b * a.acc_member_stride + (long long)f * a.acc_freq_stride;
        double2* ps0 = accf + a.face_off[f0] + pix;
        double2* dp0 = accf + a.face_off[f0] + a.face_size[f0] + pix;
        double2* ps1 = accf + a.face_off[f1] + pix;
        double2* dp1 = accf + a.face_off[f1] + a.face_size[f1] + pix;
        const double q0x = p0.x, q0y = p0.y, q1x = p1.x, q1y = p1.y;
        const double e0x = d0.x, e0y = d0.y, e1x = d1.x, e1y = d1.y;
        ps0->x += q0x * cf - q0y * sf;  ps0->y += q0x * sf + q0y * cf;
        ps1->x += q1x * cf - q1y * sf;  ps1->y += q1x * sf + q1y * cf;
        dp0->x += e0x * cf - e0y * sf;  dp0->y += e0x * sf + e0y * cf;
        dp1->x += e1x * cf - e1y * sf;  dp1->y += e1x * sf + e1y * cf;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) plane_dft_kernel(DftArgs<R> a)
{
    using C = typename DftArgs<R>::C;
    const int b = blockIdx.y;
    if (!((a.member_mask >> b) & 1ull)) return;
    const MemberDev& md = a.mem[b];
    const int nfreq = md.nfreq;
    // e^{+i omega_f t_n} for this member and window step, from the host-built table
    const double2* ef = a.phase + (long long)b * a.phase_member_stride + (a.step - a.window_first[b]);
    const long long cbase = (long long)b * a.ncell;
    if (a.axis == 0) {
        // one warp per x line; lines indexed (y, z); plane [z][y]
        const int lane = threadIdx.x & 31;
        const long long line = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
        if (line >= (long long)a.ny * a.nz) return;
        const C* row = a.cur + cbase + line * a.nx;
        C d0 = zero_c<R, C>(), d1 = zero_c<R, C>();
        for (int q = lane; q < a.nx; q += 32) {
            const C v = row[q], w0 = a.dw[q], w1 = a.dw[a.nx + q];
            d0 = cadd(d0, cmul(v, w0));
            d1 = cadd(d1, cmul(v, w1));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            d0.x += __shfl_xor_sync(0xffffffffu, d0.x, o);
            d0.y += __shfl_xor_sync(0xffffffffu, d0.y, o);
            d1.x += __shfl_xor_sync(0xffffffffu, d1.x, o);
            d1.y += __shfl_xor_sync(0xffffffffu, d1.y, o);
        }
        if (lane == 0) dft_accumulate<R>(a, b, line, ef, nfreq, row[a.h[0]], row[a.h[1]], d0, d1);
        return;
    }
    // lines along y or z: 32 lanes over x (coalesced) x 8 segments of the line per CTA,
    // partial sums reduced through shared memory
    constexpr int SEG = 8, MAXQ = 48;   // 8 segments of at most 48 nodes cover lines up to 384
    __shared__ C red[SEG][2][32];
    const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const long long line = (long long)blockIdx.x * 32 + lane;
    int n, u, w, nu;
    long long stride, base;
    const long long nlines = a.axis == 1 ? (long long)a.nx * a.nz : (long long)a.nx * a.ny;
    const bool act = line < nlines;
    const long long ln = act ? line : 0;
    if (a.axis == 1) {            // lines along y; lines (x, z); plane [z][x]
        n = a.ny; nu = a.nx;
        u = (int)(ln % a.nx); w = (int)(ln / a.nx);
        stride = a.nx;
        base = (long long)w * a.nx * a.ny + u;
    } else {                      // lines along z; lines (x, y); plane [y][x]
        n = a.nz; nu = a.nx;
        u = (int)(ln % a.nx); w = (int)(ln / a.nx);
        stride = (long long)a.nx * a.ny;
        base = (long long)w * a.nx + u;
    }
    const C* col = a.cur + cbase + base;
    const int per = (n + SEG - 1) / SEG;
    const int q0 = seg * per, q1 = min(n, q0 + per);
    C d0 = zero_c<R, C>(), d1 = zero_c<R, C>();
    if (act) {
        C vals[16];
#pragma unroll
        for (int c0 = 0; c0 < MAXQ; c0 += 16) {
            if (q0 + c0 >= q1) break;
#pragma unroll
            for (int i = 0; i < 16; ++i) vals[i] = q0 + c0 + i < q1 ? col[(long long)(q0 + c0 + i) * stride] : zero_c<R, C>();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int q = q0 + c0 + i;
                if (q < q1) {
                    d0 = cadd(d0, cmul(vals[i], a.dw[q]));
                    d1 = cadd(d1, cmul(vals[i], a.dw[n + q]));
                }
            }
        }
    }
    red[seg][0][lane] = d0;
    red[seg][1][lane] = d1;
    __syncthreads();
    if (seg != 0 || !act) return;
#pragma unroll
    for (int s2 = 1; s2 < SEG; ++s2) {
        d0 = cadd(d0, red[s2][0][lane]);
        d1 = cadd(d1, red[s2][1][lane]);
    }
    dft_accumulate<R>(a, b, (long long)w * nu + u, ef, nfreq, col[a.h[0] * stride], col[a.h[1] * stride], d0, d1);
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
    const long long lines = a.axis == 0 ? (long long)a.ny * a.nz : a.axis == 1 ? (long long)a.nx * a.nz : (long long)a.nx * a.ny;
    const long long per_block = a.axis == 0 ? 8 : 32;   // x lines: one warp each; y, z lines: 32 per CTA
    dim3 grid((unsigned)((lines + per_block - 1) / per_block), batch);
    plane_dft_kernel<R><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pstd
