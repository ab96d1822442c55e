// Leapfrog PSTD step (Eq. PSTDupdating with the mask of Eqs. expmask, Gamma), split into
// three line passes that each apply one axis of the spectral kinetic operator
// K = sum_a F_a^-1[k_a^2 F_a] (Eq. spatialFFTeigen) to psi^n:
//
//   source:  prev <- psi^{n-1} - (2 i dt / hbar) (V-term + source)   (support box only)
//   x pass:  prev <- prev - i (dt hbar eta / m) K_x psi^n
//   y pass:  prev <- prev - i (dt hbar eta / m) K_y psi^n
//   z pass:  prev <- Gamma * [prev - i (dt hbar eta / m) K_z psi^n]
//
// so the buffer that held psi^{n-1} ends up holding psi^{n+1}.  The V-term and the
// source run as their own element-wise kernel over the box where they are non-zero
// (one independent read-modify-write per cell, nothing serialised behind an FFT),
// evaluated in registers from 1-D tables:
//   EXACT form : V (psi^n + psi_inc^n)                       (state = scattered field)
//   PAPER form : V psi~^n + hbar^2/2m psi_inc^n [lap zeta + 2 i k . grad zeta]  (Eq. tildeSchrodinger)
// with psi_inc^n(r) = a(t_n) e^{-i w0 t_n} prod_a e^{i k_a (x_a - r_O,a)}; the time factor
// is tabulated in double precision on the host for the steps of each pstd_step call.
#pragma once

#include <algorithm>
#include <type_traits>

#include "fft_line.cuh"
#include "pstd_internal.h"

namespace pstd {

template <typename R, typename C> __device__ __forceinline__ C zero_c() { return mk<C>(R(0), R(0)); }

// With PSTD_PREFETCH_PREV the y and z passes load the read-modify-write operand together
// with psi^n, so its latency overlaps the FFT instead of following it (more registers).
#ifndef PSTD_PREFETCH_PREV
#define PSTD_PREFETCH_PREV 0
#endif
// The z pass on lines of 192 points or more asks for its read-modify-write operand's lines in
// L1 before its FFT when the state does not fit in L2 (StepArgs::pf_l1, set on the host): a
// hint (no registers, no fault on the in-bounds addresses it is given) that takes 13% off the
// 256^3 z pass.  In the 128-point pass the code alone, even switched off, cost 5%.
template <typename T> __device__ __forceinline__ void prefetch_l1(const T* p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Minimum resident CTAs per SM requested from the register allocator (64 registers a
// thread, 2048 threads an SM): 4 CTAs of 256 threads let the 512 CTAs of a 128^3 pass run
// in one wave on 152 SMs; for the 512-thread CTAs of N = 192 and 256 (at most 16 values a
// thread) 2 CTAs, so that HBM-bound passes keep enough loads in flight.
template <typename R, int N, int PL = 0> constexpr int pass_min_blocks()
{
    return !(sizeof(R) == 4) ? 1
           : Plan<N, PL>::T <= 8 ? (PSTD_PREFETCH_PREV ? 2 : 4) * (32 / kLanes)
           : (Plan<N, PL>::T == 16 && N / Plan<N, PL>::T <= 16) ? 2 * (32 / kLanes)
           : 1;
}

template <typename R> __device__ __forceinline__ bool finite_c(R a, R b) { return isfinite(a) && isfinite(b); }

// Programmatic dependent launch between the kernels of the step: each step kernel is
// launched so that it may be scheduled while the previous one drains, and waits for the
// previous grid's completion (and memory) at griddepcontrol.wait before it touches the
// state; launch_dependents right after lets the next kernel be scheduled as soon as all of
// this grid's CTAs are resident.  Without the launch attribute both are no-ops.
#ifndef PSTD_PDL
#define PSTD_PDL 1
#endif
__device__ __forceinline__ void step_kernel_entry()
{
#if PSTD_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

template <typename Kern, typename... Args>
cudaError_t launch_step_kernel(Kern kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const Args&... args)
{
#if PSTD_PDL
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
#else
    kernel<<<grid, block, smem, s>>>(args...);
    return cudaGetLastError();
#endif
}

// psi_inc^n at node (x, y, z) of member b: s e^{i k_x (x - O_x)} e^{i k_y (y - O_y)} e^{i k_z (z - O_z)}
template <typename R, typename C>
__device__ __forceinline__ C incident_at(const StepArgs<R>& a, int b, C s, int x, int y, int z)
{
    return cmul(cmul(cmul(s, a.phase[0][b * a.nx + x]), a.phase[1][b * a.ny + y]), a.phase[2][b * a.nz + z]);
}

// ---------------------------------------------------------------------------------
// running DFT fused into the passes (Eqs. psiphasor, dpsiphasor): on DFT-window steps each
// pass also forms, from the raw psi^n of its lines, the spectral normal derivative
// d psi / d a at the two virtual planes normal to its axis,
//     D_h(q) = (1/N) sum_m i k_m e^{2 pi i m (h - q)/N},   (d psi/d a)(h) = sum_q D_h(q) psi(q),
// and psi at the plane nodes; each thread contributes partial sums over the nodes it
// holds, the T threads of a line are reduced through shared memory, and one thread per
// line adds e^{i omega t_n} times the results to the double-precision accumulators.
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
        if constexpr (sizeof(R) == 4) {
            // FP32 values: the phase products in FP32 (the values carry FP32 precision), the
            // sums in FP64 -- half the FP64 instructions of the all-double form
            const float c = float(cf), sn = float(sf);
            ps0->x += double(p0.x * c - p0.y * sn);  ps0->y += double(p0.x * sn + p0.y * c);
            ps1->x += double(p1.x * c - p1.y * sn);  ps1->y += double(p1.x * sn + p1.y * c);
            dp0->x += double(d0.x * c - d0.y * sn);  dp0->y += double(d0.x * sn + d0.y * c);
            dp1->x += double(d1.x * c - d1.y * sn);  dp1->y += double(d1.x * sn + d1.y * c);
        } else {
            const double q0x = p0.x, q0y = p0.y, q1x = p1.x, q1y = p1.y;
            const double e0x = d0.x, e0y = d0.y, e1x = d1.x, e1y = d1.y;
            ps0->x += q0x * cf - q0y * sf;  ps0->y += q0x * sf + q0y * cf;
            ps1->x += q1x * cf - q1y * sf;  ps1->y += q1x * sf + q1y * cf;
            dp0->x += e0x * cf - e0y * sf;  dp0->y += e0x * sf + e0y * cf;
            dp1->x += e1x * cf - e1y * sf;  dp1->y += e1x * sf + e1y * cf;
        }
    }
}

// the accumulator entries that dft_accumulate will read-modify-write for pixel `pix` (first
// frequency), requested into L1 early so that the commit at the end of the pass finds them
template <typename R>
__device__ __forceinline__ void dft_prefetch_acc(const DftArgs<R>& a, int b, long long pix)
{
    const double2* accf = a.acc + (long long)b * a.acc_member_stride;
    const int f0 = 2 * a.axis, f1 = 2 * a.axis + 1;
    asm volatile("prefetch.global.L1 [%0];" ::"l"(accf + a.face_off[f0] + pix));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(accf + a.face_off[f0] + a.face_size[f0] + pix));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(accf + a.face_off[f1] + pix));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(accf + a.face_off[f1] + a.face_size[f1] + pix));
}

// partial sums of this thread's raw line values: [0] d/da at h0, [1] d/da at h1, [2] psi(h0), [3] psi(h1)
template <int N, int T, int R0, typename C, int E>
__device__ __forceinline__ void dft_partials(const C (&v)[E], int j, const C* __restrict__ dw, int h0, int h1, C (&part)[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) part[k] = mk<C>(decltype(C::x)(0), decltype(C::x)(0));
#if PSTD_F32X2
    if constexpr (std::is_same_v<C, float2>) {
        // sum_q v_q w_q as two packed sums, A = sum v.x (w.x, w.y) and B = sum v.y (w.x, w.y):
        // the complex sum is (A.x - B.y, A.y + B.x); each plane takes two fma.f32x2 a value
        unsigned long long A[2] = {0ull, 0ull}, B[2] = {0ull, 0ull};
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int pos = slot_pos<N, T, R0>(q, j);
            const unsigned long long vx = pk2(make_float2(v[q].x, v[q].x)), vy = pk2(make_float2(v[q].y, v[q].y));
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const unsigned long long w = pk2(__ldg(&dw[p * N + pos]));
                asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(A[p]) : "l"(vx), "l"(w));
                asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(B[p]) : "l"(vy), "l"(w));
            }
            if (pos == h0) part[2] = v[q];
            if (pos == h1) part[3] = v[q];
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float2 a = up2(A[p]), b = up2(B[p]);
            part[p] = make_float2(a.x - b.y, a.y + b.x);
        }
        return;
    }
#endif
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int pos = slot_pos<N, T, R0>(q, j);
        part[0] = cadd(part[0], cmul(v[q], __ldg(&dw[pos])));
        part[1] = cadd(part[1], cmul(v[q], __ldg(&dw[N + pos])));
        if (pos == h0) part[2] = v[q];
        if (pos == h1) part[3] = v[q];
    }
}

// Reduce the partials of the T threads of each line (lane) through `red` (>= 4 T 32 complex)
// and accumulate.  dft_stage stores this thread's partials; after a barrier, dft_commit sums
// a line's T partials and adds them to the double-precision accumulators.  A pass whose `red`
// is not reused commits at its very end, so that no thread waits on the accumulators'
// read-modify-write; dft_finish does both with barriers, for passes that reuse `red`.
template <int T, typename C>
__device__ __forceinline__ void dft_stage(const C (&part)[4], C* red, int lane, int j)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) red[(k * T + j) * kLanes + lane] = part[k];
}

template <typename R, int T, typename C>
__device__ __forceinline__ void dft_commit(const C* red, int lane, const DftArgs<R>& d, int b, long long pix)
{
    C tot[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        tot[k] = red[(k * T) * kLanes + lane];
        for (int t = 1; t < T; ++t) tot[k] = cadd(tot[k], red[(k * T + t) * kLanes + lane]);
    }
    const double2* ef = d.phase + (long long)b * d.phase_member_stride + (d.step - d.window_first[b]);
    dft_accumulate<R>(d, b, pix, ef, d.mem[b].nfreq, tot[2], tot[3], tot[0], tot[1]);
}

// The line passes' shared memory: the [pos][lane] exchange tile of N x kPitch values, and on
// DFT steps, where it fits, a region after it for the T partial sums of each line (4 values a
// thread), so that the partials are staged right after they are formed and hold no registers
// through the line transform.
template <typename R, int N> __host__ __device__ constexpr size_t pass_smem_bytes() { return sizeof(typename StepArgs<R>::C) * (size_t)N * kPitch; }
template <typename R, int N, int PL> __host__ __device__ constexpr size_t dft_red_bytes()
{
    return sizeof(typename StepArgs<R>::C) * (size_t)4 * Plan<N, PL>::T * kLanes;
}
template <typename R, int N, int PL> __host__ __device__ constexpr bool dft_red_separate()
{
    return pass_smem_bytes<R, N>() + dft_red_bytes<R, N, PL>() <= (size_t)227 * 1024;
}
template <typename R, int N, bool DFT, int PL> constexpr size_t line_pass_smem()
{
    return pass_smem_bytes<R, N>() + (DFT && dft_red_separate<R, N, PL>() ? dft_red_bytes<R, N, PL>() : 0);
}

template <typename R, int T, typename C>
__device__ __forceinline__ void dft_finish(const C (&part)[4], C* red, int lane, int j, const DftArgs<R>& d, int b,
                                           long long pix, bool act)
{
    dft_stage<T>(part, red, lane, j);
    __syncthreads();
    if (j == 0 && act) dft_commit<R, T>(red, lane, d, b, pix);
    __syncthreads();
}

// ---------------------------------------------------------------------------------
// x pass: 32 consecutive rows per CTA, staged through shared memory (rows are
// contiguous, so the tile is one contiguous block of 32 * nx values)
// ---------------------------------------------------------------------------------
// Offsets of a thread's line values in the y and z passes.  On lines of 192 points or more they
// are 32-bit and relative to the member (a member holds fewer than 2^32 cells): o holds the
// line's start plus j * st, and slot q adds slot_pos(q, 0) * st, one multiply-add a value
// (256^3 x 16 step 3.72 -> 3.67 ms).  Shorter lines keep 64-bit offsets from the batch's start,
// o excluding j: the 32-bit form made the 128-point z pass slower (17.8 against 16.7 us).
template <int N> using line_off_t = std::conditional_t<(N >= 192), unsigned, long long>;
template <int N, int T, int R0> __device__ __forceinline__ line_off_t<N> line_off(int q, int j, line_off_t<N> o, line_off_t<N> st)
{
    if constexpr (N >= 192) return o + (line_off_t<N>)slot_pos<N, T, R0>(q, 0) * st;
    else return o + (line_off_t<N>)slot_pos<N, T, R0>(q, j) * st;
}

// The x-line work of one CTA: rows [row0, row0 + kLanes) of member b (row = z * ny + y).
// On DFT steps the line partials go to slot SLOT of the region after the exchange tile;
// COMMIT = false leaves their commit to the caller (the fused x+y pass commits both axes at
// its end, off the path to its cluster barrier).
template <typename R, int N, bool DFT, int PL = 0, bool COMMIT = true, int SLOT = 0>
__device__ __forceinline__ void xpass_tile(const StepArgs<R>& a, const DftArgs<R>& d, int b, int row0,
                                           typename StepArgs<R>::C* sm)
{
    using C = typename StepArgs<R>::C;
    constexpr int T = Plan<N, PL>::T, E = N / T, R0 = Plan<N, PL>::R[0];
    const int rows = a.ny * a.nz;
    const int nrows = min(kLanes, rows - row0);
    const long long tile0 = (long long)b * a.ncell + (long long)row0 * N;
    if constexpr (N == 256 && PL == 0) {
        // the 16 threads of a line are consecutive lanes: thread j holds positions j + 16 q of
        // its row, so the row is read and updated straight from global memory (two 128-byte
        // segments a warp access) and only the transform's exchanges use shared memory, in
        // swizzled rows (tile_addr with PS = 0)
        static_assert(T == 16 && R0 == 16, "the swizzle assumes 16 threads of 16 values a line");
        const int lane = threadIdx.x / T, j = threadIdx.x % T;
        const bool act = lane < nrows;
        const C* __restrict__ row = a.cur + tile0 + (long long)lane * N;
        C* __restrict__ prow = a.prev + tile0 + (long long)lane * N;
        C v[E];
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = act ? row[slot_pos<N, T, R0>(q, j)] : zero_c<R, C>();
        if (a.pf_l1 && act) prefetch_l1(prow + 16 * j);   // the row's 16 cache lines, one a thread
        const bool dft = DFT && ((d.member_mask >> b) & 1ull);
        constexpr bool SEP = dft_red_separate<R, N, PL>();
        static_assert(SEP || (COMMIT && SLOT == 0), "a deferred commit needs the separate region");
        C* red = sm + (size_t)N * kPitch + (size_t)SLOT * 4 * T * kLanes;
        if (dft && threadIdx.x < nrows) dft_prefetch_acc<R>(d, b, row0 + threadIdx.x);
        C part[4];
        if (dft) dft_partials<N, T, R0>(v, j, d.dw, d.h[0], d.h[1], part);
        if constexpr (SEP)
            if (dft) dft_stage<T>(part, red, lane, j);   // read after the transform's barriers
        kinetic_line<N, false, 0, PL>(v, sm, lane, j, a.tw[0], a.kin[0], R(a.mem[b].eta));
        __syncthreads();
        if constexpr (!SEP)
            if (dft) dft_finish<R, T>(part, sm, lane, j, d, b, row0 + lane, act);   // plane [z][y]: pixel = row
        if (!act) return;
#pragma unroll
        for (int q0 = 0; q0 < E; q0 += 4) {
            C pg[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) pg[i] = prow[slot_pos<N, T, R0>(q0 + i, j)];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                prow[slot_pos<N, T, R0>(q0 + i, j)] = mk<C>(pg[i].x + v[q0 + i].y, pg[i].y - v[q0 + i].x);   // p - i w
        }
        // the commit: thread t < 32 (one warp) takes line t, so that the FP64 accumulation runs
        // in one warp instead of two lanes of every warp
        if constexpr (SEP && COMMIT)
            if (dft && threadIdx.x < nrows) dft_commit<R, T>(red, threadIdx.x, d, b, row0 + threadIdx.x);   // plane [z][y]: pixel = row
        return;
    }
    const int lane = threadIdx.x % kLanes, j = threadIdx.x / kLanes;
    // the tile's kLanes * N values, E a thread: every load of a thread in flight before its
    // first shared-memory store
    constexpr int NT = kLanes * T;
    {
        C t[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int e = threadIdx.x + i * NT;
            t[i] = e / N < nrows ? a.cur[tile0 + e] : zero_c<R, C>();
        }
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int e = threadIdx.x + i * NT, r = e / N;
            sm[(e - r * N) * kPitch + r] = t[i];
        }
    }
    if constexpr (N >= 192) {   // the tile's update operand, one 128-byte line a thread (see prefetch_l1)
        if (a.pf_l1) {
            constexpr int per = 128 / (int)sizeof(C);
            for (int e = threadIdx.x * per; e < nrows * N; e += blockDim.x * per) prefetch_l1(a.prev + tile0 + e);
        }
    }
    __syncthreads();
    C v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = sm[slot_pos<N, T, R0>(q, j) * kPitch + lane];
    __syncthreads();
    const bool dft = DFT && ((d.member_mask >> b) & 1ull);
    constexpr bool SEP = dft_red_separate<R, N, PL>();
    static_assert(SEP || (COMMIT && SLOT == 0), "a deferred commit needs the separate region");
    C* red = sm + (size_t)N * kPitch + (size_t)SLOT * 4 * T * kLanes;
    if (dft && j == 0 && lane < nrows) dft_prefetch_acc<R>(d, b, row0 + lane);
    C part[4];
    if (dft) dft_partials<N, T, R0>(v, j, d.dw, d.h[0], d.h[1], part);
    if constexpr (SEP)
        if (dft) dft_stage<T>(part, red, lane, j);   // read after the transform's barriers
    const R eta = R(a.mem[b].eta);
    kinetic_line<N, false, kPitch, PL>(v, sm, lane, j, a.tw[0], a.kin[0], eta);
    __syncthreads();
    if constexpr (!SEP)
        if (dft) dft_finish<R, T>(part, sm, lane, j, d, b, row0 + lane, lane < nrows);   // plane [z][y]: pixel = row
#pragma unroll
    for (int q = 0; q < E; ++q) sm[slot_pos<N, T, R0>(q, j) * kPitch + lane] = v[q];
    __syncthreads();
    {
        C p[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int e = threadIdx.x + i * NT;
            if (e / N < nrows) p[i] = a.prev[tile0 + e];
        }
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int e = threadIdx.x + i * NT, r = e / N;
            if (r < nrows) {
                const C w = sm[(e - r * N) * kPitch + r];
                a.prev[tile0 + e] = mk<C>(p[i].x + w.y, p[i].y - w.x);   // p - i w
            }
        }
    }
    if constexpr (SEP && COMMIT)
        if (dft && j == 0 && lane < nrows) dft_commit<R, T>(red, lane, d, b, row0 + lane);   // plane [z][y]: pixel = row
}

template <typename R, int N, bool DFT, int PL = 0>
__global__ void __launch_bounds__(kLanes * Plan<N, PL>::T, (pass_min_blocks<R, N, PL>())) xpass_kernel(const __grid_constant__ StepArgs<R> a, const __grid_constant__ DftArgs<R> d)
{
    step_kernel_entry();
    extern __shared__ __align__(16) unsigned char smraw[];
    xpass_tile<R, N, DFT, PL>(a, d, blockIdx.y, blockIdx.x * kLanes, reinterpret_cast<typename StepArgs<R>::C*>(smraw));
}

// ---------------------------------------------------------------------------------
// y pass: lines along y, 32 consecutive x per CTA (lane = x), coalesced in place
// ---------------------------------------------------------------------------------
// load of the y pass's read-modify-write operand: CG = true reads it at L2 (the fused
// cluster pass, whose other CTAs have just written it), bypassing L1
template <bool CG, typename C> __device__ __forceinline__ C load_prev(const C* p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// The y-line work of one CTA: columns [x0, x0 + kLanes) of z plane z, member b (DFT partials
// in slot SLOT of the region after the exchange tile).
template <typename R, int N, bool DFT, bool CG = false, int PL = 0, int SLOT = 0>
__device__ __forceinline__ void ypass_tile(const StepArgs<R>& a, const DftArgs<R>& d, int x0, int z, int b,
                                           typename StepArgs<R>::C* sm)
{
    using C = typename StepArgs<R>::C;
    constexpr int T = Plan<N, PL>::T, E = N / T, R0 = Plan<N, PL>::R[0];
    const int lane = threadIdx.x % kLanes, j = threadIdx.x / kLanes;
    const int x = x0 + lane;
    const bool act = x < a.nx;
    using Off = line_off_t<N>;
    constexpr bool W32 = N >= 192;
    const long long mbase = (long long)b * a.ncell;
    const C* curm = a.cur + (W32 ? mbase : 0);
    C* prevm = a.prev + (W32 ? mbase : 0);
    const Off st = (Off)a.nx;
    const Off o0 = (Off)z * (Off)a.nx * (Off)a.ny + (Off)x + (W32 ? (Off)j * st : (Off)mbase);
    C v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = act ? curm[line_off<N, T, R0>(q, j, o0, st)] : zero_c<R, C>();
#if !PSTD_PREFETCH_PREV
    if constexpr (N >= 192 && !CG) {
        if (a.pf_l1 && act) {
#pragma unroll
            for (int q = 0; q < E; ++q) prefetch_l1(prevm + line_off<N, T, R0>(q, j, o0, st));
        }
    }
#endif
#if PSTD_PREFETCH_PREV
    C pv[E];
#pragma unroll
    for (int q = 0; q < E; ++q) pv[q] = act ? load_prev<CG>(prevm + line_off<N, T, R0>(q, j, o0, st)) : zero_c<R, C>();
#endif
    const bool dft = DFT && ((d.member_mask >> b) & 1ull);
    constexpr bool SEP = dft_red_separate<R, N, PL>();
    static_assert(SEP || SLOT == 0, "slot 1 needs the separate region");
    C* red = SEP ? sm + (size_t)N * kPitch + (size_t)SLOT * 4 * T * kLanes : sm;
    if (dft && j == 0 && act) dft_prefetch_acc<R>(d, b, (long long)z * a.nx + x);
    C part[4];
    if (dft) dft_partials<N, T, R0>(v, j, d.dw, d.h[0], d.h[1], part);
    if constexpr (SEP)
        if (dft) dft_stage<T>(part, red, lane, j);   // read after the transform's barriers
    const R eta = R(a.mem[b].eta);
    kinetic_line<N, false, kPitch, PL>(v, sm, lane, j, a.tw[1], a.kin[1], eta);
    if constexpr (!SEP) {
        if (dft) {
            __syncthreads();   // the exchange tile is free again
            dft_stage<T>(part, sm, lane, j);
            __syncthreads();
        }
    }
    if (!act) return;
    constexpr int GR = N >= 192 ? 4 : 1;   // update operands read GR at a time (see the z pass)
#pragma unroll
    for (int q0 = 0; q0 < E; q0 += GR) {
#if !PSTD_PREFETCH_PREV
        C pg[GR];
#pragma unroll
        for (int i = 0; i < GR; ++i) pg[i] = load_prev<CG>(prevm + line_off<N, T, R0>(q0 + i, j, o0, st));
#endif
#pragma unroll
        for (int q = q0; q < q0 + GR; ++q) {
            const Off off = line_off<N, T, R0>(q, j, o0, st);
#if PSTD_PREFETCH_PREV
            const C p = pv[q];
#else
            const C p = pg[q - q0];
#endif
            prevm[off] = mk<C>(p.x + v[q].y, p.y - v[q].x);
        }
    }
    if (dft && j == 0) dft_commit<R, T>(red, lane, d, b, (long long)z * a.nx + x);   // plane [z][x]
}

template <typename R, int N, bool DFT, int PL = 0>
__global__ void __launch_bounds__(kLanes * Plan<N, PL>::T, (pass_min_blocks<R, N, PL>())) ypass_kernel(const __grid_constant__ StepArgs<R> a, const __grid_constant__ DftArgs<R> d)
{
    step_kernel_entry();
    extern __shared__ __align__(16) unsigned char smraw[];
    ypass_tile<R, N, DFT, false, PL>(a, d, blockIdx.x * kLanes, blockIdx.y, blockIdx.z,
                                     reinterpret_cast<typename StepArgs<R>::C*>(smraw));
}

// ---------------------------------------------------------------------------------
// fused x + y pass for large square planes (FP32, N = 192 or 256): a thread-block
// cluster of N / 32 CTAs per (z plane, member).  CTA r of the cluster first applies K_x
// to rows [32 r, 32 r + 32) of the plane and read-modify-writes them (the x pass's
// work), then, after a cluster barrier with release/acquire semantics (which orders the
// other CTAs' stores of the plane before this CTA's loads), applies K_y to columns
// [32 r, 32 r + 32) and read-modify-writes those (the y pass's work).  The plane's two
// levels (2 x 512 KB at N = 256) were touched by the cluster a few microseconds before,
// so the column phase reads psi^n and the partial level from L2: DRAM sees one read of
// psi^n and one read-modify-write of the partial per cell for both axes -- 24 B a cell
// instead of the 48 B of separate x and y passes.  The cluster is what bounds the set of
// planes in flight (and so the L2 footprint) while keeping every SM busy.
// ---------------------------------------------------------------------------------
template <typename R, int N> constexpr bool xycl_supported()
{
    return sizeof(R) == 4 && (N == 128 || N == 192 || N == 256) && N % kLanes == 0 && N / kLanes <= 8;
}

__device__ __forceinline__ void cluster_sync_acq_rel()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <typename R, int N, bool DFT, int PL = 0>
__global__ void __launch_bounds__(kLanes * Plan<N, PL>::T, (pass_min_blocks<R, N, PL>())) xycl_kernel(const __grid_constant__ StepArgs<R> a,
                                                                                                   const __grid_constant__ DftArgs<R> dx,
                                                                                                   const __grid_constant__ DftArgs<R> dy)
{
    step_kernel_entry();
    extern __shared__ __align__(16) unsigned char smraw[];
    using C = typename StepArgs<R>::C;
    C* sm = reinterpret_cast<C*>(smraw);
    const int r = blockIdx.x;                  // rank in the cluster (the grid's x extent is the cluster)
    const int z = blockIdx.y, b = blockIdx.z;
    const int row0 = z * N + r * kLanes;
    // on DFT steps the row phase's partials wait in slot 0 and are committed after the
    // column phase, whose own partials use slot 1
    xpass_tile<R, N, DFT, PL, false, 0>(a, dx, b, row0, sm);
    cluster_sync_acq_rel();
    ypass_tile<R, N, DFT, true, PL, 1>(a, dy, r * kLanes, z, b, sm);
    if constexpr (DFT) {
        // one warp commits the row phase's sums, thread t line t (the partials are stored by
        // line, whatever the phase's thread-to-line map)
        if (((dx.member_mask >> b) & 1ull) && threadIdx.x < kLanes)
            dft_commit<R, Plan<N, PL>::T>(sm + (size_t)N * kPitch, threadIdx.x, dx, b, row0 + threadIdx.x);   // plane [z][y]
    }
}

// ---------------------------------------------------------------------------------
// xy pass: one CTA per z plane (square N x N planes in FP32), applying K_x + K_y as one
// 2-D spectral operator, F_y^-1 F_x^-1 [(k_x^2 + k_y^2) F_x F_y psi], with the plane held
// in shared memory ([y][x], pitch N + 1: conflict-free for rows and for columns):
//   1. columns (lane = x, read from global, coalesced): forward FFT along y, spectrum
//      written to the plane;
//   2. rows (lane = y spectral index): forward FFT along x, multiply by
//      eta (kin_x[m_x] + kin_y[m_y]) / N (each kin table carries its own axis' 1/N),
//      inverse FFT along x, written back;
//   3. columns: inverse FFT along y, then prev -= i * result straight to global.
// One read of psi^n and one read-modify-write of the partial per cell, instead of two
// of each for separate x and y passes.
// ---------------------------------------------------------------------------------
template <int N> __host__ __device__ constexpr int xy_threads() { return (N / 32) * Plan<N>::T * 32; }
template <typename R, int N> constexpr bool xy_supported()
{
    return sizeof(R) == 4 && Plan<N>::S == 2 && N % 32 == 0 && xy_threads<N>() <= 1024 &&
           (size_t)N * (N + 1) * 8 <= 227 * 1024;
}

// On DFT-window steps (DFT = true) the pass also forms the running DFT of the planes normal
// to x and to y: for the x planes each warp reads whole rows of the z plane (coalesced) and
// reduces D_h(x) psi(x, y) over x with shuffles; for the y planes the raw column values of
// step 1 give the partial sums, reduced over the T threads of a column in shared memory
// placed after the plane.
template <int N> constexpr size_t xy_dft_red_elems() { return (size_t)4 * Plan<N>::T * N + (size_t)4 * N; }

template <typename R, typename C> __device__ __forceinline__ C warp_sum(C v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

template <typename R, int N, bool DFT>
__global__ void __launch_bounds__(xy_threads<N>(), 1) xypass_kernel(const __grid_constant__ StepArgs<R> a,
                                                                      const __grid_constant__ DftArgs<R> dx,
                                                                      const __grid_constant__ DftArgs<R> dy)
{
    step_kernel_entry();
    using C = typename StepArgs<R>::C;
    // the plane's values and FFTs: FP32 ones as cs32, whose butterflies stay scalar (packed
    // ones schedule worse in this 1024-thread kernel)
    using V = std::conditional_t<sizeof(R) == 4, cs32, C>;
    constexpr int T = Plan<N>::T, E = N / T, R0 = Plan<N>::R[0], R1 = Plan<N>::R[1], P = N + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    const int lane = threadIdx.x & 31, j = (threadIdx.x >> 5) % T, grp = threadIdx.x / (32 * T);
    const int z = blockIdx.x, b = blockIdx.y;
    const int x = grp * 32 + lane;             // column of this thread in steps 1 and 3
    const int my = grp * 32 + lane;            // row (spectral y index) in step 2
    V* smc = sm + grp * 32;                    // columns: (pos, lane) at pos * P + lane
    V* smr = sm + grp * 32 * P;                // rows:    (pos, lane) at lane * P + pos
    const long long pbase = (long long)b * a.ncell + (long long)z * N * N;
    const V* __restrict__ cur = reinterpret_cast<const V*>(a.cur + pbase + x);
    C* __restrict__ prev = a.prev + pbase + x;
    const V* __restrict__ twx = reinterpret_cast<const V*>(a.tw[0]);
    const V* __restrict__ twy = reinterpret_cast<const V*>(a.tw[1]);
    V v[E];
    const bool dft = DFT && ((dx.member_mask >> b) & 1ull);
    // DFT scratch after the plane: y-plane partials [group][4][T][32], then x-plane sums [N][4]
    C* red_y = reinterpret_cast<C*>(sm + (size_t)N * P);
    C* sum_x = red_y + (size_t)4 * T * N;
    if (dft && threadIdx.x < N) {
        dft_prefetch_acc<R>(dx, b, (long long)z * N + threadIdx.x);   // plane [z][y]
        dft_prefetch_acc<R>(dy, b, (long long)z * N + threadIdx.x);   // plane [z][x]
    }
    if (dft) {
        // x planes: row y of this z plane, lanes over x (the warp count is the launch's, known
        // at compile time, so a warp's rows are unrolled and their loads overlap)
        constexpr int nwarps = xy_threads<N>() / 32;
        static_assert(N % nwarps == 0, "rows per warp");
        const int warp = threadIdx.x >> 5;
#pragma unroll
        for (int y = warp; y < N; y += nwarps) {
            const C* row = a.cur + pbase + (long long)y * N;
            C d0 = zero_c<R, C>(), d1 = zero_c<R, C>(), p0 = zero_c<R, C>(), p1 = zero_c<R, C>();
#pragma unroll
            for (int k = 0; k < N / 32; ++k) {
                const int xx = lane + 32 * k;
                const C u = row[xx];
                d0 = cadd(d0, cmul(u, dx.dw[xx]));
                d1 = cadd(d1, cmul(u, dx.dw[N + xx]));
                if (xx == dx.h[0]) p0 = u;
                if (xx == dx.h[1]) p1 = u;
            }
            d0 = warp_sum<R, C>(d0);
            d1 = warp_sum<R, C>(d1);
            p0 = warp_sum<R, C>(p0);
            p1 = warp_sum<R, C>(p1);
            if (lane == 0) {
                sum_x[4 * y + 0] = d0;
                sum_x[4 * y + 1] = d1;
                sum_x[4 * y + 2] = p0;
                sum_x[4 * y + 3] = p1;
            }
        }
    }
    // 1. forward along y
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = cur[slot_pos<N, T, R0>(q, j) * N];
    if (dft) {
        // y planes from the raw column values (the barriers of the FFT stages below order
        // these stores before the commit at the end)
        C part[4], vc[E];
#pragma unroll
        for (int q = 0; q < E; ++q) vc[q] = mk<C>(v[q].x, v[q].y);
        dft_partials<N, T, R0>(vc, j, dy.dw, dy.h[0], dy.h[1], part);
        dft_stage<T>(part, red_y + (size_t)grp * 4 * T * 32, lane, j);
    }
    stockham_stage<N, T, R0, 1, -1, false, true, P, 1>(v, smc, lane, j, twy);
    stockham_stage<N, T, R1, R0, -1, true, false, P, 1>(v, smc, lane, j, twy);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < E; ++q) smc[spec_pos<N, T, R1>(q, j) * P + lane] = v[q];
    __syncthreads();
    // 2. along x: forward, spectral multiply, inverse
    stockham_stage<N, T, R0, 1, -1, true, true, 1, P>(v, smr, lane, j, twx);
    stockham_stage<N, T, R1, R0, -1, true, false, 1, P>(v, smr, lane, j, twx);
    {
        const R eta = R(a.mem[b].eta) * (R(1) / R(N));
        const R ky = __ldg(&a.kin[1][my]);
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = cscale(v[q], (__ldg(&a.kin[0][spec_pos<N, T, R1>(q, j)]) + ky) * eta);
    }
    __syncthreads();
    stockham_stage<N, T, R1, 1, +1, false, true, 1, P>(v, smr, lane, j, twx);
    stockham_stage<N, T, R0, R1, +1, true, false, 1, P>(v, smr, lane, j, twx);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < E; ++q) smr[lane * P + slot_pos<N, T, R0>(q, j)] = v[q];
    __syncthreads();
    // 3. inverse along y, then the update
    stockham_stage<N, T, R1, 1, +1, true, true, P, 1>(v, smc, lane, j, twy);
    stockham_stage<N, T, R0, R1, +1, true, false, P, 1>(v, smc, lane, j, twy);
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int off = slot_pos<N, T, R0>(q, j) * N;
        const C p = prev[off];
        prev[off] = mk<C>(p.x + v[q].y, p.y - v[q].x);
    }
    if (dft && threadIdx.x < N) {
        // commit: thread t adds row t's x-plane sums and column t's y-plane sums
        const int t = threadIdx.x;
        const double2* efx = dx.phase + (long long)b * dx.phase_member_stride + (dx.step - dx.window_first[b]);
        dft_accumulate<R>(dx, b, (long long)z * N + t, efx, dx.mem[b].nfreq, sum_x[4 * t + 2], sum_x[4 * t + 3],
                          sum_x[4 * t + 0], sum_x[4 * t + 1]);                       // plane [z][y]
        dft_commit<R, T>(red_y + (size_t)(t / 32) * 4 * T * 32, t % 32, dy, b, (long long)z * N + t);   // plane [z][x]
    }
}

// ---------------------------------------------------------------------------------
// V-term and TF/SF source over their support box [lo, hi) (x fastest), one cell per thread:
//   EXACT: prev -= (2 i dt / hbar) V (psi^n + psi_inc^n)
//   PAPER: prev -= (2 i dt / hbar) [V psi~^n + hbar^2/2m psi_inc^n (lap zeta + 2 i k . grad zeta)]
// ---------------------------------------------------------------------------------
constexpr int kSourceZ = 4;   // z planes per thread of the source kernel

// Gaussian envelope of a wave-packet member at node (x, y, z):
// exp(-alpha_n (d - c_n)^2) with d = khat . (r - r_O) from the per-axis projection tables
template <typename R, typename C>
__device__ __forceinline__ C packet_envelope(const StepArgs<R>& a, int b, int x, int y, int z)
{
    const R* e = a.tenv + 3 * ((a.step - a.tfac_base) * a.batch + b);
    const R d = a.proj[0][b * a.nx + x] + a.proj[1][b * a.ny + y] + a.proj[2][b * a.nz + z];
    const R u = d - e[2];
    const R u2 = u * u;
    R sn, cs, mag;
    if constexpr (sizeof(R) == 4) {
        sincosf(-e[1] * u2, &sn, &cs);
        mag = expf(-e[0] * u2);
    } else {
        sincos(-e[1] * u2, &sn, &cs);
        mag = exp(-e[0] * u2);
    }
    return mk<C>(mag * cs, mag * sn);
}

// the incident wave of member b at node (x, y, z), step a.step; s = the member's time factor
// index of (x, y, z) in the auxiliary-wave buffers of member b (an aux member, node in the box)
template <typename R>
__device__ __forceinline__ long long aux_index(const StepArgs<R>& a, int b, int x, int y, int z)
{
    const int slot = __popcll(a.aux_mask & ((1ull << b) - 1ull));
    const long long nb = (long long)a.abox_n[0] * a.abox_n[1] * a.abox_n[2];
    return slot * nb + ((long long)(z - a.abox_lo[2]) * a.abox_n[1] + (y - a.abox_lo[1])) * a.abox_n[0] + (x - a.abox_lo[0]);
}

// psi_inc of an aux member: the step's evaluated value
template <typename R, typename C>
__device__ __forceinline__ C aux_wave(const StepArgs<R>& a, int b, C s, int x, int y, int z)
{
    return cmul(s, a.aux_inc[aux_index(a, b, x, y, z)]);
}

// the PAPER form's taper source of an aux member
template <typename R, typename C>
__device__ __forceinline__ C aux_taper_source(const StepArgs<R>& a, int b, int x, int y, int z, R lap, R zx, R zy, R zz, R zx1,
                                           R zy1, R zz1)
{
    const MemberDev& md = a.mem[b];
    // hbar^2/2m [lap(zeta) psi_inc + 2 (khat . grad zeta) d psi_inc / d d] (Eq. pstd_dpsiinc)
    const R kg = R(md.khat[0]) * zx1 * zy * zz + R(md.khat[1]) * zx * zy1 * zz + R(md.khat[2]) * zx * zy * zz1;
    const long long e = aux_index(a, b, x, y, z);
    return cscale(cadd(cscale(a.aux_inc[e], lap), cscale(a.aux_dinc[e], R(2) * kg)), a.h2m);
}

template <typename R, typename C>
__device__ __forceinline__ C incident_wave(const StepArgs<R>& a, int b, C s, int x, int y, int z)
{
    if ((a.aux_mask >> b) & 1ull) return aux_wave<R, C>(a, b, s, x, y, z);
    C w = incident_at<R, C>(a, b, s, x, y, z);
    if ((a.packet_mask >> b) & 1ull) w = cmul(w, packet_envelope<R, C>(a, b, x, y, z));
    return w;
}

// spinor member b: W (u + psi_inc) of its component, with W = V I + gamma sigma . B,
// sigma . B = [[Bz, Bx - i By], [Bx + i By, -Bz]] (EXACT form); the partner component b ^ 1
// is read at the same node
template <typename R, typename C>
__device__ __forceinline__ C spinor_acc(const StepArgs<R>& a, int b, C s, int x, int y, int z, long long idx)
{
    const int bo = b ^ 1;
    const long long idx_o = idx + (b & 1 ? -a.ncell : a.ncell);
    const C so = a.tfac[(a.step - a.tfac_base) * a.batch + bo];
    const C ts = cadd(a.cur[idx], incident_wave<R, C>(a, b, s, x, y, z));
    const C to = cadd(a.cur[idx_o], incident_wave<R, C>(a, bo, so, x, y, z));
    R Vv = R(0), Bx = R(0), By = R(0), Bz = R(0);
    if (x >= a.vlo[0] && x < a.vhi[0] && y >= a.vlo[1] && y < a.vhi[1] && z >= a.vlo[2] && z < a.vhi[2]) {
        const int vnx = a.vhi[0] - a.vlo[0], vny = a.vhi[1] - a.vlo[1];
        Vv = a.V[((long long)(z - a.vlo[2]) * vny + (y - a.vlo[1])) * vnx + (x - a.vlo[0])];
    }
    if (x >= a.blo[0] && x < a.bhi[0] && y >= a.blo[1] && y < a.bhi[1] && z >= a.blo[2] && z < a.bhi[2]) {
        const int bnx = a.bhi[0] - a.blo[0], bny = a.bhi[1] - a.blo[1];
        const long long e = ((long long)(z - a.blo[2]) * bny + (y - a.blo[1])) * bnx + (x - a.blo[0]);
        Bx = a.gamma * a.B[0][e];
        By = a.gamma * a.B[1][e];
        Bz = a.gamma * a.B[2][e];
    }
    const bool up = (b & 1) == 0;
    const R wss = Vv + (up ? Bz : -Bz);
    const C wso = mk<C>(Bx, up ? -By : By);   // up: gamma (Bx - i By); down: gamma (Bx + i By)
    return cadd(cscale(ts, wss), cmul(wso, to));
}

// V-term + source at node (x, y, z) of member b (before the factor -(2 i dt / hbar));
// s = the member's incident time factor at step n, idx the node's state index.  KIND 1: a
// scalar CW member (the common case, inlined into the pass epilogues); 3: a CW or wave-packet
// member; 4: a CW or 1-D auxiliary-wave member (both also inlined); 2: any member (spinor
// pairs as well), reached through source_general.
template <typename R, typename C, int KIND>
__device__ __forceinline__ C source_impl(const StepArgs<R>& a, int b, C s, int x, int y, int z, long long idx)
{
    if constexpr (KIND == 2) {
        if (a.spinor) return spinor_acc<R, C>(a, b, s, x, y, z, idx);
    }
    const bool paper = a.mode == PSTD_TFSF_PAPER;
    C acc = mk<C>(R(0), R(0));
    if (x >= a.vlo[0] && x < a.vhi[0] && y >= a.vlo[1] && y < a.vhi[1] && z >= a.vlo[2] && z < a.vhi[2]) {
        const int vnx = a.vhi[0] - a.vlo[0], vny = a.vhi[1] - a.vlo[1];
        const R Vv = a.V[((long long)(z - a.vlo[2]) * vny + (y - a.vlo[1])) * vnx + (x - a.vlo[0])];
        C src = a.cur[idx];
        if (!paper) {
            C w;
            if constexpr (KIND == 1) {
                w = incident_at<R, C>(a, b, s, x, y, z);
            } else if constexpr (KIND == 3) {
                w = incident_at<R, C>(a, b, s, x, y, z);
                if ((a.packet_mask >> b) & 1ull) w = cmul(w, packet_envelope<R, C>(a, b, x, y, z));
            } else if constexpr (KIND == 4) {
                w = ((a.aux_mask >> b) & 1ull) ? aux_wave<R, C>(a, b, s, x, y, z) : incident_at<R, C>(a, b, s, x, y, z);
            } else {
                w = incident_wave<R, C>(a, b, s, x, y, z);
            }
            src = cadd(src, w);
        }
        acc = cscale(src, Vv);
    }
    if (paper && x > a.tf_lo[0] && x < a.tf_hi[0] && y > a.tf_lo[1] && y < a.tf_hi[1] && z > a.tf_lo[2] && z < a.tf_hi[2]) {
        const R zx = a.zeta[0][x], zx1 = a.zeta1[0][x], zx2 = a.zeta2[0][x];
        const R zy = a.zeta[1][y], zy1 = a.zeta1[1][y], zy2 = a.zeta2[1][y];
        const R zz = a.zeta[2][z], zz1 = a.zeta1[2][z], zz2 = a.zeta2[2][z];
        const R lap = zx2 * zy * zz + zx * zy2 * zz + zx * zy * zz2;
        if ((KIND == 2 || KIND == 4) && ((a.aux_mask >> b) & 1ull)) {
            acc = cadd(acc, aux_taper_source<R, C>(a, b, x, y, z, lap, zx, zy, zz, zx1, zy1, zz1));
        } else {
            const MemberDev& md = a.mem[b];
            const R kg = R(md.k[0]) * zx1 * zy * zz + R(md.k[1]) * zx * zy1 * zz + R(md.k[2]) * zx * zy * zz1;
            acc = cadd(acc, cscale(cmul(incident_at<R, C>(a, b, s, x, y, z), mk<C>(lap, R(2) * kg)), a.h2m));   // CW
        }
    }
    return acc;
}

template <typename R, typename C>
__device__ __noinline__ C source_general(const StepArgs<R>& a, int b, C s, int x, int y, int z, long long idx)
{
    return source_impl<R, C, 2>(a, b, s, x, y, z, idx);
}

// KIND (chosen per grid on the host): 1 scalar CW members only; 3 CW and wave-packet members;
// 4 CW and auxiliary-wave members; 2 any members, with the uncommon paths out of line
template <typename R, typename C, int KIND = 2>
__device__ __forceinline__ C source_acc(const StepArgs<R>& a, int b, C s, int x, int y, int z, long long idx)
{
    if constexpr (KIND != 2) {
        return source_impl<R, C, KIND>(a, b, s, x, y, z, idx);
    } else {
        const bool plain = !a.spinor && !(((a.aux_mask | a.packet_mask) >> b) & 1ull);
        return plain ? source_impl<R, C, 1>(a, b, s, x, y, z, idx) : source_general<R, C>(a, b, s, x, y, z, idx);
    }
}

// the box [lo, hi) on which the V-term or the source can be non-zero: the V box, or for the
// PAPER form the interior of the TF/SF box (which contains it)
template <typename R> __host__ __device__ inline void source_box(const StepArgs<R>& a, int lo[3], int hi[3])
{
    for (int d = 0; d < 3; ++d) {
        if (a.mode == PSTD_TFSF_PAPER) { lo[d] = a.tf_lo[d] + 1; hi[d] = a.tf_hi[d]; }
        else { lo[d] = a.vlo[d]; hi[d] = a.vhi[d]; }
    }
    // spinor grids: the union with B's box (an empty box has lo == hi)
    if (a.spinor && a.bhi[0] > a.blo[0]) {
        const bool vempty = !(a.vhi[0] > a.vlo[0]);
        for (int d = 0; d < 3; ++d) {
            lo[d] = vempty ? a.blo[d] : (a.blo[d] < lo[d] ? a.blo[d] : lo[d]);
            hi[d] = vempty ? a.bhi[d] : (a.bhi[d] > hi[d] ? a.bhi[d] : hi[d]);
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(128) source_kernel(const __grid_constant__ StepArgs<R> a, int lox, int loy, int loz, int bx, int by, int bz)
{
    step_kernel_entry();
    using C = typename StepArgs<R>::C;
    // block: 32 x 4 (x, y) columns, each thread kSourceZ consecutive z; grid: (x tiles, y tiles, z chunks * batch)
    const int x = lox + blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = loy + blockIdx.y * 4 + (threadIdx.x >> 5);
    const int zchunks = (bz + kSourceZ - 1) / kSourceZ;
    const int b = blockIdx.z / zchunks, z0 = loz + (blockIdx.z % zchunks) * kSourceZ;
    if (x >= lox + bx || y >= loy + by) return;
    const C s = a.tfac[(a.step - a.tfac_base) * a.batch + b];   // a(t_n) e^{-i w0 t_n}
    const R c2 = a.c2;
#pragma unroll
    for (int zz = 0; zz < kSourceZ; ++zz) {
        const int z = z0 + zz;
        if (z >= loz + bz) break;
        const long long idx = (long long)b * a.ncell + ((long long)z * a.ny + y) * a.nx + x;
        const C acc = source_acc<R, C>(a, b, s, x, y, z, idx);
        const C p = a.prev[idx];
        a.prev[idx] = mk<C>(p.x + c2 * acc.y, p.y - c2 * acc.x);
    }
}

// ---------------------------------------------------------------------------------
// z pass: lines along z, lane = x; completes psi^{n+1} with the mask
// ---------------------------------------------------------------------------------
// SRC: 0 no V-term or source; otherwise the source form (source_acc's KIND: 1 scalar CW
// members only, 3 CW and wave packets, 4 CW and the auxiliary wave, 2 any members)
// The z-line work of one CTA: columns [x0, x0 + kLanes) of row y, member b.
template <typename R, int N, bool DFT, int SRC, int PL = 0>
__device__ __forceinline__ void ztile(const StepArgs<R>& a, const DftArgs<R>& d, int x0, int y, int b,
                                      typename StepArgs<R>::C* sm)
{
    using C = typename StepArgs<R>::C;
    constexpr int T = Plan<N, PL>::T, E = N / T, R0 = Plan<N, PL>::R[0];
    const int lane = threadIdx.x % kLanes, j = threadIdx.x / kLanes;
    const int x = x0 + lane;
    const bool act = x < a.nx;
    using Off = line_off_t<N>;
    constexpr bool W32 = N >= 192;
    const long long mbase = (long long)b * a.ncell;
    const C* curm = a.cur + (W32 ? mbase : 0);
    C* prevm = a.prev + (W32 ? mbase : 0);
    const Off st = (Off)a.nx * (Off)a.ny;
    const Off o0 = (Off)y * (Off)a.nx + (Off)x + (W32 ? (Off)j * st : (Off)mbase);
    C v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = act ? curm[line_off<N, T, R0>(q, j, o0, st)] : zero_c<R, C>();
#if PSTD_PREFETCH_PREV
    C pv[E];
#pragma unroll
    for (int q = 0; q < E; ++q) pv[q] = act ? prevm[line_off<N, T, R0>(q, j, o0, st)] : zero_c<R, C>();
#endif
    const bool dft = DFT && ((d.member_mask >> b) & 1ull);
    if (dft && j == 0 && act) dft_prefetch_acc<R>(d, b, (long long)y * a.nx + x);   // plane [y][x]
#if !PSTD_PREFETCH_PREV
    if constexpr (N >= 192) {   // compiled in for long lines only: its mere presence slows the 128-point pass
        if (a.pf_l1 && act) {
#pragma unroll
            for (int q = 0; q < E; ++q) prefetch_l1(prevm + line_off<N, T, R0>(q, j, o0, st));
        }
    }
#endif
    constexpr bool SEP = dft_red_separate<R, N, PL>();
    C* red = SEP ? sm + (size_t)N * kPitch : sm;
    C part[4];
    if (dft) dft_partials<N, T, R0>(v, j, d.dw, d.h[0], d.h[1], part);
    if constexpr (SEP)
        if (dft) dft_stage<T>(part, red, lane, j);   // read after the transform's barriers
    kinetic_line<N, false, kPitch, PL>(v, sm, lane, j, a.tw[2], a.kin[2], R(a.mem[b].eta));
    if constexpr (!SEP) {
        if (dft) {
            __syncthreads();   // the exchange tile is free again
            dft_stage<T>(part, sm, lane, j);
            __syncthreads();
        }
    }
    if (!act) return;
    const R gxy = a.mask[0][x] * a.mask[1][y];
    bool ok = true;
    // with SRC the V-term and source of this column are added here instead of by source_kernel
    int slo[3] = {0, 0, 0}, shi[3] = {0, 0, 0};
    if constexpr (SRC) source_box<R>(a, slo, shi);
    const bool src_col = SRC != 0 && x >= slo[0] && x < shi[0] && y >= slo[1] && y < shi[1];
    const C s = src_col ? a.tfac[(a.step - a.tfac_base) * a.batch + b] : zero_c<R, C>();
    // on long lines the update operand is read four values at a time, so that its loads do
    // not wait on the stores before them (at 128 points the extra registers cost more)
    constexpr int GR = N >= 192 ? 4 : 1;
    static_assert(E % GR == 0, "E");
    // the update loop; on lines of 192 points or more it is compiled twice, so that the columns
    // that miss the source box (nearly all) carry no per-value test (256^3 x 16 z pass 1.29 ->
    // 1.23 ms); at 128 points the doubled code made the pass slower (20.6 against 16.9 us)
    auto update = [&](auto with_src) {
        constexpr bool WS = decltype(with_src)::value;
#pragma unroll
        for (int q0 = 0; q0 < E; q0 += GR) {
#if !PSTD_PREFETCH_PREV
            C pg[GR];
#pragma unroll
            for (int i = 0; i < GR; ++i) pg[i] = prevm[line_off<N, T, R0>(q0 + i, j, o0, st)];
#endif
#pragma unroll
            for (int q = q0; q < q0 + GR; ++q) {
                const int z = slot_pos<N, T, R0>(q, j);
                const Off off = line_off<N, T, R0>(q, j, o0, st);
#if PSTD_PREFETCH_PREV
                C p = pv[q];
#else
                C p = pg[q - q0];
#endif
                if constexpr (SRC != 0 && WS) {
                    if (z >= slo[2] && z < shi[2]) {
                        const C sa = source_acc<R, C, SRC>(a, b, s, x, y, z, (W32 ? mbase : 0) + (long long)off);
                        p = mk<C>(p.x + a.c2 * sa.y, p.y - a.c2 * sa.x);
                    }
                }
                const R g = gxy * a.mask[2][z];
                const C acc = mk<C>(g * (p.x + v[q].y), g * (p.y - v[q].x));
                ok = ok && finite_c<R>(acc.x, acc.y);
                prevm[off] = acc;
            }
        }
    };
    if constexpr (N >= 192) {
        if (src_col) update(std::true_type{});
        else update(std::false_type{});
    } else {
        update(std::true_type{});
    }
    if (!ok) atomicOr(a.flag, 1);
    if (dft && j == 0) dft_commit<R, T>(red, lane, d, b, (long long)y * a.nx + x);   // plane [y][x]
}

template <typename R, int N, bool DFT, int SRC, int PL = 0>
__global__ void __launch_bounds__(kLanes * Plan<N, PL>::T, (pass_min_blocks<R, N, PL>())) zpass_kernel(const __grid_constant__ StepArgs<R> a, const __grid_constant__ DftArgs<R> d)
{
    step_kernel_entry();
    extern __shared__ __align__(16) unsigned char smraw[];
    ztile<R, N, DFT, SRC, PL>(a, d, blockIdx.x * kLanes, blockIdx.y, blockIdx.z, reinterpret_cast<typename StepArgs<R>::C*>(smraw));
}

// ---------------------------------------------------------------------------------
// pipelined y and z passes for large planes (FP32, N = 192 or 256, steps without the
// DFT): a persistent CTA per SM walks its tiles of kLanes lines; while it transforms one
// tile, cp.async stages the next tile's psi^n values, and during the transform of the next
// the partial level it will update, into shared memory (each thread stages and later reads
// back only its own values, so cp.async.wait_group orders them and no barrier is needed).
// Stores of the updated level are fire-and-forget.  HBM sees the loads of one tile while
// the SM computes another, instead of each CTA alternating between the two.  At 256^3 the
// y pass gains 8% this way; the z pass (whose epilogue also applies the mask and source)
// is not faster with one 512-thread CTA per SM than the two-CTA kernel, so it keeps that one
// (AXIS 2 stays available here).
// ---------------------------------------------------------------------------------
template <typename R, int N> constexpr bool pipe_supported()
{
    return sizeof(R) == 4 && Plan<N>::T == 16 && N / Plan<N>::T <= 16 &&
           sizeof(float2) * ((size_t)N * kPitch + 2 * (size_t)N * kLanes) <= 227 * 1024;
}
template <typename R, int N> constexpr size_t pipe_smem()
{
    return sizeof(typename StepArgs<R>::C) * ((size_t)N * kPitch + 2 * (size_t)N * kLanes);
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// AXIS 1: lines along y (tile = x block, z plane); AXIS 2: lines along z (tile = x block, y row)
template <typename R, int N, int AXIS, bool SRC>
__global__ void __launch_bounds__(kLanes * Plan<N>::T, 1) colpass_pipe_kernel(const __grid_constant__ StepArgs<R> a)
{
    step_kernel_entry();
    using C = typename StepArgs<R>::C;
    constexpr int T = Plan<N>::T, E = N / T, R0 = Plan<N>::R[0];
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);            // FFT exchange tile [N][kPitch]
    C* cst = sm + (size_t)N * kPitch;               // staged psi^n      [N][kLanes]
    C* pst = cst + (size_t)N * kLanes;              // staged partial    [N][kLanes]
    const int lane = threadIdx.x % kLanes, j = threadIdx.x / kLanes;
    const int xtiles = (a.nx + kLanes - 1) / kLanes;
    const int other = AXIS == 1 ? a.nz : a.ny;
    const long long ntiles = (long long)xtiles * other * a.batch;
    const long long stride = AXIS == 1 ? (long long)a.nx : (long long)a.nx * a.ny;
    const C* __restrict__ tw = a.tw[AXIS];
    const R* __restrict__ kin = a.kin[AXIS];
    // tile t -> member b, in-plane index o, column x of this thread, base index
    auto decode = [&](long long t, int& b, int& o, int& x) -> long long {
        const int xt = (int)(t % xtiles);
        const long long r = t / xtiles;
        o = (int)(r % other);
        b = (int)(r / other);
        x = xt * kLanes + lane;
        return (long long)b * a.ncell + (AXIS == 1 ? (long long)o * a.nx * a.ny : (long long)o * a.nx) + x;
    };
    auto stage = [&](C* buf, const C* src, long long t) {
        int b, o, x;
        const long long base = decode(t, b, o, x);
        if (x < a.nx) {
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const int pos = slot_pos<N, T, R0>(q, j);
                cp_async8(&buf[pos * kLanes + lane], src + base + pos * stride);
            }
        }
        cp_async_commit();
    };
    long long t = blockIdx.x;
    if (t < ntiles) {
        stage(cst, a.cur, t);
        stage(pst, a.prev, t);
    }
    for (; t < ntiles; t += gridDim.x) {
        const long long tn = t + gridDim.x;
        int b, o, x;
        const long long base = decode(t, b, o, x);
        const bool act = x < a.nx;
        cp_async_wait<1>();                          // this tile's psi^n
        C v[E];
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = act ? cst[slot_pos<N, T, R0>(q, j) * kLanes + lane] : zero_c<R, C>();
        if (tn < ntiles) stage(cst, a.cur, tn);
        else cp_async_commit();
        kinetic_line<N, false>(v, sm, lane, j, tw, kin, R(a.mem[b].eta));
        cp_async_wait<1>();                          // this tile's partial level
        if (act) {
            if constexpr (AXIS == 1) {
#pragma unroll
                for (int q = 0; q < E; ++q) {
                    const int pos = slot_pos<N, T, R0>(q, j);
                    const C p = pst[pos * kLanes + lane];
                    a.prev[base + pos * stride] = mk<C>(p.x + v[q].y, p.y - v[q].x);
                }
            } else {
                const int y = o;
                const R gxy = a.mask[0][x] * a.mask[1][y];
                bool ok = true;
                int slo[3] = {0, 0, 0}, shi[3] = {0, 0, 0};
                if constexpr (SRC) source_box<R>(a, slo, shi);
                const bool src_col = SRC && x >= slo[0] && x < shi[0] && y >= slo[1] && y < shi[1];
                const C s = src_col ? a.tfac[(a.step - a.tfac_base) * a.batch + b] : zero_c<R, C>();
#pragma unroll
                for (int q = 0; q < E; ++q) {
                    const int z = slot_pos<N, T, R0>(q, j);
                    const long long idx = base + z * stride;
                    C p = pst[z * kLanes + lane];
                    if constexpr (SRC) {
                        if (src_col && z >= slo[2] && z < shi[2]) {
                            const C sa = source_acc<R, C>(a, b, s, x, y, z, idx);
                            p = mk<C>(p.x + a.c2 * sa.y, p.y - a.c2 * sa.x);
                        }
                    }
                    const R g = gxy * a.mask[2][z];
                    const C acc = mk<C>(g * (p.x + v[q].y), g * (p.y - v[q].x));
                    ok = ok && finite_c<R>(acc.x, acc.y);
                    a.prev[idx] = acc;
                }
                if (!ok) atomicOr(a.flag, 1);
            }
        }
        if (tn < ntiles) stage(pst, a.prev, tn);
        else cp_async_commit();
        __syncthreads();                             // the exchange tile is reused by the next tile
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------------
// TMA-fed y and z passes (FP32, lines of 128, 192 or 256 points, steps without the DFT).
// A persistent CTA per SM walks its tiles of kLanes lines.  Each tile's psi^n arrives by one
// tensor copy (cp.async.bulk.tensor, box 32 x N) into a ring of S shared-memory slots laid
// out [position][lane], completing on the slot's mbarrier.  The CTA reads its tile from the
// slot, issues the loads of the tile's read-modify-write operand into registers, and runs
// the line transform using the slot itself as the exchange tile (pitch kLanes: the lanes of
// a warp are consecutive, so every exchange is conflict-free).  Once every thread is done
// with the slot, thread 0 refills it with the tile S steps ahead, so S - 1 tiles of psi^n
// stream in from HBM while one is transformed; the operand's latency is covered by the
// transform.  Waits on the mbarriers are bounded in time: past the limit the kernel sets
// bit 1 of the grid's flag (reported as PSTD_ETIMEOUT), waits (bounded again) for its own
// copies in flight and returns.
// ---------------------------------------------------------------------------------
template <typename R, int N> constexpr bool tma_pass_supported()
{
    return sizeof(R) == 4 && (N == 128 || N == 192 || N == 256) && Plan<N>::S == 2 + (N == 192);
}
// ring depth: about 192 KB of slots per SM (two CTAs an SM share it at N = 128), at most 6
template <int N> __host__ __device__ constexpr int tma_ctas_sm() { return N == 128 ? 2 : 1; }
template <int N> __host__ __device__ constexpr int tma_slots()
{
    return (192 * 1024 / tma_ctas_sm<N>()) / (N * kLanes * 8) > 6 ? 6 : (192 * 1024 / tma_ctas_sm<N>()) / (N * kLanes * 8);
}
// dynamic shared memory: the slots (1024-byte aligned at run time, hence the pad), then the
// slots' mbarriers and the CTA's wait verdict
template <int N> constexpr size_t tma_smem() { return (size_t)tma_slots<N>() * N * kLanes * 8 + 1024 + 8 * 8 + 16; }

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// wait for phase `parity` of the mbarrier, for at most `limit_ns`; false when the limit passed
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// 3-D tiled tensor copy global -> shared, completing `bytes` on the mbarrier
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2, unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s: a tile normally lands in microseconds

template <typename R, int N, int AXIS, int SRC>
__global__ void __launch_bounds__(kLanes * Plan<N>::T, tma_ctas_sm<N>()) colpass_tma_kernel(const __grid_constant__ StepArgs<R> a)
{
    step_kernel_entry();
    using C = typename StepArgs<R>::C;
    constexpr int T = Plan<N>::T, E = N / T, R0 = Plan<N>::R[0];
    constexpr int S = tma_slots<N>();
    constexpr unsigned SLOT = (unsigned)N * kLanes;            // complex values per slot
    extern __shared__ __align__(16) unsigned char smraw[];
    // tensor copies land on 1024-byte-aligned slots: round the window's start up
    unsigned char* base_sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
    C* slots = reinterpret_cast<C*>(base_sm);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(base_sm + (size_t)S * SLOT * sizeof(C));
    int& ok_s = *reinterpret_cast<int*>(full + S);
    const int lane = threadIdx.x % kLanes, j = threadIdx.x / kLanes;
    const int xtiles = (a.nx + kLanes - 1) / kLanes;
    const int other = AXIS == 1 ? a.nz : a.ny;
    const long long ntiles = (long long)xtiles * other * a.batch;
    const long long stride = AXIS == 1 ? (long long)a.nx : (long long)a.nx * a.ny;
    const void* tmap = AXIS == 1 ? a.tmap_y : a.tmap_z;
    const C* __restrict__ tw = a.tw[AXIS];
    const R* __restrict__ kin = a.kin[AXIS];
    // tile t -> member b, in-plane index o (z for y lines, y for z lines), first column x0
    auto decode = [&](long long t, int& b, int& o, int& x0) {
        x0 = (int)(t % xtiles) * kLanes;
        const long long r = t / xtiles;
        o = (int)(r % other);
        b = (int)(r / other);
    };
    auto issue = [&](long long t, int s) {
        int b, o, x0;
        decode(t, b, o, x0);
        mbar_expect_tx(&full[s], SLOT * (unsigned)sizeof(C));
        if constexpr (AXIS == 1) tma_load_3d(slots + (size_t)s * SLOT, tmap, x0, 0, b * a.nz + o, &full[s]);
        else tma_load_3d(slots + (size_t)s * SLOT, tmap, x0, o, b * a.nz, &full[s]);
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int s = 0; s < S; ++s) {
            const long long t = blockIdx.x + (long long)s * gridDim.x;
            if (t < ntiles) issue(t, s);
        }
    }
    __syncthreads();
    int it = 0;
    bool timed_out = false;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int s = it % S;
        const unsigned parity = (unsigned)(it / S) & 1u;
        // one thread decides (so that every thread leaves together), then all observe the phase
        if (threadIdx.x == 0) ok_s = mbar_wait_bounded(&full[s], parity, kWaitLimitNs) ? 1 : 0;
        __syncthreads();
        if (!ok_s) { timed_out = true; break; }
        mbar_wait_bounded(&full[s], parity, kWaitLimitNs);
        C* slot = slots + (size_t)s * SLOT;
        int b, o, x0;
        decode(t, b, o, x0);
        const int x = x0 + lane;
        const bool act = x < a.nx;
        const long long base = (long long)b * a.ncell + (AXIS == 1 ? (long long)o * a.nx * a.ny : (long long)o * a.nx) + x;
        C v[E], pv[E];
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = slot[slot_pos<N, T, R0>(q, j) * kLanes + lane];
#pragma unroll
        for (int q = 0; q < E; ++q) pv[q] = act ? a.prev[base + slot_pos<N, T, R0>(q, j) * stride] : zero_c<R, C>();
        __syncthreads();                 // every value read before the slot becomes the exchange tile
        kinetic_line<N, false, kLanes>(v, slot, lane, j, tw, kin, R(a.mem[b].eta));
        // the slot is free: order this thread's accesses before the tensor copy that refills it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long tn = t + (long long)S * gridDim.x;
            if (tn < ntiles) issue(tn, s);
        }
        if (!act) continue;
        if constexpr (AXIS == 1) {
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const C p = pv[q];
                a.prev[base + slot_pos<N, T, R0>(q, j) * stride] = mk<C>(p.x + v[q].y, p.y - v[q].x);
            }
        } else {
            const int y = o;
            const R gxy = a.mask[0][x] * a.mask[1][y];
            bool ok = true;
            int slo[3] = {0, 0, 0}, shi[3] = {0, 0, 0};
            if constexpr (SRC) source_box<R>(a, slo, shi);
            const bool src_col = SRC != 0 && x >= slo[0] && x < shi[0] && y >= slo[1] && y < shi[1];
            const C sf = src_col ? a.tfac[(a.step - a.tfac_base) * a.batch + b] : zero_c<R, C>();
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const int z = slot_pos<N, T, R0>(q, j);
                const long long idx = base + z * stride;
                C p = pv[q];
                if constexpr (SRC) {
                    if (src_col && z >= slo[2] && z < shi[2]) {
                        const C sa = source_acc<R, C, SRC>(a, b, sf, x, y, z, idx);
                        p = mk<C>(p.x + a.c2 * sa.y, p.y - a.c2 * sa.x);
                    }
                }
                const R g = gxy * a.mask[2][z];
                const C acc = mk<C>(g * (p.x + v[q].y), g * (p.y - v[q].x));
                ok = ok && finite_c<R>(acc.x, acc.y);
                a.prev[idx] = acc;
            }
            if (!ok) atomicOr(a.flag, 1);
        }
    }
    if (timed_out) {
        if (threadIdx.x == 0) {
            atomicOr(a.flag, 2);
            // the copies this CTA still has in flight land in its own shared memory: wait for
            // them (bounded) before the CTA exits
            for (int k = 0; k < S; ++k) {
                const int itk = it + k;
                const long long tk = blockIdx.x + (long long)itk * gridDim.x;
                if (tk >= ntiles) break;
                mbar_wait_bounded(&full[itk % S], (unsigned)(itk / S) & 1u, kWaitLimitNs);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------
template <typename R, int N> size_t pass_smem() { return pass_smem_bytes<R, N>(); }

// Raise a kernel's dynamic shared-memory limit once per device instead of on every launch
// (one flag word per kernel: the template is keyed on the kernel itself).
template <auto kernel> cudaError_t set_smem_once(size_t bytes)
{
    static int done_mask = 0;   // bit d: set on device d (devices 0..30)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 31 && (__atomic_load_n(&done_mask, __ATOMIC_ACQUIRE) >> dev) & 1) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && dev < 31) __atomic_fetch_or(&done_mask, 1 << dev, __ATOMIC_RELEASE);
    return e;
}

// the alternative plan of a size where it exists, for FP32 (the per-axis choice in StepArgs::plan)
template <typename R, int N> constexpr bool alt_plan_built() { return sizeof(R) == 4 && has_alt_plan<N>(); }

template <typename R, int N, int PL> cudaError_t xpass_pl(const StepArgs<R>& a, const DftArgs<R>* d, int batch, cudaStream_t s)
{
    const size_t sm = d ? line_pass_smem<R, N, true, PL>() : line_pass_smem<R, N, false, PL>();
    cudaError_t e = d ? set_smem_once<xpass_kernel<R, N, true, PL>>(sm) : set_smem_once<xpass_kernel<R, N, false, PL>>(sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.ny * a.nz + kLanes - 1) / kLanes, batch);
    const DftArgs<R> none{};
    if (d) return launch_step_kernel(xpass_kernel<R, N, true, PL>, grid, dim3(kLanes * Plan<N, PL>::T), sm, s, a, *d);
    return launch_step_kernel(xpass_kernel<R, N, false, PL>, grid, dim3(kLanes * Plan<N, PL>::T), sm, s, a, none);
}

template <typename R, int N> cudaError_t xpass_n(const StepArgs<R>& a, const DftArgs<R>* d, int batch, cudaStream_t s)
{
    if constexpr (alt_plan_built<R, N>())
        if (a.plan[0]) return xpass_pl<R, N, 1>(a, d, batch, s);
    return xpass_pl<R, N, 0>(a, d, batch, s);
}
inline int sm_count()
{
    static int count[32] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 32) return 152;
    if (!count[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        count[dev] = n > 0 ? n : 152;
    }
    return count[dev];
}

template <typename R, int N, int AXIS, bool SRC> cudaError_t colpass_pipe_n(const StepArgs<R>& a, int batch, cudaStream_t s)
{
    if constexpr (pipe_supported<R, N>()) {
        const size_t sm = pipe_smem<R, N>();
        cudaError_t e = set_smem_once<colpass_pipe_kernel<R, N, AXIS, SRC>>(sm);
        if (e != cudaSuccess) return e;
        const long long ntiles = (long long)((a.nx + kLanes - 1) / kLanes) * (AXIS == 1 ? a.nz : a.ny) * batch;
        const dim3 grid((unsigned)std::min<long long>(ntiles, sm_count()));
        return launch_step_kernel(colpass_pipe_kernel<R, N, AXIS, SRC>, grid, dim3(kLanes * Plan<N>::T), sm, s, a);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename R, int N, int AXIS, int SRC> cudaError_t colpass_tma_n(const StepArgs<R>& a, int batch, cudaStream_t s)
{
    if constexpr (tma_pass_supported<R, N>()) {
        const size_t sm = tma_smem<N>();
        cudaError_t e = set_smem_once<colpass_tma_kernel<R, N, AXIS, SRC>>(sm);
        if (e != cudaSuccess) return e;
        const long long ntiles = (long long)((a.nx + kLanes - 1) / kLanes) * (AXIS == 1 ? a.nz : a.ny) * batch;
        const dim3 grid((unsigned)std::min<long long>(ntiles, (long long)sm_count() * tma_ctas_sm<N>()));
        return launch_step_kernel(colpass_tma_kernel<R, N, AXIS, SRC>, grid, dim3(kLanes * Plan<N>::T), sm, s, a);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename R, int N, int PL> cudaError_t ypass_pl(const StepArgs<R>& a, const DftArgs<R>* d, int batch, cudaStream_t s)
{
    const size_t sm = d ? line_pass_smem<R, N, true, PL>() : line_pass_smem<R, N, false, PL>();
    cudaError_t e = d ? set_smem_once<ypass_kernel<R, N, true, PL>>(sm) : set_smem_once<ypass_kernel<R, N, false, PL>>(sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.nx + kLanes - 1) / kLanes, a.nz, batch);
    const DftArgs<R> none{};
    if (d) return launch_step_kernel(ypass_kernel<R, N, true, PL>, grid, dim3(kLanes * Plan<N, PL>::T), sm, s, a, *d);
    return launch_step_kernel(ypass_kernel<R, N, false, PL>, grid, dim3(kLanes * Plan<N, PL>::T), sm, s, a, none);
}

template <typename R, int N> cudaError_t ypass_n(const StepArgs<R>& a, const DftArgs<R>* d, int batch, cudaStream_t s)
{
    if constexpr (tma_pass_supported<R, N>())
        if (!d && a.pipe_y == PSTD_LINE_TMA) return colpass_tma_n<R, N, 1, 0>(a, batch, s);
    if constexpr (pipe_supported<R, N>())
        if (!d && a.pipe_y == PSTD_LINE_PIPELINED) return colpass_pipe_n<R, N, 1, false>(a, batch, s);
    if constexpr (alt_plan_built<R, N>())
        if (a.plan[1]) return ypass_pl<R, N, 1>(a, d, batch, s);
    return ypass_pl<R, N, 0>(a, d, batch, s);
}
template <typename R, int N, bool DFT, int SRC, int PL>
cudaError_t zpass_launch_pl(const StepArgs<R>& a, const DftArgs<R>& d, int batch, cudaStream_t s)
{
    const size_t sm = line_pass_smem<R, N, DFT, PL>();
    cudaError_t e = set_smem_once<zpass_kernel<R, N, DFT, SRC, PL>>(sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.nx + kLanes - 1) / kLanes, a.ny, batch);
    return launch_step_kernel(zpass_kernel<R, N, DFT, SRC, PL>, grid, dim3(kLanes * Plan<N, PL>::T), sm, s, a, d);
}

template <typename R, int N, bool DFT, int SRC>
cudaError_t zpass_launch(const StepArgs<R>& a, const DftArgs<R>& d, int batch, cudaStream_t s)
{
    if constexpr (!DFT && tma_pass_supported<R, N>())
        if (a.tma_z) return colpass_tma_n<R, N, 2, SRC>(a, batch, s);
    if constexpr (alt_plan_built<R, N>())
        if (a.plan[2]) return zpass_launch_pl<R, N, DFT, SRC, 1>(a, d, batch, s);
    return zpass_launch_pl<R, N, DFT, SRC, 0>(a, d, batch, s);
}

template <typename R, int N>
cudaError_t zpass_n(const StepArgs<R>& a, const DftArgs<R>* d, int src, int batch, cudaStream_t s)
{
    const DftArgs<R> none{};
    const DftArgs<R>& dd = d ? *d : none;
    // FP64 keeps the plain and the general epilogue only (packets and the auxiliary wave take
    // the general one): half the FP64 z-pass variants to compile
    if (sizeof(R) == 8 && (src == 3 || src == 4)) src = 2;
    if constexpr (sizeof(R) == 8) {
        if (d) {
            if (src == 2) return zpass_launch<R, N, true, 2>(a, dd, batch, s);
            if (src == 1) return zpass_launch<R, N, true, 1>(a, dd, batch, s);
            return zpass_launch<R, N, true, 0>(a, dd, batch, s);
        }
        if (src == 2) return zpass_launch<R, N, false, 2>(a, dd, batch, s);
        if (src == 1) return zpass_launch<R, N, false, 1>(a, dd, batch, s);
        return zpass_launch<R, N, false, 0>(a, dd, batch, s);
    }
    if (d) {
        if (src == 4) return zpass_launch<R, N, true, 4>(a, dd, batch, s);
        if (src == 3) return zpass_launch<R, N, true, 3>(a, dd, batch, s);
        if (src == 2) return zpass_launch<R, N, true, 2>(a, dd, batch, s);
        if (src == 1) return zpass_launch<R, N, true, 1>(a, dd, batch, s);
        return zpass_launch<R, N, true, 0>(a, dd, batch, s);
    }
    if (src == 4) return zpass_launch<R, N, false, 4>(a, dd, batch, s);
    if (src == 3) return zpass_launch<R, N, false, 3>(a, dd, batch, s);
    if (src == 2) return zpass_launch<R, N, false, 2>(a, dd, batch, s);
    if (src == 1) return zpass_launch<R, N, false, 1>(a, dd, batch, s);
    return zpass_launch<R, N, false, 0>(a, dd, batch, s);
}

template <typename R, int N>
cudaError_t xypass_n(const StepArgs<R>& a, const DftArgs<R>* dx, const DftArgs<R>* dy, int batch, cudaStream_t s)
{
    if constexpr (xy_supported<R, N>()) {
        using C = typename StepArgs<R>::C;
        const dim3 grid(a.nz, batch);
        if (dx && dy) {
            const size_t sm = sizeof(C) * ((size_t)N * (N + 1) + xy_dft_red_elems<N>());
            cudaError_t e = set_smem_once<xypass_kernel<R, N, true>>(sm);
            if (e != cudaSuccess) return e;
            return launch_step_kernel(xypass_kernel<R, N, true>, grid, dim3(xy_threads<N>()), sm, s, a, *dx, *dy);
        }
        const size_t sm = sizeof(C) * (size_t)N * (N + 1);
        cudaError_t e = set_smem_once<xypass_kernel<R, N, false>>(sm);
        if (e != cudaSuccess) return e;
        const DftArgs<R> none{};
        return launch_step_kernel(xypass_kernel<R, N, false>, grid, dim3(xy_threads<N>()), sm, s, a, none, none);
    } else {
        return cudaErrorInvalidValue;
    }
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

template <typename R> cudaError_t launch_xpass(const StepArgs<R>& a, const DftArgs<R>* d, int batch, cudaStream_t s)
{
    PSTD_SIZE_DISPATCH(xpass_n, a.nx, a, d, batch, s)
}
template <typename R> cudaError_t launch_ypass(const StepArgs<R>& a, const DftArgs<R>* d, int batch, cudaStream_t s)
{
    PSTD_SIZE_DISPATCH(ypass_n, a.ny, a, d, batch, s)
}
template <typename R>
cudaError_t launch_zpass(const StepArgs<R>& a, const DftArgs<R>* d, int src, int batch, cudaStream_t s)
{
    PSTD_SIZE_DISPATCH(zpass_n, a.nz, a, d, src, batch, s)
}
// pipelined y pass: FP32, 192- or 256-point y lines
template <typename R> bool pipe_y_available(int ny)
{
    return (ny == 192 && pipe_supported<R, 192>()) || (ny == 256 && pipe_supported<R, 256>());
}
template <typename R> bool tma_pass_available(int n)
{
    return (n == 128 && tma_pass_supported<R, 128>()) || (n == 192 && tma_pass_supported<R, 192>()) ||
           (n == 256 && tma_pass_supported<R, 256>());
}
// fused xy pass, FP32 square planes: PSTD_XY_PLANE (one CTA per plane) for 64, 96 or 128;
// PSTD_XY_CLUSTER (a cluster of N / 32 CTAs per plane) for 128, 192 or 256
template <typename R> bool xypass_available(int nx, int ny, int mode)
{
    if (sizeof(R) != 4 || nx != ny) return false;
    if (mode == PSTD_XY_PLANE) return nx == 64 || nx == 96 || nx == 128;
    if (mode == PSTD_XY_CLUSTER) return nx == 128 || nx == 192 || nx == 256;
    return false;
}
template <typename R, int N, bool DFT, int PL = 0>
cudaError_t xycl_launch(const StepArgs<R>& a, const DftArgs<R>& dx, const DftArgs<R>& dy, int batch, cudaStream_t s)
{
    static_assert(!DFT || pass_smem_bytes<R, N>() + 2 * dft_red_bytes<R, N, PL>() <= (size_t)227 * 1024, "two DFT slots");
    const size_t sm = pass_smem_bytes<R, N>() + (DFT ? 2 * dft_red_bytes<R, N, PL>() : 0);
    cudaError_t e = set_smem_once<xycl_kernel<R, N, DFT, PL>>(sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(N / kLanes, a.nz, batch);
    cfg.blockDim = dim3(kLanes * Plan<N, PL>::T);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = N / kLanes;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    int na = 1;
#if PSTD_PDL
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    na = 2;
#endif
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, xycl_kernel<R, N, DFT, PL>, a, dx, dy);
}

template <typename R, int N>
cudaError_t xycl_n(const StepArgs<R>& a, const DftArgs<R>* dx, const DftArgs<R>* dy, int batch, cudaStream_t s)
{
    if constexpr (xycl_supported<R, N>()) {
        const DftArgs<R> none{};
        if constexpr (alt_plan_built<R, N>()) {
            if (a.plan[0] && a.plan[1]) {
                if (dx && dy) return xycl_launch<R, N, true, 1>(a, *dx, *dy, batch, s);
                return xycl_launch<R, N, false, 1>(a, none, none, batch, s);
            }
        }
        if (dx && dy) return xycl_launch<R, N, true>(a, *dx, *dy, batch, s);
        return xycl_launch<R, N, false>(a, none, none, batch, s);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename R>
cudaError_t launch_xypass(const StepArgs<R>& a, const DftArgs<R>* dx, const DftArgs<R>* dy, int batch, cudaStream_t s,
                          int mode)
{
    if (!xypass_available<R>(a.nx, a.ny, mode)) return cudaErrorInvalidValue;
    if (mode == PSTD_XY_PLANE) {
        switch (a.nx) {
        case 64: return xypass_n<R, 64>(a, dx, dy, batch, s);
        case 96: return xypass_n<R, 96>(a, dx, dy, batch, s);
        case 128: return xypass_n<R, 128>(a, dx, dy, batch, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (a.nx) {
    case 128: return xycl_n<R, 128>(a, dx, dy, batch, s);
    case 192: return xycl_n<R, 192>(a, dx, dy, batch, s);
    case 256: return xycl_n<R, 256>(a, dx, dy, batch, s);
    default: return cudaErrorInvalidValue;
    }
}
// ---------------------------------------------------------------------------------
// the 1-D auxiliary incident wave (Section 2.2.3)
// ---------------------------------------------------------------------------------
// G_m^n = G0_m e^{-i theta_m n} for the steps of one call: the Fourier coefficients of the 1-D
// leapfrog's solution, in which every mode advances by its root e^{-i theta_m} per step
// (theta_m = asin(dt eta hbar q_m^2 / 2m)); phases and products in FP64, rounded once
template <typename R>
__global__ void __launch_bounds__(256) aux_table_kernel(const double2* G0, const double* theta, const double* q, int nslot,
                                                        int nm, long long n0, long nsteps, int deriv,
                                                        typename StepArgs<R>::C* G, typename StepArgs<R>::C* dG)
{
    step_kernel_entry();
    using C = typename StepArgs<R>::C;
    const long long total = (long long)nslot * nsteps * nm;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(e % nm);
        const long long rest = e / nm;
        const long long st = rest % nsteps;
        const int slot = (int)(rest / nsteps);
        const long long k = (long long)slot * nm + m;
        double sn, cs;
        sincos(-theta[k] * (double)(n0 + st), &sn, &cs);
        const double gr = G0[k].x * cs - G0[k].y * sn, gi = G0[k].x * sn + G0[k].y * cs;
        G[e] = mk<C>(R(gr), R(gi));
        if (deriv) dG[e] = mk<C>(R(-q[k] * gi), R(q[k] * gr));
    }
}

constexpr int kAuxChunk = 1024;   // modes staged in shared memory at a time (a multiple of 32)

// one Horner step p u + g as four fused multiply-adds
template <typename C> __device__ __forceinline__ C horner_step(C p, C u, C g)
{
    if constexpr (sizeof(C) == 8) {
        return mk<C>(__fmaf_rn(p.x, u.x, __fmaf_rn(-p.y, u.y, g.x)), __fmaf_rn(p.x, u.y, __fmaf_rn(p.y, u.x, g.y)));
    } else {
        return mk<C>(__fma_rn(p.x, u.x, __fma_rn(-p.y, u.y, g.x)), __fma_rn(p.x, u.y, __fma_rn(p.y, u.x, g.y)));
    }
}

// psi_inc^n (and d psi_inc^n / d d) at every node of the box for every aux slot: the series of
// Eqs. pstd_psiinc, pstd_dpsiinc, sum_m G_m e^{i (q_0 + m dq) d} = e^{i q_0 d} P(u), u = e^{i dq d},
// P(u) = sum_m G_m u^m evaluated by Horner's rule in blocks of 32 modes (u within a block, u^32
// from block to block): one complex multiply-add per mode, at most 32 + nm / 32 rounded steps
template <typename R> __global__ void __launch_bounds__(256) aux_eval_kernel(const __grid_constant__ AuxEvalArgs<R> a)
{
    step_kernel_entry();
    using C = typename StepArgs<R>::C;
    __shared__ __align__(16) C sg[kAuxChunk];
    __shared__ __align__(16) C sd[kAuxChunk];
    const int slot = blockIdx.y;
    const long long nb = (long long)a.bn[0] * a.bn[1] * a.bn[2];
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool act = e < nb;
    const bool deriv = a.dG != nullptr;
    const C zero = mk<C>(R(0), R(0));
    C base = zero, u = zero, u32 = zero, acc = zero, dacc = zero;
    if (act) {
        const int x = a.lo[0] + (int)(e % a.bn[0]);
        const int y = a.lo[1] + (int)((e / a.bn[0]) % a.bn[1]);
        const int z = a.lo[2] + (int)(e / ((long long)a.bn[0] * a.bn[1]));
        const long long ix = (long long)slot * a.n[0] + x, iy = (long long)slot * a.n[1] + y, iz = (long long)slot * a.n[2] + z;
        base = cmul(cmul(a.t0[0][ix], a.t0[1][iy]), a.t0[2][iz]);
        u = cmul(cmul(a.t1[0][ix], a.t1[1][iy]), a.t1[2][iz]);
        u32 = cmul(cmul(a.t32[0][ix], a.t32[1][iy]), a.t32[2][iz]);
    }
    const C* G = a.G + slot * a.slot_stride + a.step_off * a.nm;
    const C* dG = deriv ? a.dG + slot * a.slot_stride + a.step_off * a.nm : nullptr;
    for (int c0 = ((a.nm - 1) / kAuxChunk) * kAuxChunk; c0 >= 0; c0 -= kAuxChunk) {
        const int cn = min(kAuxChunk, a.nm - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < cn; i += blockDim.x) {
            sg[i] = G[c0 + i];
            if (deriv) sd[i] = dG[c0 + i];
        }
        __syncthreads();
        if (!act) continue;
        for (int b0 = cn - 32; b0 >= 0; b0 -= 32) {
            C p;
            if constexpr (sizeof(C) == 8) {
                // FP32: two modes per 16-byte shared-memory read (b0 is a multiple of 32)
                const float4* g4 = reinterpret_cast<const float4*>(sg + b0);
                float4 q = g4[15];
                p = mk<C>(q.z, q.w);
                p = horner_step(p, u, mk<C>(q.x, q.y));
#pragma unroll
                for (int t = 14; t >= 0; --t) {
                    q = g4[t];
                    p = horner_step(p, u, mk<C>(q.z, q.w));
                    p = horner_step(p, u, mk<C>(q.x, q.y));
                }
            } else {
                p = sg[b0 + 31];
#pragma unroll
                for (int j = 30; j >= 0; --j) p = horner_step(p, u, sg[b0 + j]);
            }
            acc = horner_step(acc, u32, p);
            if (deriv) {
                C dp = sd[b0 + 31];
#pragma unroll
                for (int j = 30; j >= 0; --j) dp = horner_step(dp, u, sd[b0 + j]);
                dacc = horner_step(dacc, u32, dp);
            }
        }
    }
    if (act) {
        a.out[slot * nb + e] = cmul(base, acc);
        if (deriv) a.dout[slot * nb + e] = cmul(base, dacc);
    }
}

template <typename R>
cudaError_t launch_aux_table(const double2* G0, const double* theta, const double* q, int nslot, int nm, long long n0,
                             long nsteps, bool deriv, typename std::conditional<sizeof(R) == 4, float2, double2>::type* G,
                             typename std::conditional<sizeof(R) == 4, float2, double2>::type* dG, cudaStream_t s)
{
    const long long total = (long long)nslot * nsteps * nm;
    if (total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 152LL * 16);
    return launch_step_kernel(aux_table_kernel<R>, dim3(blocks), dim3(256), 0, s, G0, theta, q, nslot, nm, n0, nsteps,
                              deriv ? 1 : 0, G, dG);
}

template <typename R> cudaError_t launch_aux_eval(const AuxEvalArgs<R>& a, cudaStream_t s)
{
    const long long nb = (long long)a.bn[0] * a.bn[1] * a.bn[2];
    if (nb <= 0 || a.nslot <= 0) return cudaSuccess;
    return launch_step_kernel(aux_eval_kernel<R>, dim3((unsigned)((nb + 255) / 256), (unsigned)a.nslot), dim3(256), 0, s, a);
}

template <typename R> cudaError_t launch_source(const StepArgs<R>& a, int batch, cudaStream_t s)
{
    int lo[3], hi[3];
    source_box<R>(a, lo, hi);
    const int bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
    if (bx <= 0 || by <= 0 || bz <= 0) return cudaSuccess;
    dim3 grid((unsigned)((bx + 31) / 32), (unsigned)((by + 3) / 4), (unsigned)(((bz + kSourceZ - 1) / kSourceZ) * batch));
    return launch_step_kernel(source_kernel<R>, grid, dim3(128), 0, s, a, lo[0], lo[1], lo[2], bx, by, bz);
}

}  // namespace pstd
