// Line FFT engine for the spectral kinetic operator F_a^-1[k_a^2 F_a u] (Eq. spatialFFTeigen).
//
// A CTA works on LANES lines at once (one warp lane per line) with T threads per
// line (thread slot j = warp index).  Each thread keeps E = N/T complex values in
// registers.  A length-N transform is a chain of Stockham radix stages; stage s
// (radix R_s, sub-transform size Ns before it) computes, for butterfly b,
//     v_r = x[b + r N/R] * w_{Ns R}^{r (b mod Ns)},   X = DFT_R(v),
//     y[(b / Ns) Ns R + (b mod Ns) + r Ns] = X_r,
// which ends in natural order.  Between stages the values are exchanged through a
// shared-memory tile laid out [position][lane] (row pitch LANES + 1 complex, which
// keeps both the lane-major exchanges and the transposing loads of x-lines free of
// bank conflicts).  The last forward stage leaves each thread holding spectrum
// entries b + r N/R_last -- exactly the inputs of the first inverse stage when the
// inverse runs the radices in reverse order -- so the k^2 multiply happens in
// registers with no exchange, and the final inverse stage returns the values to the
// positions the thread loaded.  Twiddles w_N^m come from a per-axis table computed
// on the host in double precision from the definition.
#pragma once

#include <cuda_runtime.h>

namespace pstd {

template <typename R> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) { C c; c.x = a; c.y = b; return c; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __device__ __forceinline__ C cconjmul(C a, C w) { return mk<C>(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// Butterfly sums, differences and scalings of the small DFTs below.  With PSTD_F32X2 those of
// FP32 values (float2) are single packed two-lane instructions (add/sub/mul .f32x2, round to
// nearest: each lane rounds exactly as the scalar operation does).  cs32, an FP32 complex of
// another type, keeps the scalar forms for kernels where they schedule better.
#ifndef PSTD_F32X2
#define PSTD_F32X2 1
#endif
struct __align__(8) cs32 { float x, y; };
template <typename C> __device__ __forceinline__ C ldg_c(const C* p) { return __ldg(p); }
template <> __device__ __forceinline__ cs32 ldg_c<cs32>(const cs32* p)
{
    const float2 w = __ldg(reinterpret_cast<const float2*>(p));
    return cs32{w.x, w.y};
}
template <typename C> __device__ __forceinline__ C bfadd(C a, C b) { return cadd(a, b); }
template <typename C> __device__ __forceinline__ C bfsub(C a, C b) { return csub(a, b); }
template <typename C> __device__ __forceinline__ C bfscale(C a, decltype(C::x) s) { return cscale(a, s); }
#if PSTD_F32X2
__device__ __forceinline__ unsigned long long pk2(float2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 up2(unsigned long long r)
{
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(r));
    return d;
}
template <> __device__ __forceinline__ float2 bfadd<float2>(float2 a, float2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return up2(d);
}
template <> __device__ __forceinline__ float2 bfsub<float2>(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return up2(d);
}
template <> __device__ __forceinline__ float2 bfscale<float2>(float2 a, float s)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(make_float2(s, s))));
    return up2(d);
}
#endif
#ifndef PSTD_F32X2_KIN
#define PSTD_F32X2_KIN 1
#endif
// the spectral multiply of kinetic_line (packed with PSTD_F32X2_KIN: 5% off the 256-point passes)
template <typename C> __device__ __forceinline__ C kscale(C a, decltype(C::x) s)
{
#if PSTD_F32X2_KIN
    return bfscale(a, s);
#else
    return cscale(a, s);
#endif
}
// multiply by -i*DIR... helpers: i*a and -i*a
template <typename C> __device__ __forceinline__ C mul_i(C a) { return mk<C>(-a.y, a.x); }
template <typename C> __device__ __forceinline__ C mul_mi(C a) { return mk<C>(a.y, -a.x); }
// multiply by (DIR * i): DIR = -1 forward (e^{-i...}), +1 inverse
template <int DIR, typename C> __device__ __forceinline__ C mul_dir_i(C a) { return DIR < 0 ? mul_mi(a) : mul_i(a); }

// ---------------------------------------------------------------------------------
// small DFTs in registers, X_k = sum_n x_n e^{DIR 2 pi i n k / R}
// ---------------------------------------------------------------------------------
template <int DIR, typename C> __device__ __forceinline__ void dft2(C& a, C& b)
{
    C t = a;
    a = bfadd(t, b);
    b = bfsub(t, b);
}

template <int DIR, typename C> __device__ __forceinline__ void dft3(C& a, C& b, C& c)
{
    using R = decltype(C::x);
    const R h = R(0.8660254037844386467637231707529362);   // sin(2 pi / 3)
    C s = bfadd(b, c);
    C d = bfsub(b, c);
    C m = mk<C>(a.x - R(0.5) * s.x, a.y - R(0.5) * s.y);
    a = bfadd(a, s);
    // DIR i sin(2pi/3) (b - c)
    C r = bfscale(mul_dir_i<DIR>(d), h);
    b = bfadd(m, r);
    c = bfsub(m, r);
}

template <int DIR, typename C> __device__ __forceinline__ void dft4(C& a, C& b, C& c, C& d)
{
    C t0 = bfadd(a, c), t1 = bfsub(a, c), t2 = bfadd(b, d), t3 = bfsub(b, d);
    C r = mul_dir_i<DIR>(t3);
    a = bfadd(t0, t2);
    c = bfsub(t0, t2);
    b = bfadd(t1, r);
    d = bfsub(t1, r);
}

// twiddle w_R^k for compile-time R, k with sign DIR (cos 2pi k/R + DIR i sin 2pi k/R)
template <int DIR, typename C> __device__ __forceinline__ C tw_mul8(C a, int k)
{
    // a * e^{DIR 2 pi i k / 8} for k = 0..3
    using R = decltype(C::x);
    const R s = R(0.7071067811865475244008443621048490);
    if (k == 0) return a;
    if (k == 1) return bfscale(bfadd(a, mul_dir_i<DIR>(a)), s);
    if (k == 2) return mul_dir_i<DIR>(a);
    return bfscale(bfsub(mul_dir_i<DIR>(a), a), s);
}

template <int DIR, typename C> __device__ __forceinline__ void dft8(C* x)
{
    // radix-2 split: even part x0 x2 x4 x6, odd part x1 x3 x5 x7
    C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    o1 = tw_mul8<DIR>(o1, 1);
    o2 = tw_mul8<DIR>(o2, 2);
    o3 = tw_mul8<DIR>(o3, 3);
    x[0] = bfadd(e0, o0); x[4] = bfsub(e0, o0);
    x[1] = bfadd(e1, o1); x[5] = bfsub(e1, o1);
    x[2] = bfadd(e2, o2); x[6] = bfsub(e2, o2);
    x[3] = bfadd(e3, o3); x[7] = bfsub(e3, o3);
}

template <int DIR, typename C> __device__ __forceinline__ C tw16(C a, int k)
{
    // multiply by e^{DIR 2 pi i k / 16}, k in 0..9 (compile-time after unrolling)
    using R = decltype(C::x);
    const R c1 = R(0.9238795325112867561281831893967883);   // cos(pi/8)
    const R s1 = R(0.3826834323650897717284599840303989);   // sin(pi/8)
    const R c2 = R(0.7071067811865475244008443621048490);
    R cr, ci;
    switch (k) {
    case 0: return a;
    case 1: cr = c1; ci = s1; break;
    case 2: cr = c2; ci = c2; break;
    case 3: cr = s1; ci = c1; break;
    case 4: cr = 0; ci = 1; break;
    case 6: cr = -c2; ci = c2; break;
    case 9: cr = -c1; ci = -s1; break;
    default: {
        // generic (not reached for the 4x4 split)
        cr = R(1); ci = R(0); break;
    }
    }
    ci = DIR < 0 ? -ci : ci;
    return mk<C>(a.x * cr - a.y * ci, a.x * ci + a.y * cr);
}

template <int DIR, typename C> __device__ __forceinline__ void dft16(C* x)
{
    // 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2
    C y[16];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        C a = x[n2], b = x[4 + n2], c = x[8 + n2], d = x[12 + n2];
        dft4<DIR>(a, b, c, d);
        y[0 * 4 + n2] = a;
        y[1 * 4 + n2] = tw16<DIR>(b, 1 * n2);
        y[2 * 4 + n2] = tw16<DIR>(c, 2 * n2);
        y[3 * 4 + n2] = tw16<DIR>(d, 3 * n2);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C a = y[k1 * 4 + 0], b = y[k1 * 4 + 1], c = y[k1 * 4 + 2], d = y[k1 * 4 + 3];
        dft4<DIR>(a, b, c, d);
        x[k1 + 0] = a;
        x[k1 + 4] = b;
        x[k1 + 8] = c;
        x[k1 + 12] = d;
    }
}

template <int DIR, typename C> __device__ __forceinline__ void dft12(C* x)
{
    // Good-Thomas 4 x 3 (coprime, no twiddles): n = (3 n1 + 4 n2) mod 12, k = (9 k1 + 4 k2) mod 12
    C y[12];
#pragma unroll
    for (int n2 = 0; n2 < 3; ++n2) {
        C a = x[(0 + 4 * n2) % 12], b = x[(3 + 4 * n2) % 12], c = x[(6 + 4 * n2) % 12], d = x[(9 + 4 * n2) % 12];
        dft4<DIR>(a, b, c, d);
        y[0 * 3 + n2] = a;
        y[1 * 3 + n2] = b;
        y[2 * 3 + n2] = c;
        y[3 * 3 + n2] = d;
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C a = y[k1 * 3 + 0], b = y[k1 * 3 + 1], c = y[k1 * 3 + 2];
        dft3<DIR>(a, b, c);
        x[(9 * k1 + 0) % 12] = a;
        x[(9 * k1 + 4) % 12] = b;
        x[(9 * k1 + 8) % 12] = c;
    }
}

template <int RAD, int DIR, typename C> __device__ __forceinline__ void dft(C* x)
{
    if constexpr (RAD == 2) dft2<DIR>(x[0], x[1]);
    else if constexpr (RAD == 3) dft3<DIR>(x[0], x[1], x[2]);
    else if constexpr (RAD == 4) dft4<DIR>(x[0], x[1], x[2], x[3]);
    else if constexpr (RAD == 8) dft8<DIR>(x);
    else if constexpr (RAD == 12) dft12<DIR>(x);
    else if constexpr (RAD == 16) dft16<DIR>(x);
    else static_assert(RAD == 2, "unsupported radix");
}

// ---------------------------------------------------------------------------------
// plans: radices (forward order) and threads per line; E = N / T must be a multiple
// of every radix so each thread runs E / R butterflies per stage
// ---------------------------------------------------------------------------------
// PL = 0: the default plan of each size; PL = 1: an alternative for 128 and 256 with twice the
// threads a line and half the values a thread (radix-8 and radix-4 stages, one more exchange),
// whose butterflies fit the 64-register budget of two resident CTAs without spilling.  The
// step variants' autotuner picks between them per axis.
template <int N, int PL = 0> struct Plan;
template <int N> constexpr bool has_alt_plan() { return N == 128 || N == 256; }
template <> struct Plan<128, 1> { static constexpr int T = 16; static constexpr int S = 3; static constexpr int R[4] = {8, 4, 4, 0}; };
template <> struct Plan<256, 1> { static constexpr int T = 32; static constexpr int S = 3; static constexpr int R[4] = {8, 8, 4, 0}; };
template <> struct Plan<8>   { static constexpr int T = 1;  static constexpr int S = 1; static constexpr int R[4] = {8, 0, 0, 0}; };
template <> struct Plan<12>  { static constexpr int T = 1;  static constexpr int S = 1; static constexpr int R[4] = {12, 0, 0, 0}; };
template <> struct Plan<16>  { static constexpr int T = 1;  static constexpr int S = 1; static constexpr int R[4] = {16, 0, 0, 0}; };
template <> struct Plan<24>  { static constexpr int T = 2;  static constexpr int S = 2; static constexpr int R[4] = {12, 2, 0, 0}; };
template <> struct Plan<32>  { static constexpr int T = 4;  static constexpr int S = 2; static constexpr int R[4] = {8, 4, 0, 0}; };
template <> struct Plan<48>  { static constexpr int T = 4;  static constexpr int S = 2; static constexpr int R[4] = {12, 4, 0, 0}; };
template <> struct Plan<64>  { static constexpr int T = 8;  static constexpr int S = 2; static constexpr int R[4] = {8, 8, 0, 0}; };
template <> struct Plan<96>  { static constexpr int T = 4;  static constexpr int S = 2; static constexpr int R[4] = {12, 8, 0, 0}; };
template <> struct Plan<128> { static constexpr int T = 8;  static constexpr int S = 2; static constexpr int R[4] = {16, 8, 0, 0}; };
template <> struct Plan<192> { static constexpr int T = 16; static constexpr int S = 3; static constexpr int R[4] = {12, 4, 4, 0}; };
template <> struct Plan<256> { static constexpr int T = 16; static constexpr int S = 2; static constexpr int R[4] = {16, 16, 0, 0}; };
// 384: four stages with 32 threads a line, so that a thread holds 12 values (not 24) and a
// 1024-thread CTA of 32 lines fits 64 registers a thread
template <> struct Plan<384> { static constexpr int T = 32; static constexpr int S = 4; static constexpr int R[4] = {12, 4, 4, 2}; };

#ifndef PSTD_LANES
#define PSTD_LANES 32
#endif
constexpr int kLanes = PSTD_LANES;    // lines per CTA (thread index = j * kLanes + line)
constexpr int kPitch = kLanes + 1;    // shared-memory row pitch (complex elements)

// Element (pos, lane) of an exchange tile: at pos * PS + lane * LS (the [pos][lane] tile of
// kLanes lines by default), or, with PS == 0, in row `lane` of N values with the low four bits
// of pos XORed with the next four.  The swizzled rows serve lines whose 16 threads are
// consecutive lanes (the x pass at N = 256): a stage writing positions 16 j + r and the next
// reading positions j + 16 r then touch 16 distinct bank pairs per half-warp.
template <int N, int PS, int LS> __device__ __forceinline__ int tile_addr(int pos, int lane)
{
    if constexpr (PS == 0) return lane * N + (pos ^ ((pos >> 4) & 15));
    else return pos * PS + lane * LS;
}

// One Stockham stage.  v holds the thread's E values; on entry they are the stage's
// inputs when !FROM_SMEM, otherwise the inputs are read from the tile.  On exit the
// outputs are in v, and also in the tile when TO_SMEM (addressed by tile_addr).
template <int N, int T, int RAD, int NS, int DIR, bool FROM_SMEM, bool TO_SMEM, int PS = kPitch, int LS = 1,
          typename C, int E>
__device__ __forceinline__ void stockham_stage(C (&v)[E], C* sm, int lane, int j, const C* __restrict__ tw)
{
    constexpr int NB = E / RAD;
    static_assert(NB * RAD == E, "radix must divide E");
    if constexpr (FROM_SMEM) {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            const int b = j + t * T;
#pragma unroll
            for (int r = 0; r < RAD; ++r) v[t * RAD + r] = sm[tile_addr<N, PS, LS>(b + r * (N / RAD), lane)];
        }
        if constexpr (TO_SMEM) __syncthreads();
    }
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        const int b = j + t * T;
        C* x = &v[t * RAD];
        if constexpr (NS > 1) {
            const int bm = b % NS;
            constexpr int step = N / (NS * RAD);
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                const C w = ldg_c(&tw[r * bm * step]);
                x[r] = DIR < 0 ? cmul(x[r], w) : cconjmul(x[r], w);
            }
        }
        dft<RAD, DIR>(x);
    }
    if constexpr (TO_SMEM) {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            const int b = j + t * T;
            const int base = (b / NS) * NS * RAD + (b % NS);
#pragma unroll
            for (int r = 0; r < RAD; ++r) sm[tile_addr<N, PS, LS>(base + r * NS, lane)] = v[t * RAD + r];
        }
        __syncthreads();
    }
}

// position of register slot q (= t * RAD0 + r) in the natural-order line, for the
// distribution that the first forward stage reads and the last inverse stage writes
template <int N, int T, int RAD0> __device__ __forceinline__ int slot_pos(int q, int j)
{
    return j + (q / RAD0) * T + (q % RAD0) * (N / RAD0);
}
// position of register slot q in the spectrum after the last forward stage
template <int N, int T, int RADL> __device__ __forceinline__ int spec_pos(int q, int j)
{
    return j + (q / RADL) * T + (q % RADL) * (N / RADL);
}

// F^-1[ mult * F[v] ] for one line held as described above.  `kin` is the real
// multiplier in FFT index order (already including 1/N).  FIRST_FROM_SMEM: the
// inputs sit in the tile (x-lines loaded by a transposing copy) instead of v.  PS: the
// exchange tile's row pitch (kLanes itself is conflict-free for the column passes, whose
// lanes are consecutive; the transposing x-line copy needs kLanes + 1).
template <int N, bool FIRST_FROM_SMEM, int PS = kPitch, int PL = 0, typename C, int E>
__device__ __forceinline__ void kinetic_line(C (&v)[E], C* sm, int lane, int j, const C* __restrict__ tw,
                                             const decltype(C::x)* __restrict__ kin, decltype(C::x) scale)
{
    using P = Plan<N, PL>;
    constexpr int T = P::T;
    static_assert(E == N / T, "E");
    constexpr int R0 = P::R[0], R1 = P::R[1], R2 = P::R[2], R3 = P::R[3];
    if constexpr (P::S == 1) {
        if constexpr (FIRST_FROM_SMEM) {
#pragma unroll
            for (int q = 0; q < E; ++q) v[q] = sm[tile_addr<N, PS, 1>(slot_pos<N, T, R0>(q, j), lane)];
        }
        stockham_stage<N, T, R0, 1, -1, false, false, PS>(v, sm, lane, j, tw);
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = kscale(v[q], __ldg(&kin[spec_pos<N, T, R0>(q, j)]) * scale);
        stockham_stage<N, T, R0, 1, +1, false, false, PS>(v, sm, lane, j, tw);
    } else if constexpr (P::S == 2) {
        stockham_stage<N, T, R0, 1, -1, FIRST_FROM_SMEM, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R1, R0, -1, true, false, PS>(v, sm, lane, j, tw);
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = kscale(v[q], __ldg(&kin[spec_pos<N, T, R1>(q, j)]) * scale);
        __syncthreads();   // every thread has read the tile before it is rewritten
        stockham_stage<N, T, R1, 1, +1, false, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R0, R1, +1, true, false, PS>(v, sm, lane, j, tw);
    } else if constexpr (P::S == 4) {
        stockham_stage<N, T, R0, 1, -1, FIRST_FROM_SMEM, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R1, R0, -1, true, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R2, R0 * R1, -1, true, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R3, R0 * R1 * R2, -1, true, false, PS>(v, sm, lane, j, tw);
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = kscale(v[q], __ldg(&kin[spec_pos<N, T, R3>(q, j)]) * scale);
        __syncthreads();
        stockham_stage<N, T, R3, 1, +1, false, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R2, R3, +1, true, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R1, R3 * R2, +1, true, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R0, R3 * R2 * R1, +1, true, false, PS>(v, sm, lane, j, tw);
    } else {
        stockham_stage<N, T, R0, 1, -1, FIRST_FROM_SMEM, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R1, R0, -1, true, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R2, R0 * R1, -1, true, false, PS>(v, sm, lane, j, tw);
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = kscale(v[q], __ldg(&kin[spec_pos<N, T, R2>(q, j)]) * scale);
        __syncthreads();
        stockham_stage<N, T, R2, 1, +1, false, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R1, R2, +1, true, true, PS>(v, sm, lane, j, tw);
        stockham_stage<N, T, R0, R2 * R1, +1, true, false, PS>(v, sm, lane, j, tw);
    }
}

}  // namespace pstd
