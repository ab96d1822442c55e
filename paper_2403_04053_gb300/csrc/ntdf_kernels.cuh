// Near-to-distant-field transform (Section 3).
//
// Points (transform_kernel): per surface cell, the integral of the trigonometric
// interpolant psi_an (Eq. AnBottomPsi) times the linearised Green's phase
// e^{-ik Rhat . dr'} (the approximation behind Eqs. bottomPsi_lm ... leftrightPsi_ln),
//
//   Psi_cell(r) = -sigma/(4 pi) e^{ikR}/R  int_cell [d_a psi_an + (ik - 1/R) Rhat_a psi_an] e^{-ik Rhat . dr'} dS',
//
// summed over the cells of the six faces (Eq. Psi).  Each cell integral is a G x G
// Gauss-Legendre sum over node values prepared once per (member, frequency)
// ("records", weights and the cell Jacobian folded in); the in-plane phase at the
// nodes factors into e_g(axis b) f_h(axis c).  The distance is split as
// R = R0 + dR, R0 = |r - face centre| in double precision and
// dR = (|dc|^2 - 2 d0 . dc) / (R + R0) in the working precision, so single-precision
// phases stay accurate at kR ~ 10^3.
//
// Far field (farfield_kernel): in the r -> infinity limit the per-cell phase is exactly
// linear across the whole face, so the sum over cells of the per-cell sinc sums of
// Eq. bottomPsi_lm factorises.  With C the 2-D DFT of the plane (Eq. AnBottomPsi),
//   f_face = -sigma D_b D_c / (4 pi N_b N_c) e^{-ik rhat_a a_plane}
//            sum_{i',j'} C[j', i'] at_{i'} bt_{j'} [d_a-plane ... ]
//   at_{i'} = sum_l (-1)^{i'} e^{2 pi i i' x^c_l / L_b} sinc(pi i'/N_b - k D_b rhat_b / 2) e^{-ik rhat_b x^c_l}
//           = n sinc(n phi / 2) e^{i (k rhat_b L_b / 2 + phi (lo + hi) / 2)},  phi = 2 pi i'/N_b - k rhat_b D_b,
// n = hi - lo surface cells along b (and bt likewise along c): the paper's far-field sum in
// closed form, N_b N_c multiply-adds per direction and face.
#pragma once

#include <type_traits>

#include "fft_line.cuh"
#include "pstd_internal.h"

namespace pstd {

template <typename R> __device__ __forceinline__ void sincos_r(R x, R* s, R* c)
{
    if constexpr (sizeof(R) == 4) sincosf(x, s, c);
    else sincos(x, s, c);
}

// sin/cos of a small argument (|x| <= pi/2 for any grid with >= 2 points per wavelength):
// the hardware approximation in single precision (absolute error ~4e-7), exact in double.
template <typename R> __device__ __forceinline__ void sincos_small(R x, R* s, R* c)
{
    if constexpr (sizeof(R) == 4) __sincosf(x, s, c);
    else sincos(x, s, c);
}

// sin/cos of a moderate argument (|x| up to ~10^4): in single precision a two-constant
// Cody-Waite reduction by 2 pi (6.28125 is exact in 8 bits) then the hardware approximation.
template <typename R> __device__ __forceinline__ void sincos_mid(R x, R* s, R* c)
{
    if constexpr (sizeof(R) == 4) {
        const float n = rintf(x * 0.159154943091895336f);
        float r = fmaf(-n, 6.28125f, x);
        r = fmaf(-n, 1.93530717958647692529e-3f, r);
        __sincosf(r, s, c);
    } else {
        sincos(x, s, c);
    }
}

constexpr int kTransformThreads = 128;
constexpr int kTransformPT = PSTD_TRANSFORM_PT;

// Cell records hold, for psi and for d psi/d a, the node values (quadrature weights and
// cell Jacobian folded in) regrouped over the mirrored Gauss-Legendre nodes
// s_{G-1-g} = -s_g.  With H = G/2, "+" = node g' (< H), "-" = node G-1-g', first sign for
// the fast in-plane axis b and second for c:
//   SS = P++ + P-+ + P+- + P--,  AA = P++ - P-+ - P+- + P--,
//   AS = P++ - P-+ + P+- - P--,  SA = P++ + P-+ - P+- - P--,
// so that sum_{g,h} e^{-i(u_g + v_h)} P[h][g]
//   = sum_{g',h'} [cos u cos v SS - sin u sin v AA - i (sin u cos v AS + cos u sin v SA)],
// u = beta_b s_g', v = beta_c s_h'.  Layout per cell: [h'][g'][psi: SS AA AS SA][dpsi: SS AA AS SA],
// eight contiguous complex values per node group (four 16-byte loads in single precision).
template <typename C, int H>
__device__ __forceinline__ void node_sum(const C* __restrict__ rec, const decltype(C::x)* cb, const decltype(C::x)* sb,
                                         const decltype(C::x)* cc, const decltype(C::x)* sc, C& ip_out, C& id_out)
{
    using R = decltype(C::x);
    // two interleaved accumulator sets (even / odd h') halve the dependent FMA chains
    C ipa[2] = {mk<C>(R(0), R(0)), mk<C>(R(0), R(0))}, ida[2] = {mk<C>(R(0), R(0)), mk<C>(R(0), R(0))};
#pragma unroll
    for (int h = 0; h < H; ++h) {
        C& ip = ipa[h & 1];
        C& id = ida[h & 1];
#pragma unroll
        for (int g = 0; g < H; ++g) {
            const R c_c = cb[g] * cc[h], s_s = sb[g] * sc[h], s_c = sb[g] * cc[h], c_s = cb[g] * sc[h];
            const C* r = rec + 8 * (h * H + g);
            C pSS, pAA, pAS, pSA, dSS, dAA, dAS, dSA;
            if constexpr (sizeof(R) == 4) {
                const float4* r4 = reinterpret_cast<const float4*>(r);
                const float4 a0 = r4[0], a1 = r4[1], a2 = r4[2], a3 = r4[3];
                pSS = mk<C>(a0.x, a0.y); pAA = mk<C>(a0.z, a0.w); pAS = mk<C>(a1.x, a1.y); pSA = mk<C>(a1.z, a1.w);
                dSS = mk<C>(a2.x, a2.y); dAA = mk<C>(a2.z, a2.w); dAS = mk<C>(a3.x, a3.y); dSA = mk<C>(a3.z, a3.w);
            } else {
                pSS = r[0]; pAA = r[1]; pAS = r[2]; pSA = r[3];
                dSS = r[4]; dAA = r[5]; dAS = r[6]; dSA = r[7];
            }
            ip.x += c_c * pSS.x - s_s * pAA.x + s_c * pAS.y + c_s * pSA.y;
            ip.y += c_c * pSS.y - s_s * pAA.y - s_c * pAS.x - c_s * pSA.x;
            id.x += c_c * dSS.x - s_s * dAA.x + s_c * dAS.y + c_s * dSA.y;
            id.y += c_c * dSS.y - s_s * dAA.y - s_c * dAS.x - c_s * dSA.x;
        }
    }
    ip_out = cadd(ip_out, cadd(ipa[0], ipa[1]));
    id_out = cadd(id_out, cadd(ida[0], ida[1]));
}

// blockIdx.z selects the member when several are transformed in one launch (a.members > 0:
// records [member][cell], wavenumbers a.km, partial sums [split][member][M]); PT points a thread.
template <typename R, int G, int PT = kTransformPT>
__global__ void __launch_bounds__(kTransformThreads) transform_kernel(const __grid_constant__ TransformArgs<R> a)
{
    using C = typename TransformArgs<R>::C;
    constexpr int H = G / 2;
    constexpr int REC = 2 * G * G;
    constexpr int CH = sizeof(R) == 4 ? 32 : 16;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* srec = reinterpret_cast<C*>(smraw);
    C* scen = srec + CH * REC;   // per-cell centre offsets of the chunk
    const int member = blockIdx.z;
    const C* __restrict__ rec = a.rec + (size_t)member * a.ncells * REC;
    const double k = a.members > 0 ? a.km[member] : a.k;

    long long pidx[PT];
    bool valid[PT];
    double px[PT], py[PT], pz[PT];
#pragma unroll
    for (int i = 0; i < PT; ++i) {
        pidx[i] = (long long)blockIdx.x * (kTransformThreads * PT) + i * kTransformThreads + threadIdx.x;
        valid[i] = pidx[i] < a.M;
        const long long p = valid[i] ? pidx[i] : 0;
        px[i] = a.pts[3 * p + 0]; py[i] = a.pts[3 * p + 1]; pz[i] = a.pts[3 * p + 2];
    }
    double accx[PT], accy[PT];
#pragma unroll
    for (int i = 0; i < PT; ++i) { accx[i] = 0.0; accy[i] = 0.0; }
    R node[H];
#pragma unroll
    for (int g = 0; g < H; ++g) node[g] = R(a.gl_node[g]);

    const long long c_begin = (long long)blockIdx.y * a.cells_per_split;
    const long long c_end = min(a.ncells, c_begin + a.cells_per_split);

    for (int fi = 0; fi < 6; ++fi) {
        const FaceGeom F = a.face[fi];
        const long long f_begin = max(c_begin, F.cell0);
        const long long f_end = min(c_end, F.cell0 + (long long)F.L * F.M);
        if (f_begin >= f_end) continue;
        // face centre (midpoint of the surface cells) as the reference point
        const double cbm = F.cb0 + 0.5 * (F.L - 1) * F.db;
        const double ccm = F.cc0 + 0.5 * (F.M - 1) * F.dc;
        const R hkb = R(0.5 * k * F.db), hkc = R(0.5 * k * F.dc);
        // per point: d0 = r - c0 (components along a, b, c), R0 and e^{ikR0}
        R d0a[PT], d0b[PT], d0c[PT];
        R R0[PT];
        C ph0[PT];
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            const double pa = F.axis == 0 ? px[i] : F.axis == 1 ? py[i] : pz[i];
            const double pb = F.b == 0 ? px[i] : F.b == 1 ? py[i] : pz[i];
            const double pc = F.c == 0 ? px[i] : F.c == 1 ? py[i] : pz[i];
            double s, c;
            const double da = pa - F.plane, db = pb - cbm, dc = pc - ccm;
            d0a[i] = R(da); d0b[i] = R(db); d0c[i] = R(dc);
            const double r0 = sqrt(da * da + db * db + dc * dc);
            R0[i] = R(r0);
            sincos(k * r0, &s, &c);
            ph0[i] = mk<C>(R(c), R(s));
        }
        const R kr = R(k);
        const R pref = R(-F.sigma / (4.0 * 3.14159265358979323846));
        C fsum[PT];
#pragma unroll
        for (int i = 0; i < PT; ++i) fsum[i] = mk<C>(R(0), R(0));

        for (long long cc0 = f_begin; cc0 < f_end; cc0 += CH) {
            const int nch = (int)min((long long)CH, f_end - cc0);
            __syncthreads();
            for (int e = threadIdx.x; e < nch * REC; e += kTransformThreads) srec[e] = rec[cc0 * REC + e];
            if (threadIdx.x < nch) {
                // cell centre minus face centre, once per cell of the chunk (double precision
                // and the index division stay out of the per-point loop)
                const long long local = cc0 + threadIdx.x - F.cell0;
                const int m = (int)(local / F.L), l = (int)(local - (long long)m * F.L);
                scen[threadIdx.x] = mk<C>(R((l - 0.5 * (F.L - 1)) * F.db), R((m - 0.5 * (F.M - 1)) * F.dc));
            }
            __syncthreads();
            for (int ci = 0; ci < nch; ++ci) {
                const C cen = scen[ci];
                const R dcb = cen.x, dcc = cen.y;
                const C* P = srec + ci * REC;
#pragma unroll
                for (int i = 0; i < PT; ++i) {
                    C ip = mk<C>(R(0), R(0)), id = mk<C>(R(0), R(0));
                    C w;               // e^{ikR}/R
                    R ha, cfr;         // bracket = Id + (cfr + i k) ha Ip
                    {
                        const R rb = d0b[i] - dcb, rc = d0c[i] - dcc, ra = d0a[i];
                        const R q = dcb * dcb + dcc * dcc - R(2) * (d0b[i] * dcb + d0c[i] * dcc);
                        const R R2 = ra * ra + rb * rb + rc * rc;
                        const R Rinv = sizeof(R) == 4 ? rsqrtf(float(R2)) : R(1) / sqrt(R2);
                        const R den = R2 * Rinv + R0[i];
                        R dR;
                        if constexpr (sizeof(R) == 4) dR = __fdividef(q, den);
                        else dR = q / den;
                        R s, c;
                        sincos_mid<R>(kr * dR, &s, &c);
                        w = cscale(cmul(ph0[i], mk<C>(c, s)), Rinv);
                        const R bb = hkb * rb * Rinv, bc = hkc * rc * Rinv;
                        R cb[H], sb[H], cc[H], sc[H];
#pragma unroll
                        for (int g = 0; g < H; ++g) {
                            sincos_small<R>(bb * node[g], &sb[g], &cb[g]);
                            sincos_small<R>(bc * node[g], &sc[g], &cc[g]);
                        }
                        node_sum<C, H>(P, cb, sb, cc, sc, ip, id);
                        ha = ra * Rinv;
                        cfr = -Rinv;
                    }
                    const C cf = mk<C>(cfr * ha, kr * ha);
                    const C br = cadd(id, cmul(cf, ip));
                    fsum[i] = cadd(fsum[i], cmul(w, br));
                }
            }
            // flush the chunk's partial sums into double accumulators
#pragma unroll
            for (int i = 0; i < PT; ++i) {
                accx[i] += double(pref * fsum[i].x);
                accy[i] += double(pref * fsum[i].y);
                fsum[i] = mk<C>(R(0), R(0));
            }
        }
    }
#pragma unroll
    for (int i = 0; i < PT; ++i)
        if (valid[i]) a.partial[((long long)blockIdx.y * gridDim.z + member) * a.M + pidx[i]] = make_double2(accx[i], accy[i]);
}

template <typename R, int G> cudaError_t transform_g(const TransformArgs<R>& a, int splits, cudaStream_t s)
{
    using C = typename TransformArgs<R>::C;
    constexpr int CH = sizeof(R) == 4 ? 32 : 16;
    const size_t sm = sizeof(C) * CH * (2 * G * G + 1);
    dim3 grid((unsigned)((a.M + kTransformThreads * kTransformPT - 1) / (kTransformThreads * kTransformPT)), splits,
              (unsigned)(a.members > 0 ? a.members : 1));
    transform_kernel<R, G><<<grid, kTransformThreads, sm, s>>>(a);
    return cudaGetLastError();
}

template <typename R> cudaError_t launch_transform(const TransformArgs<R>& a, int G, int splits, cudaStream_t s)
{
    switch (G) {
    case 4: return transform_g<R, 4>(a, splits, s);
    case 6: return transform_g<R, 6>(a, splits, s);
    case 8: return transform_g<R, 8>(a, splits, s);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------------
// far field from the plane spectra
// ---------------------------------------------------------------------------------
constexpr int kFarWarps = 8;       // warps of a far-field CTA; warp w takes far_dw() directions
// directions per warp: each spectrum value read from L1 serves far_dw() directions (8 in FP32;
// 4 in FP64, whose [i'][direction] factor table must fit shared memory at 384-point planes)
template <typename R> __host__ __device__ constexpr int far_dw() { return sizeof(R) == 4 ? 8 : 4; }
template <typename R> __host__ __device__ constexpr int far_dirs() { return kFarWarps * far_dw<R>(); }

template <typename C> __device__ __forceinline__ C warp_sum_c(C v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// n sinc(n phi / 2) e^{i psi}, phi = 2 pi m'/N - k rhat D, psi = k rhat L / 2 + phi (lo + n/2)
// (see the header).  psi is split as base + pi ((m' (2 lo + n)) mod 2N) / N with
// base = k rhat (L/2 - D (lo + n/2)) evaluated in double and reduced to [-pi, pi] once per
// direction and face, so the single-precision phase stays exact to rounding of O(1) values.
template <typename R, typename C>
__device__ __forceinline__ C face_factor(int m, int N, R krd, R base, int lo, int n)
{
    const int mp = m < (N + 1) / 2 ? m : m - N;          // index order -N/2..N/2-1
    const R phi = R(6.283185307179586476925286766559) * R(mp) / R(N) - krd;
    const R x = R(0.5) * R(n) * phi;
    R sx, cx;
    sincos_mid<R>(x, &sx, &cx);
    const R amp = fabs(x) < R(1e-6) ? R(n) : R(n) * sx / x;
    const int twoN = 2 * N;
    const int q = ((mp * (2 * lo + n)) % twoN + twoN) % twoN;
    R sp, cp;
    sincos_mid<R>(base + R(3.14159265358979323846) * R(q) / R(N), &sp, &cp);
    return mk<C>(amp * cp, amp * sp);
}

__device__ __forceinline__ double reduce_2pi(double x)
{
    return x - 6.283185307179586476925286766559 * rint(x * 0.15915494309189533576888376337251);
}

// One CTA takes DIRS = 8 DW directions through every face (face_split 1) or one face
// (face_split 6).  Per face, with at_{i'} of the CTA's directions in shared memory ([i'][d]),
// warp w forms for its DW directions d and lane l the column sums
//     T_q[d][j'] = sum_{i'} at_{i'}(d) C_q[i'][j'],   j' = j0 + l and j0 + 32 + l in the sweep
// of 64 columns from j0, q = psi and d psi
// (a register tile of DW directions by two columns: each spectrum value read serves DW
// directions, each at value, a broadcast read, four columns), then each sweep adds
// sum_j' bt_{j'}(d) T_q[d][j'] by a warp reduction to lane d's sums S_q[d].  FP32 sums over
// one face's spectrum; faces are added in double.
template <typename R>
__global__ void __launch_bounds__(kFarWarps * 32, sizeof(R) == 4 ? 2 : 1) farfield_kernel(const __grid_constant__ FarArgs<R> a)
{
    using C = typename FarArgs<R>::C;
    constexpr int DW = far_dw<R>(), DIRS = far_dirs<R>();
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sa = reinterpret_cast<C*>(smraw);                       // [Nb][DIRS]
    __shared__ double rh[DIRS][3];                             // direction unit vectors
    __shared__ R krd_s[2][DIRS], base_s[2][DIRS];              // face-factor arguments along b, c
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long p0 = (long long)blockIdx.x * DIRS;
    const double k = a.k;
    if (threadIdx.x < DIRS) {
        const long long p = p0 + threadIdx.x < a.M ? p0 + threadIdx.x : 0;
        double st, ct, sp, cp;
        sincos(a.theta[p], &st, &ct);
        sincos(a.phi[p], &sp, &cp);
        rh[threadIdx.x][0] = st * cp;
        rh[threadIdx.x][1] = st * sp;
        rh[threadIdx.x][2] = ct;
    }
    double tx = 0.0, ty = 0.0;                                 // lane dd < DW: direction DW w + dd
    const int f_first = a.face_split == 6 ? (int)blockIdx.y : 0;
    const int f_last = a.face_split == 6 ? (int)blockIdx.y + 1 : 6;
    for (int fi = f_first; fi < f_last; ++fi) {
        const FaceGeom F = a.face[fi];
        __syncthreads();   // rh written; the previous face's table and arguments no longer read
        if (threadIdx.x < DIRS) {
            const int d = threadIdx.x;
            const double rb = rh[d][F.b], rc = rh[d][F.c];
            krd_s[0][d] = R(k * rb * F.db);
            base_s[0][d] = R(reduce_2pi(k * rb * (0.5 * F.Nb * F.db - F.db * (F.lo_b + 0.5 * F.L))));
            krd_s[1][d] = R(k * rc * F.dc);
            base_s[1][d] = R(reduce_2pi(k * rc * (0.5 * F.Nc * F.dc - F.dc * (F.lo_c + 0.5 * F.M))));
        }
        __syncthreads();
        for (int e = threadIdx.x; e < F.Nb * DIRS; e += kFarWarps * 32) {
            const int d = e % DIRS, m = e / DIRS;
            sa[e] = face_factor<R, C>(m, F.Nb, krd_s[0][d], base_s[0][d], F.lo_b, F.L);
        }
        __syncthreads();
        const C* ctp = a.ct + a.ct_off[fi];                    // [q][m][j]
        const C* ctd = ctp + (long long)F.Nb * F.Nc;
        const C* arow = sa + DW * w;
        C sp_l = mk<C>(R(0), R(0)), sd_l = mk<C>(R(0), R(0)); // lane dd: direction DW w + dd, this face
        for (int j0 = 0; j0 < F.Nc; j0 += 64) {
            const int ja = j0 + lane, jb = ja + 32;
            const bool va = ja < F.Nc, vb = jb < F.Nc;
            const int la = va ? ja : 0, lb = vb ? jb : 0;      // columns past the plane read column 0, unused
            C tp[DW][2], td[DW][2];
#pragma unroll
            for (int dd = 0; dd < DW; ++dd)
#pragma unroll
                for (int t = 0; t < 2; ++t) { tp[dd][t] = mk<C>(R(0), R(0)); td[dd][t] = mk<C>(R(0), R(0)); }
#pragma unroll 1
            for (int m = 0; m < F.Nb; ++m) {
                const long long row = (long long)m * F.Nc;
                const C cpa = __ldg(ctp + row + la), cpb = __ldg(ctp + row + lb);
                const C cda = __ldg(ctd + row + la), cdb = __ldg(ctd + row + lb);
#pragma unroll
                for (int dd = 0; dd < DW; ++dd) {
                    const C av = arow[m * DIRS + dd];
                    tp[dd][0].x += av.x * cpa.x - av.y * cpa.y;
                    tp[dd][0].y += av.x * cpa.y + av.y * cpa.x;
                    tp[dd][1].x += av.x * cpb.x - av.y * cpb.y;
                    tp[dd][1].y += av.x * cpb.y + av.y * cpb.x;
                    td[dd][0].x += av.x * cda.x - av.y * cda.y;
                    td[dd][0].y += av.x * cda.y + av.y * cda.x;
                    td[dd][1].x += av.x * cdb.x - av.y * cdb.y;
                    td[dd][1].y += av.x * cdb.y + av.y * cdb.x;
                }
            }
#pragma unroll
            for (int dd = 0; dd < DW; ++dd) {
                const int d = DW * w + dd;
                C vp = mk<C>(R(0), R(0)), vd = mk<C>(R(0), R(0));
                if (va) {
                    const C bt = face_factor<R, C>(ja, F.Nc, krd_s[1][d], base_s[1][d], F.lo_c, F.M);
                    vp = cmul(bt, tp[dd][0]);
                    vd = cmul(bt, td[dd][0]);
                }
                if (vb) {
                    const C bt = face_factor<R, C>(jb, F.Nc, krd_s[1][d], base_s[1][d], F.lo_c, F.M);
                    vp = cadd(vp, cmul(bt, tp[dd][1]));
                    vd = cadd(vd, cmul(bt, td[dd][1]));
                }
                vp = warp_sum_c(vp);
                vd = warp_sum_c(vd);
                if (lane == dd) { sp_l = cadd(sp_l, vp); sd_l = cadd(sd_l, vd); }
            }
        }
        if (lane < DW) {
            const double ra = rh[DW * w + lane][F.axis];
            // -sigma D_b D_c / (4 pi) e^{-ik rhat_a a_plane} (S_d + i k rhat_a S_psi)
            double s0, c0;
            sincos(-k * ra * F.plane, &s0, &c0);
            const double spx = double(sp_l.x), spy = double(sp_l.y);
            const double bx = double(sd_l.x) - k * ra * spy, by = double(sd_l.y) + k * ra * spx;
            const double pref = -F.sigma * F.db * F.dc / (4.0 * 3.14159265358979323846);
            tx += pref * (c0 * bx - s0 * by);
            ty += pref * (c0 * by + s0 * bx);
        }
    }
    const long long p = p0 + DW * w + lane;
    if (lane < DW && p < a.M)
        a.partial[(long long)(a.face_split == 6 ? blockIdx.y : 0) * a.M + p] = make_double2(tx, ty);
}

template <typename R> cudaError_t launch_farfield(const FarArgs<R>& a, cudaStream_t s)
{
    using C = typename FarArgs<R>::C;
    int nbmax = 0;
    for (int f = 0; f < 6; ++f) nbmax = max(nbmax, a.face[f].Nb);
    const size_t sm = sizeof(C) * far_dirs<R>() * (size_t)nbmax;
    cudaError_t e = cudaFuncSetAttribute(farfield_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((a.M + far_dirs<R>() - 1) / far_dirs<R>()), a.face_split);
    farfield_kernel<R><<<grid, kFarWarps * 32, sm, s>>>(a);
    return cudaGetLastError();
}

template <typename R, typename C>
__global__ void spectrum_pack_kernel(const C* __restrict__ cp, const C* __restrict__ cd, int Nb, int Nc, R scale,
                                     C* __restrict__ ct)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)Nb * Nc;
    if (e >= n) return;
    const int j = (int)(e % Nc), m = (int)(e / Nc);          // output [m][j]
    const C vp = cp[(long long)j * Nb + m], vd = cd[(long long)j * Nb + m];
    ct[e] = mk<C>(vp.x * scale, vp.y * scale);
    ct[n + e] = mk<C>(vd.x * scale, vd.y * scale);
}

template <typename R>
cudaError_t launch_spectrum_pack(const typename std::conditional<sizeof(R) == 4, float2, double2>::type* c_psi,
                                 const typename std::conditional<sizeof(R) == 4, float2, double2>::type* c_dpsi,
                                 int Nb, int Nc, double scale,
                                 typename std::conditional<sizeof(R) == 4, float2, double2>::type* ct, cudaStream_t s)
{
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const long long n = (long long)Nb * Nc;
    spectrum_pack_kernel<R, C><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c_psi, c_dpsi, Nb, Nc, R(scale), ct);
    return cudaGetLastError();
}

template <typename R, typename C>
__global__ void pack_records_kernel(const C* __restrict__ op, const C* __restrict__ od, int L, int M, int G,
                                    const double* __restrict__ glw, double cw, long long cell0, C* __restrict__ rec)
{
    // one thread per (cell, h', g'); see the record layout above transform_kernel
    const int H = G / 2, HH = H * H;
    const long long total = (long long)L * M * HH;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int g = (int)(e % H);
    const int h = (int)((e / H) % H);
    const long long cell = e / HH;
    const int l = (int)(cell % L), m = (int)(cell / L);
    const long long ld = (long long)L * G;
    const int gp = g, gm = G - 1 - g, hp = h, hm = G - 1 - h;
    const R w = R(glw[g] * glw[h] * cw);   // mirrored nodes share their weights
    const long long r0 = (long long)m * G;
    const long long c0 = (long long)l * G;
    C* out = rec + (cell0 + cell) * (2LL * G * G) + 8 * (h * H + g);
    for (int q = 0; q < 2; ++q) {
        const C* src = q == 0 ? op : od;
        const C pp = src[(r0 + hp) * ld + c0 + gp], mp = src[(r0 + hp) * ld + c0 + gm];
        const C pm = src[(r0 + hm) * ld + c0 + gp], mm = src[(r0 + hm) * ld + c0 + gm];
        // first sign: node along b (g), second: node along c (h)
        const R ssx = pp.x + mp.x + pm.x + mm.x, ssy = pp.y + mp.y + pm.y + mm.y;
        const R aax = pp.x - mp.x - pm.x + mm.x, aay = pp.y - mp.y - pm.y + mm.y;
        const R asx = pp.x - mp.x + pm.x - mm.x, asy = pp.y - mp.y + pm.y - mm.y;
        const R sax = pp.x + mp.x - pm.x - mm.x, say = pp.y + mp.y - pm.y - mm.y;
        C* o = out + 4 * q;
        o[0] = mk<C>(ssx * w, ssy * w);
        o[1] = mk<C>(aax * w, aay * w);
        o[2] = mk<C>(asx * w, asy * w);
        o[3] = mk<C>(sax * w, say * w);
    }
}

template <typename R>
cudaError_t launch_pack_records(const typename std::conditional<sizeof(R) == 4, float2, double2>::type* out_psi,
                                const typename std::conditional<sizeof(R) == 4, float2, double2>::type* out_dpsi,
                                int L, int M, int G, const double* glw, double cw, long long cell0,
                                typename std::conditional<sizeof(R) == 4, float2, double2>::type* rec, cudaStream_t s)
{
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const long long total = (long long)L * M * (G / 2) * (G / 2);
    pack_records_kernel<R, C><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(out_psi, out_dpsi, L, M, G, glw, cw, cell0, rec);
    return cudaGetLastError();
}

}  // namespace pstd
