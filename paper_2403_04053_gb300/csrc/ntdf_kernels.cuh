// Near-to-distant-field transform (Section 3): per surface cell, the integral of the
// trigonometric interpolant psi_an (Eq. AnBottomPsi) times the linearised Green's
// phase e^{-ik Rhat . dr'} (the approximation behind Eqs. bottomPsi_lm ... leftrightPsi_ln),
//
//   Psi_cell(r) = -sigma/(4 pi) e^{ikR}/R  int_cell [d_a psi_an + (ik - 1/R) Rhat_a psi_an] e^{-ik Rhat . dr'} dS',
//
// summed over the cells of the six faces (Eq. Psi).  Each cell integral is a G x G
// Gauss-Legendre sum over node values prepared once per (member, frequency)
// ("records", weights and the cell Jacobian folded in); the in-plane phase at the
// nodes factors into e_g(axis b) f_h(axis c).  The distance is split as
// R = R0 + dR, R0 = |r - face centre| in double precision and
// dR = (|dc|^2 - 2 d0 . dc) / (R + R0) in the working precision, so single-precision
// phases stay accurate at kR ~ 10^3.  Far field: e^{ikR}/R -> e^{-ik rhat . r_c} and
// Rhat -> rhat, (ik - 1/R) -> ik.
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
// observation points per thread: near field 1 (keeps registers low enough for 4 resident
// CTAs), far field 2 (the node phases are per point and face, so records are reused)
template <bool FAR> __host__ __device__ constexpr int transform_pt() { return FAR ? 2 : 1; }

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

template <typename R, int G, bool FAR>
__global__ void __launch_bounds__(kTransformThreads) transform_kernel(TransformArgs<R> a)
{
    using C = typename TransformArgs<R>::C;
    constexpr int H = G / 2;
    constexpr int REC = 2 * G * G;
    constexpr int CH = sizeof(R) == 4 ? 32 : 16;
    constexpr int PT = transform_pt<FAR>();
    extern __shared__ __align__(16) unsigned char smraw[];
    C* srec = reinterpret_cast<C*>(smraw);
    const double k = a.k;

    long long pidx[PT];
    bool valid[PT];
    double px[PT], py[PT], pz[PT];
#pragma unroll
    for (int i = 0; i < PT; ++i) {
        pidx[i] = (long long)blockIdx.x * (kTransformThreads * PT) + i * kTransformThreads + threadIdx.x;
        valid[i] = pidx[i] < a.M;
        const long long p = valid[i] ? pidx[i] : 0;
        if (FAR) {
            double st, ct, sp, cp;
            sincos(a.theta[p], &st, &ct);
            sincos(a.phi[p], &sp, &cp);
            px[i] = st * cp; py[i] = st * sp; pz[i] = ct;
        } else {
            px[i] = a.pts[3 * p + 0]; py[i] = a.pts[3 * p + 1]; pz[i] = a.pts[3 * p + 2];
        }
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
        // per point: d0 = r - c0 (components along a, b, c) and R0, e^{ikR0} (near), or the
        // direction, e^{-ik rhat . c0} and the node phases (far: the same for every cell)
        R d0a[PT], d0b[PT], d0c[PT];
        R R0[PT];
        C ph0[PT];
        R fcb[PT][H], fsb[PT][H], fcc[PT][H], fsc[PT][H];
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            const double pa = F.axis == 0 ? px[i] : F.axis == 1 ? py[i] : pz[i];
            const double pb = F.b == 0 ? px[i] : F.b == 1 ? py[i] : pz[i];
            const double pc = F.c == 0 ? px[i] : F.c == 1 ? py[i] : pz[i];
            double s, c;
            if (FAR) {
                d0a[i] = R(pa); d0b[i] = R(pb); d0c[i] = R(pc);
                R0[i] = R(0);
                sincos(-k * (pa * F.plane + pb * cbm + pc * ccm), &s, &c);
                ph0[i] = mk<C>(R(c), R(s));
#pragma unroll
                for (int g = 0; g < H; ++g) {
                    sincos_small<R>(hkb * d0b[i] * node[g], &fsb[i][g], &fcb[i][g]);
                    sincos_small<R>(hkc * d0c[i] * node[g], &fsc[i][g], &fcc[i][g]);
                }
            } else {
                const double da = pa - F.plane, db = pb - cbm, dc = pc - ccm;
                d0a[i] = R(da); d0b[i] = R(db); d0c[i] = R(dc);
                const double r0 = sqrt(da * da + db * db + dc * dc);
                R0[i] = R(r0);
                sincos(k * r0, &s, &c);
                ph0[i] = mk<C>(R(c), R(s));
            }
        }
        const R kr = R(k);
        const R pref = R(-F.sigma / (4.0 * 3.14159265358979323846));
        C fsum[PT];
#pragma unroll
        for (int i = 0; i < PT; ++i) fsum[i] = mk<C>(R(0), R(0));

        for (long long cc0 = f_begin; cc0 < f_end; cc0 += CH) {
            const int nch = (int)min((long long)CH, f_end - cc0);
            __syncthreads();
            for (int e = threadIdx.x; e < nch * REC; e += kTransformThreads) srec[e] = a.rec[cc0 * REC + e];
            __syncthreads();
            for (int ci = 0; ci < nch; ++ci) {
                const long long local = cc0 + ci - F.cell0;
                const int m = (int)(local / F.L), l = (int)(local - (long long)m * F.L);
                const R dcb = R((l - 0.5 * (F.L - 1)) * F.db);   // cell centre minus face centre
                const R dcc = R((m - 0.5 * (F.M - 1)) * F.dc);
                const C* P = srec + ci * REC;
#pragma unroll
                for (int i = 0; i < PT; ++i) {
                    C ip = mk<C>(R(0), R(0)), id = mk<C>(R(0), R(0));
                    C w;               // e^{ikR}/R (near) or e^{-ik rhat . r_c} (far)
                    R ha, cfr;         // bracket = Id + (cfr + i k) ha Ip
                    if (FAR) {
                        R s, c;
                        sincos_mid<R>(-kr * (d0b[i] * dcb + d0c[i] * dcc), &s, &c);
                        w = cmul(ph0[i], mk<C>(c, s));
                        node_sum<C, H>(P, fcb[i], fsb[i], fcc[i], fsc[i], ip, id);
                        ha = d0a[i];
                        cfr = R(0);
                    } else {
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
        if (valid[i]) a.partial[(long long)blockIdx.y * a.M + pidx[i]] = make_double2(accx[i], accy[i]);
}

template <typename R, int G> cudaError_t transform_g(const TransformArgs<R>& a, int splits, bool far, cudaStream_t s)
{
    using C = typename TransformArgs<R>::C;
    constexpr int CH = sizeof(R) == 4 ? 32 : 16;
    const size_t sm = sizeof(C) * CH * 2 * G * G;
    const int pt = far ? transform_pt<true>() : transform_pt<false>();
    dim3 grid((unsigned)((a.M + kTransformThreads * pt - 1) / (kTransformThreads * pt)), splits);
    if (far) {
        cudaError_t e = cudaFuncSetAttribute(transform_kernel<R, G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        transform_kernel<R, G, true><<<grid, kTransformThreads, sm, s>>>(a);
    } else {
        cudaError_t e = cudaFuncSetAttribute(transform_kernel<R, G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        transform_kernel<R, G, false><<<grid, kTransformThreads, sm, s>>>(a);
    }
    return cudaGetLastError();
}

template <typename R> cudaError_t launch_transform(const TransformArgs<R>& a, int G, int splits, bool far, cudaStream_t s)
{
    switch (G) {
    case 6: return transform_g<R, 6>(a, splits, far, s);
    case 8: return transform_g<R, 8>(a, splits, far, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename R, typename C>
__global__ void pack_records_kernel(const double2* __restrict__ op, const double2* __restrict__ od, int L, int M, int G,
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
    const double w = glw[g] * glw[h] * cw;   // mirrored nodes share their weights
    const long long r0 = (long long)m * G;
    const long long c0 = (long long)l * G;
    C* out = rec + (cell0 + cell) * (2LL * G * G) + 8 * (h * H + g);
    for (int q = 0; q < 2; ++q) {
        const double2* src = q == 0 ? op : od;
        const double2 pp = src[(r0 + hp) * ld + c0 + gp], mp = src[(r0 + hp) * ld + c0 + gm];
        const double2 pm = src[(r0 + hm) * ld + c0 + gp], mm = src[(r0 + hm) * ld + c0 + gm];
        // first sign: node along b (g), second: node along c (h)
        const double ssx = pp.x + mp.x + pm.x + mm.x, ssy = pp.y + mp.y + pm.y + mm.y;
        const double aax = pp.x - mp.x - pm.x + mm.x, aay = pp.y - mp.y - pm.y + mm.y;
        const double asx = pp.x - mp.x + pm.x - mm.x, asy = pp.y - mp.y + pm.y - mm.y;
        const double sax = pp.x + mp.x - pm.x - mm.x, say = pp.y + mp.y - pm.y - mm.y;
        C* o = out + 4 * q;
        o[0] = mk<C>(R(ssx * w), R(ssy * w));
        o[1] = mk<C>(R(aax * w), R(aay * w));
        o[2] = mk<C>(R(asx * w), R(asy * w));
        o[3] = mk<C>(R(sax * w), R(say * w));
    }
}

template <typename R>
cudaError_t launch_pack_records(const double2* out_psi, const double2* out_dpsi, int L, int M, int G, const double* glw,
                                double cw, long long cell0,
                                typename std::conditional<sizeof(R) == 4, float2, double2>::type* rec, cudaStream_t s)
{
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const long long total = (long long)L * M * (G / 2) * (G / 2);
    pack_records_kernel<R, C><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(out_psi, out_dpsi, L, M, G, glw, cw, cell0, rec);
    return cudaGetLastError();
}

}  // namespace pstd
