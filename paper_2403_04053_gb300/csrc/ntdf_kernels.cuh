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

constexpr int kTransformThreads = 128;
constexpr int kTransformPT = 2;   // points per thread

template <typename R, int G, bool FAR>
__global__ void __launch_bounds__(kTransformThreads) transform_kernel(TransformArgs<R> a)
{
    using C = typename TransformArgs<R>::C;
    constexpr int REC = 2 * G * G;
    constexpr int CH = sizeof(R) == 4 ? 32 : 16;
    constexpr int PT = kTransformPT;
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
        // per point: d0 = r - c0 (components along a, b, c), R0, e^{ikR0} (near) or
        // e^{-ik rhat . c0} (far), and the far-field in-plane phases at the nodes
        R d0a[PT], d0b[PT], d0c[PT];
        double R0[PT];
        C ph0[PT];
        C ef[PT][G], ff[PT][G];
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            const double pa = F.axis == 0 ? px[i] : F.axis == 1 ? py[i] : pz[i];
            const double pb = F.b == 0 ? px[i] : F.b == 1 ? py[i] : pz[i];
            const double pc = F.c == 0 ? px[i] : F.c == 1 ? py[i] : pz[i];
            double s, c;
            if (FAR) {
                d0a[i] = R(pa); d0b[i] = R(pb); d0c[i] = R(pc);
                R0[i] = 0.0;
                sincos(-k * (pa * F.plane + pb * cbm + pc * ccm), &s, &c);
                ph0[i] = mk<C>(R(c), R(s));
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    double sb, cb2, sc2, cc2;
                    sincos(-k * pb * 0.5 * F.db * a.gl_node[g], &sb, &cb2);
                    sincos(-k * pc * 0.5 * F.dc * a.gl_node[g], &sc2, &cc2);
                    ef[i][g] = mk<C>(R(cb2), R(sb));
                    ff[i][g] = mk<C>(R(cc2), R(sc2));
                }
            } else {
                const double da = pa - F.plane, db = pb - cbm, dc = pc - ccm;
                d0a[i] = R(da); d0b[i] = R(db); d0c[i] = R(dc);
                R0[i] = sqrt(da * da + db * db + dc * dc);
                sincos(k * R0[i], &s, &c);
                ph0[i] = mk<C>(R(c), R(s));
            }
        }
        const R kr = R(k);
        const R pref = R(-F.sigma / (4.0 * 3.14159265358979323846));
        C fsum[PT];
#pragma unroll
        for (int i = 0; i < PT; ++i) fsum[i] = mk<C>(R(0), R(0));

        for (long long cc = f_begin; cc < f_end; cc += CH) {
            const int nch = (int)min((long long)CH, f_end - cc);
            __syncthreads();
            for (int e = threadIdx.x; e < nch * REC; e += kTransformThreads) srec[e] = a.rec[cc * REC + e];
            __syncthreads();
            for (int ci = 0; ci < nch; ++ci) {
                const long long local = cc + ci - F.cell0;
                const int m = (int)(local / F.L), l = (int)(local - (long long)m * F.L);
                const R dcb = R((l - 0.5 * (F.L - 1)) * F.db);   // cell centre minus face centre
                const R dcc = R((m - 0.5 * (F.M - 1)) * F.dc);
                const C* P = srec + ci * REC;
                const C* D = P + G * G;
#pragma unroll
                for (int i = 0; i < PT; ++i) {
                    C eb[G], fc[G];
                    C w;               // e^{ikR}/R (near) or e^{-ik rhat . r_c} (far)
                    R ha, cfac_re, cfac_im;   // bracket: Id + (cfac) ha Ip
                    if (FAR) {
                        R s, c;
                        const R arg = -kr * (d0b[i] * dcb + d0c[i] * dcc);
                        sincos_r<R>(arg, &s, &c);
                        w = cmul(ph0[i], mk<C>(c, s));
#pragma unroll
                        for (int g = 0; g < G; ++g) { eb[g] = ef[i][g]; fc[g] = ff[i][g]; }
                        ha = d0a[i];
                        cfac_re = R(0); cfac_im = kr;
                    } else {
                        const R rb = d0b[i] - dcb, rc = d0c[i] - dcc, ra = d0a[i];
                        const R q = dcb * dcb + dcc * dcc - R(2) * (d0b[i] * dcb + d0c[i] * dcc);
                        const R R2 = ra * ra + rb * rb + rc * rc;
                        const R Rinv = sizeof(R) == 4 ? rsqrtf(float(R2)) : R(1) / sqrt(R2);
                        const R Rr = R2 * Rinv;
                        const R dR = q / (Rr + R(R0[i]));
                        R s, c;
                        sincos_r<R>(kr * dR, &s, &c);
                        w = cscale(cmul(ph0[i], mk<C>(c, s)), Rinv);
                        const R hb = rb * Rinv, hc = rc * Rinv;
                        ha = ra * Rinv;
                        cfac_re = -Rinv; cfac_im = kr;
#pragma unroll
                        for (int g = 0; g < G / 2; ++g) {
                            R sb, cb, sc, cc2;
                            sincos_r<R>(-kr * hb * R(0.5 * F.db * a.gl_node[g]), &sb, &cb);
                            sincos_r<R>(-kr * hc * R(0.5 * F.dc * a.gl_node[g]), &sc, &cc2);
                            eb[g] = mk<C>(cb, sb);
                            eb[G - 1 - g] = mk<C>(cb, -sb);    // symmetric nodes: s_{G-1-g} = -s_g
                            fc[g] = mk<C>(cc2, sc);
                            fc[G - 1 - g] = mk<C>(cc2, -sc);
                        }
                    }
                    C ip = mk<C>(R(0), R(0)), id = mk<C>(R(0), R(0));
#pragma unroll
                    for (int h = 0; h < G; ++h) {
                        C tp = mk<C>(R(0), R(0)), td = mk<C>(R(0), R(0));
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            const C pv = P[h * G + g], dv = D[h * G + g];
                            tp.x += eb[g].x * pv.x - eb[g].y * pv.y; tp.y += eb[g].x * pv.y + eb[g].y * pv.x;
                            td.x += eb[g].x * dv.x - eb[g].y * dv.y; td.y += eb[g].x * dv.y + eb[g].y * dv.x;
                        }
                        ip = cadd(ip, cmul(fc[h], tp));
                        id = cadd(id, cmul(fc[h], td));
                    }
                    // bracket = Id + (cfac_re + i cfac_im) ha Ip
                    const C cf = mk<C>(cfac_re * ha, cfac_im * ha);
                    const C br = cadd(id, cmul(cf, ip));
                    fsum[i] = cadd(fsum[i], cmul(w, br));
                }
            }
            // flush the chunk's single-precision partial sums into double accumulators
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
    dim3 grid((unsigned)((a.M + kTransformThreads * kTransformPT - 1) / (kTransformThreads * kTransformPT)), splits);
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
    const long long total = (long long)L * M * G * G;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int g = (int)(e % G);
    const int h = (int)((e / G) % G);
    const long long cell = e / (G * G);
    const int l = (int)(cell % L), m = (int)(cell / L);
    const long long src = ((long long)m * G + h) * ((long long)L * G) + (long long)l * G + g;
    const double w = glw[g] * glw[h] * cw;
    const long long dst = (cell0 + cell) * (2LL * G * G) + h * G + g;
    rec[dst] = mk<C>(R(op[src].x * w), R(op[src].y * w));
    rec[dst + G * G] = mk<C>(R(od[src].x * w), R(od[src].y * w));
}

template <typename R>
cudaError_t launch_pack_records(const double2* out_psi, const double2* out_dpsi, int L, int M, int G, const double* glw,
                                double cw, long long cell0,
                                typename std::conditional<sizeof(R) == 4, float2, double2>::type* rec, cudaStream_t s)
{
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const long long total = (long long)L * M * G * G;
    pack_records_kernel<R, C><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(out_psi, out_dpsi, L, M, G, glw, cw, cell0, rec);
    return cudaGetLastError();
}

}  // namespace pstd
