// Discrete adjoint of the PSTD run and of the surface transform (no counterpart in the
// paper: the transposes of the forward kernels, for gradients with respect to V).
//
// Convention: for a real loss L and complex z, g_z = dL/dRe z + i dL/dIm z, so a
// complex-linear map y = M z pulls back as g_z = M^H g_y.  The leapfrog
// u^{n+1} = Gamma [u^{n-1} + A u^n + b^n], A = -(2 i dt / hbar)(eta hbar^2/2m K + V)
// (K real symmetric, Gamma and V real diagonal) has the adjoint recursion
// mu^n = Gamma [mu^{n+2} + A^H mu^{n+1} + o^n]; its complex conjugate nu = conj(mu) obeys
//     nu^n = Gamma [nu^{n+2} + A nu^{n+1} + conj(o^n)],
// the forward update itself with no incident wave, so the step kernels run it unchanged.
// The observation term conj(o^n) = sum_f (e^{i w_f t_n} / S_f) E^T conj(g_{P_f}) is built
// once per frequency as a volume J_f (injection_kernel) and added on the DFT-window steps
// (inject_kernel); dL/dV_j = (2 dt / hbar) sum_n Im[nu^{n+1}_j (u^n_j + psi_inc^n_j)]
// (grad_kernel; without psi_inc in the PAPER form).
#pragma once

#include <type_traits>

#include "fft_line.cuh"
#include "ntdf_kernels.cuh"
#include "pstd_internal.h"
#include "step_kernels.cuh"

namespace pstd {

// ---------------------------------------------------------------------------------
// J = scale * E^T conj(g): for every node, the plane values where it lies on a plane
// and D_h(q) times the normal-derivative plane value along every normal line.
// ---------------------------------------------------------------------------------
template <typename R>
__global__ void injection_kernel(const __grid_constant__ InjectionArgs<R> a)
{
    using C = typename InjectionArgs<R>::C;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.ncell) return;
    const int x = (int)(e % a.n[0]);
    const int y = (int)((e / a.n[0]) % a.n[1]);
    const int z = (int)(e / ((long long)a.n[0] * a.n[1]));
    const int pos[3] = {x, y, z};
    // in-plane pixel of the node on the planes normal to each axis: [c][b]
    const long long pix[3] = {(long long)z * a.n[1] + y, (long long)z * a.n[0] + x, (long long)y * a.n[0] + x};
    double sx = 0.0, sy = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        const int q = pos[ax];
        for (int side = 0; side < 2; ++side) {
            const int f = 2 * ax + side;
            const double2 gp = a.g[a.face_off[f] + pix[ax]];
            const double2 gd = a.g[a.face_off[f] + a.face_size[f] + pix[ax]];
            // conj(g_psi) on the plane itself
            if (q == a.h[ax][side]) { sx += gp.x; sy -= gp.y; }
            // D_h(q) conj(g_dpsi) along the normal line
            const C w = a.dw[ax][side * a.n[ax] + q];
            const double wx = double(w.x), wy = double(w.y);
            sx += wx * gd.x + wy * gd.y;
            sy += wy * gd.x - wx * gd.y;
        }
    }
    a.J[e] = mk<C>(R(sx * a.scale.x - sy * a.scale.y), R(sx * a.scale.y + sy * a.scale.x));
}

// prev += coef * J over one member's state
template <typename R, typename C>
__global__ void inject_kernel(C* __restrict__ prev, const C* __restrict__ J, C coef, long long n)
{
    step_kernel_entry();
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const C j = J[e], p = prev[e];
    prev[e] = mk<C>(p.x + coef.x * j.x - coef.y * j.y, p.y + coef.x * j.y + coef.y * j.x);
}

// grad[box] += (2 dt / hbar) sum_b Im[nu_b (u_b + s_b phase_b)] on the box [lo, hi) (x
// fastest): the members share V, so their contributions add
template <typename R>
__global__ void grad_kernel(const __grid_constant__ GradArgs<R> a)
{
    using C = typename GradArgs<R>::C;
    step_kernel_entry();
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int bx = a.hi[0] - a.lo[0], by = a.hi[1] - a.lo[1], bz = a.hi[2] - a.lo[2];
    if (e >= (long long)bx * by * bz) return;
    const int x = a.lo[0] + (int)(e % bx);
    const int y = a.lo[1] + (int)((e / bx) % by);
    const int z = a.lo[2] + (int)(e / ((long long)bx * by));
    const long long idx = ((long long)z * a.ny + y) * a.nx + x;
    double acc = 0.0;
    for (int b = 0; b < a.batch; ++b) {
        const C nu = a.nu[b * a.ncell + idx];
        C u = a.u[b * a.ncell + idx];
        if (a.with_inc) {
            const C p = cmul(cmul(cmul(a.s[b], a.phase[0][b * a.nx + x]), a.phase[1][b * a.ny + y]), a.phase[2][b * a.nz + z]);
            u = cadd(u, p);
        }
        acc += double(nu.x) * double(u.y) + double(nu.y) * double(u.x);
    }
    a.grad[e] += a.c2 * acc;
}

// ---------------------------------------------------------------------------------
// transform adjoint: records' gradient from the points' gradient (transpose of
// transform_kernel; see the record layout above node_sum)
// ---------------------------------------------------------------------------------
template <typename R>
__global__ void adj_points_kernel(const __grid_constant__ AdjointTransformArgs<R> a)
{
    // per (face, point): d0 = r - face centre (a, b, c), R0 = |d0|, A = pref conj(e^{ikR0}) g_p
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 6 * a.M) return;
    const int fi = (int)(e / a.M);
    const long long p = e - (long long)fi * a.M;
    const FaceGeom& F = a.face[fi];
    const double r[3] = {a.pts[3 * p], a.pts[3 * p + 1], a.pts[3 * p + 2]};
    const double cbm = F.cb0 + 0.5 * (F.L - 1) * F.db;
    const double ccm = F.cc0 + 0.5 * (F.M - 1) * F.dc;
    const double da = r[F.axis] - F.plane, db = r[F.b] - cbm, dc = r[F.c] - ccm;
    const double r0 = sqrt(da * da + db * db + dc * dc);
    double s, c;
    sincos(a.k * r0, &s, &c);
    const double pref = -F.sigma / (4.0 * 3.14159265358979323846);
    const double2 g = a.gpts[p];
    // conj(e^{ikR0}) g = (c - i s)(gx + i gy)
    const double ax = pref * (c * g.x + s * g.y), ay = pref * (c * g.y - s * g.x);
    AdjPoint<R> q;
    q.d0a = R(da); q.d0b = R(db); q.d0c = R(dc); q.R0 = R(r0); q.ax = R(ax); q.ay = R(ay);
    a.table[e] = q;
}

constexpr int kAdjThreads = 128;

template <typename R, int G>
__global__ void __launch_bounds__(kAdjThreads) transform_adjoint_kernel(const __grid_constant__ AdjointTransformArgs<R> a)
{
    using C = typename AdjointTransformArgs<R>::C;
    constexpr int H = G / 2;
    constexpr int REC = 2 * G * G;
    __shared__ AdjPoint<R> sp[kAdjThreads];
    const int fi = blockIdx.z;
    const FaceGeom& F = a.face[fi];
    const long long items = (long long)F.L * F.M * H;
    const long long item = (long long)blockIdx.x * kAdjThreads + threadIdx.x;
    if ((long long)blockIdx.x * kAdjThreads >= items) return;   // whole CTA beyond this face
    const bool act = item < items;
    const long long cell = act ? item / H : 0;
    const int hq = act ? (int)(item % H) : 0;                    // this thread's mirrored-node row h'
    const int l = (int)(cell % F.L), m = (int)(cell / F.L);
    const R dcb = R((l - 0.5 * (F.L - 1)) * F.db), dcc = R((m - 0.5 * (F.M - 1)) * F.dc);
    const R kr = R(a.k);
    const R hkb = R(0.5 * a.k * F.db), hkc = R(0.5 * a.k * F.dc);
    R node[H];
#pragma unroll
    for (int g = 0; g < H; ++g) node[g] = R(a.gl_node[g]);
    const R nodeh = R(a.gl_node[hq]);
    C accp[H][4], accd[H][4];
#pragma unroll
    for (int g = 0; g < H; ++g)
#pragma unroll
        for (int t = 0; t < 4; ++t) { accp[g][t] = mk<C>(R(0), R(0)); accd[g][t] = mk<C>(R(0), R(0)); }

    const long long p_begin = (long long)blockIdx.y * a.points_per_split;
    const long long p_end = min(a.M, p_begin + a.points_per_split);
    const AdjPoint<R>* tab = a.table + (long long)fi * a.M;
    for (long long p0 = p_begin; p0 < p_end; p0 += kAdjThreads) {
        const int np = (int)min((long long)kAdjThreads, p_end - p0);
        __syncthreads();
        if (threadIdx.x < np) sp[threadIdx.x] = tab[p0 + threadIdx.x];
        __syncthreads();
        if (!act) continue;
        for (int i = 0; i < np; ++i) {
            const AdjPoint<R> P = sp[i];
            const R rb = P.d0b - dcb, rc = P.d0c - dcc, ra = P.d0a;
            const R q = dcb * dcb + dcc * dcc - R(2) * (P.d0b * dcb + P.d0c * dcc);
            const R R2 = ra * ra + rb * rb + rc * rc;
            const R Rinv = sizeof(R) == 4 ? rsqrtf(float(R2)) : R(1) / sqrt(R2);
            const R den = R2 * Rinv + P.R0;
            R dR;
            if constexpr (sizeof(R) == 4) dR = __fdividef(q, den);
            else dR = q / den;
            R s, c;
            sincos_mid<R>(kr * dR, &s, &c);
            // Z = A conj(e^{ik dR}) / R  (gradient weight of the dpsi records)
            const C Z = mk<C>((P.ax * c + P.ay * s) * Rinv, (P.ay * c - P.ax * s) * Rinv);
            // Zp = conj(cf) Z with cf = (-1/R + i k) Rhat_a  (weight of the psi records)
            const R ha = ra * Rinv;
            const R cfr = -Rinv * ha, cfi = -kr * ha;   // conj(cf) = cfr + i cfi
            const C Zp = mk<C>(cfr * Z.x - cfi * Z.y, cfr * Z.y + cfi * Z.x);
            const R bb = hkb * rb * Rinv, bc = hkc * rc * Rinv;
            R sc, cc;
            sincos_small<R>(bc * nodeh, &sc, &cc);
#pragma unroll
            for (int g = 0; g < H; ++g) {
                R sb, cb;
                sincos_small<R>(bb * node[g], &sb, &cb);
                const R c_c = cb * cc, s_s = sb * sc, s_c = sb * cc, c_s = cb * sc;
                // forward: c_c SS - s_s AA - i s_c AS - i c_s SA; adjoint: conj(coefficient) * Z
                accp[g][0].x += c_c * Zp.x;  accp[g][0].y += c_c * Zp.y;
                accp[g][1].x -= s_s * Zp.x;  accp[g][1].y -= s_s * Zp.y;
                accp[g][2].x -= s_c * Zp.y;  accp[g][2].y += s_c * Zp.x;
                accp[g][3].x -= c_s * Zp.y;  accp[g][3].y += c_s * Zp.x;
                accd[g][0].x += c_c * Z.x;   accd[g][0].y += c_c * Z.y;
                accd[g][1].x -= s_s * Z.x;   accd[g][1].y -= s_s * Z.y;
                accd[g][2].x -= s_c * Z.y;   accd[g][2].y += s_c * Z.x;
                accd[g][3].x -= c_s * Z.y;   accd[g][3].y += c_s * Z.x;
            }
        }
    }
    if (!act) return;
    C* out = a.partial + ((long long)blockIdx.y * a.ncells + F.cell0 + cell) * REC + 8 * (hq * H);
#pragma unroll
    for (int g = 0; g < H; ++g)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            out[8 * g + t] = accp[g][t];
            out[8 * g + 4 + t] = accd[g][t];
        }
}

// sum the per-split record gradients: rec[i] = sum_s partial[s][i]
template <typename C>
__global__ void sum_splits_kernel(const C* __restrict__ partial, int splits, long long n, C* __restrict__ rec)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    C s = partial[e];
    for (int k = 1; k < splits; ++k) s = cadd(s, partial[(long long)k * n + e]);
    rec[e] = s;
}

// transpose of pack_records_kernel: node-value gradients from record gradients
template <typename R, typename C>
__global__ void unpack_records_kernel(const C* __restrict__ rec, int L, int M, int G, const double* __restrict__ glw,
                                      double cw, long long cell0, C* __restrict__ op, C* __restrict__ od)
{
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
    const R w = R(glw[g] * glw[h] * cw);
    const long long r0 = (long long)m * G;
    const long long c0 = (long long)l * G;
    const C* in = rec + (cell0 + cell) * (2LL * G * G) + 8 * (h * H + g);
    for (int q = 0; q < 2; ++q) {
        const C* r = in + 4 * q;
        const C SS = r[0], AA = r[1], AS = r[2], SA = r[3];
        C* dst = q == 0 ? op : od;
        dst[(r0 + hp) * ld + c0 + gp] = mk<C>(w * (SS.x + AA.x + AS.x + SA.x), w * (SS.y + AA.y + AS.y + SA.y));
        dst[(r0 + hp) * ld + c0 + gm] = mk<C>(w * (SS.x - AA.x - AS.x + SA.x), w * (SS.y - AA.y - AS.y + SA.y));
        dst[(r0 + hm) * ld + c0 + gp] = mk<C>(w * (SS.x - AA.x + AS.x - SA.x), w * (SS.y - AA.y + AS.y - SA.y));
        dst[(r0 + hm) * ld + c0 + gm] = mk<C>(w * (SS.x + AA.x - AS.x - SA.x), w * (SS.y + AA.y - AS.y - SA.y));
    }
}

// widen a working-precision array into double2
template <typename C>
__global__ void widen_kernel(const C* __restrict__ in, double2* __restrict__ out, long long n)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    out[e] = make_double2(double(in[e].x), double(in[e].y));
}

// ---------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------
template <typename R> cudaError_t launch_injection(const InjectionArgs<R>& a, cudaStream_t s)
{
    injection_kernel<R><<<(unsigned)((a.ncell + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_inject(typename std::conditional<sizeof(R) == 4, float2, double2>::type* prev,
                          const typename std::conditional<sizeof(R) == 4, float2, double2>::type* J,
                          typename std::conditional<sizeof(R) == 4, float2, double2>::type coef, long long n, cudaStream_t s)
{
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    return launch_step_kernel(inject_kernel<R, C>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, prev, J, coef, n);
}

template <typename R> cudaError_t launch_grad(const GradArgs<R>& a, cudaStream_t s)
{
    const long long n = (long long)(a.hi[0] - a.lo[0]) * (a.hi[1] - a.lo[1]) * (a.hi[2] - a.lo[2]);
    if (n <= 0) return cudaSuccess;
    return launch_step_kernel(grad_kernel<R>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, a);
}

template <typename R> cudaError_t launch_adj_points(const AdjointTransformArgs<R>& a, cudaStream_t s)
{
    const long long n = 6 * a.M;
    adj_points_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename R, int G> cudaError_t transform_adjoint_g(const AdjointTransformArgs<R>& a, int splits, cudaStream_t s)
{
    long long maxitems = 0;
    for (int f = 0; f < 6; ++f) maxitems = max(maxitems, (long long)a.face[f].L * a.face[f].M * (G / 2));
    const dim3 grid((unsigned)((maxitems + kAdjThreads - 1) / kAdjThreads), splits, 6);
    transform_adjoint_kernel<R, G><<<grid, kAdjThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename R> cudaError_t launch_transform_adjoint(const AdjointTransformArgs<R>& a, int G, int splits, cudaStream_t s)
{
    switch (G) {
    case 4: return transform_adjoint_g<R, 4>(a, splits, s);
    case 6: return transform_adjoint_g<R, 6>(a, splits, s);
    case 8: return transform_adjoint_g<R, 8>(a, splits, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename R>
cudaError_t launch_sum_splits(const typename std::conditional<sizeof(R) == 4, float2, double2>::type* partial, int splits,
                              long long n, typename std::conditional<sizeof(R) == 4, float2, double2>::type* rec,
                              cudaStream_t s)
{
    sum_splits_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(partial, splits, n, rec);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_unpack_records(const typename std::conditional<sizeof(R) == 4, float2, double2>::type* rec, int L, int M,
                                  int G, const double* glw, double cw, long long cell0,
                                  typename std::conditional<sizeof(R) == 4, float2, double2>::type* op,
                                  typename std::conditional<sizeof(R) == 4, float2, double2>::type* od, cudaStream_t s)
{
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const long long total = (long long)L * M * (G / 2) * (G / 2);
    unpack_records_kernel<R, C><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(rec, L, M, G, glw, cw, cell0, op, od);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_widen(const typename std::conditional<sizeof(R) == 4, float2, double2>::type* in, double2* out,
                         long long n, cudaStream_t s)
{
    widen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

}  // namespace pstd
