// Internal declarations shared by the C ABI (api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <type_traits>
#include <vector>

#include "pstd.h"

namespace pstd {

// Per-member constants read by the kernels (device array, uploaded by pstd_set_incidence).
struct MemberDev {
    double w0;      // E / hbar of the incident wave
    double ramp;    // raised-cosine switch-on time
    double eta;     // sinc(E dt / hbar), Eq. numdis2
    double k[3];    // wave vector k * khat
    double omega[PSTD_MAX_FREQ];   // DFT angular frequencies
    int nfreq;
    int packet;     // incident Gaussian wave packet (else CW)
    double khat[3]; // unit incidence direction (the 1-D auxiliary wave's d axis)
    int dft_active; // set per step by the host (bit mask passed separately)
};

// Everything the step passes need; one struct per grid, passed by value.
template <typename R> struct StepArgs {
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const C* cur;
    C* prev;
    int nx, ny, nz;
    long long ncell;
    const C* tw[3];          // w_N^m = e^{-2 pi i m / N} per axis
    const R* kin[3];         // dt hbar k_m^2 / (m N) per axis, FFT index order
    const R* mask[3];        // exp(-gamma dt) per axis
    const R* V;              // potential on its support box [vlo, vhi)
    int vlo[3], vhi[3];
    const C* phase[3];       // exp(i k_a (x_a - r_O,a)) per member per axis: [b * n_a + i]
    const R* zeta[3];        // taper and its first two derivatives per axis (PAPER form)
    const R* zeta1[3];
    const R* zeta2[3];
    int tf_lo[3], tf_hi[3];
    const MemberDev* mem;
    long long step;          // n: index of the current state
    double dt, hbar, mass;
    R c2;                    // 2 dt / hbar, rounded once on the host
    R h2m;                   // hbar^2 / 2m
    int mode;                // PSTD_TFSF_EXACT / PSTD_TFSF_PAPER
    int pipe_y;              // y pass form where available: PSTD_LINE_PIPELINED or PSTD_LINE_TMA (autotuner)
    int tma_z;               // z pass fed by tensor copies where available (autotuner)
    int plan[3];             // per axis: 1 = the alternative FFT plan of the size (128, 256; FP32)
    const void* tmap_y;      // tensor maps of the current level (device memory): boxes of 32 y lines
    const void* tmap_z;      //   and of 32 z lines (see colpass_tma_kernel)
    int pf_l1;               // the state exceeds L2: the z pass prefetches its update operand to L1
    int* flag;               // bit 0: non-finite value written
    const C* tfac;           // a(t_n) e^{-i w0 t_n}: [(n - tfac_base) * batch + member], evaluated in FP64 on the host
    long long tfac_base;
    // wave-packet members: psi_inc = tfac * phases * exp(-alpha_n (d - c_n)^2), d = sum of the
    // per-axis projections khat_a (x_a - r_O,a); tenv = [(n - tfac_base) * batch + member][Re alpha, Im alpha, c]
    unsigned long long packet_mask;
    const R* proj[3];        // [member * n_a + i]
    const R* tenv;
    // spinor grids: members (2p, 2p+1) are the up and down components of spinor p, coupled by
    // W = V I + gamma sigma . B on the node box [blo, bhi) where B is stored
    int spinor;
    const R* B[3];
    int blo[3], bhi[3];
    R gamma;
    // members driven by the 1-D auxiliary incident wave (pstd_set_incidence_aux): psi_inc (and,
    // for the PAPER form, d psi_inc / d d) at the source box's nodes for the current step, from
    // aux_eval_kernel; [slot][node of the box], slot = rank of the member among aux_mask's bits
    unsigned long long aux_mask;
    const C* aux_inc;
    const C* aux_dinc;
    int abox_lo[3], abox_n[3];
    int batch;
};

// The 1-D auxiliary incident wave of one step (Eqs. pstd_psiinc, pstd_dpsiinc) on a node box:
// psi_inc(d) = sum_m G_m^n e^{i q_m d}, q_m = q_0 + m dq, d = khat . (r - r_O), with
// e^{i q_0 d}, e^{i dq d} and e^{i 32 dq d} as products of per-axis tables.
template <typename R> struct AuxEvalArgs {
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const C* t0[3];           // e^{i q_0 khat_a (x_a - r_O,a)}: [slot * n_a + i]
    const C* t1[3];           // e^{i dq khat_a (x_a - r_O,a)}
    const C* t32[3];          // e^{i 32 dq khat_a (x_a - r_O,a)}
    const C* G;               // G_m^n: [slot][step of the call][m], nm a multiple of 32 (zero padded)
    const C* dG;              // i q_m G_m^n (PAPER form), same layout; null for the EXACT form
    int nm;
    long long slot_stride;    // entries per slot of G (steps of the call * nm)
    long long step_off;       // (step - first step of the call)
    int nslot;
    int n[3];                 // grid size
    int lo[3], bn[3];         // the box
    C* out;                   // [slot][box node]
    C* dout;                  // PAPER form: d psi_inc / d d
};

// G_m^n = G0_m e^{-i theta_m n} (and i q_m G_m^n) for steps [n0, n0 + nsteps) of every slot,
// phases in FP64; G0, theta, q: [slot][m] doubles (G0 complex)
template <typename R>
cudaError_t launch_aux_table(const double2* G0, const double* theta, const double* q, int nslot, int nm, long long n0,
                             long nsteps, bool deriv, typename std::conditional<sizeof(R) == 4, float2, double2>::type* G,
                             typename std::conditional<sizeof(R) == 4, float2, double2>::type* dG, cudaStream_t s);
template <typename R> cudaError_t launch_aux_eval(const AuxEvalArgs<R>& a, cudaStream_t s);

// Running-DFT arguments for the passes that accumulate on DFT-window steps.
template <typename R> struct DftArgs {
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const C* cur;
    int nx, ny, nz;
    long long ncell;
    int axis;
    int h[2];                 // node indices of the two planes normal to `axis`
    const C* dw;              // [2][N_axis] spectral-derivative weights for the two planes
    double2* acc;             // accumulators, see Grid::acc_offset
    long long acc_member_stride;   // doubles2 per member
    long long acc_freq_stride;     // per frequency
    long long face_off[6];         // offset of face (psi plane) within a frequency block
    long long face_size[6];
    const MemberDev* mem;
    unsigned long long member_mask;
    long long step;
    double dt;
    const double2* phase;          // e^{+i omega_f t_n}: [member][freq][window step], built on the host
    long long phase_member_stride;  // entries per member
    long long phase_len;            // window steps per frequency
    const long long* window_first;  // per member
};

// d == nullptr: plain pass; otherwise the pass also accumulates the running DFT on the two
// virtual planes normal to its axis (d->axis must match the pass)
template <typename R> cudaError_t launch_xpass(const StepArgs<R>& a, const DftArgs<R>* d, int batch, cudaStream_t s);
template <typename R> cudaError_t launch_ypass(const StepArgs<R>& a, const DftArgs<R>* d, int batch, cudaStream_t s);
// src: 0 plain z pass; otherwise also add the V-term and source in the epilogue: 1 for
// scalar CW members only, 3 for CW and wave-packet members, 4 for CW and auxiliary-wave
// members, 2 for any members (spinor pairs as well)
template <typename R> cudaError_t launch_zpass(const StepArgs<R>& a, const DftArgs<R>* d, int src, int batch, cudaStream_t s);
template <typename R> cudaError_t launch_source(const StepArgs<R>& a, int batch, cudaStream_t s);
// fused x + y pass (one CTA per z plane); available for FP32 square planes of 64, 96, 128
template <typename R> bool xypass_available(int nx, int ny, int mode);
template <typename R> bool pipe_y_available(int ny);
// tensor-copy-fed y or z pass: FP32 lines of 128, 192 or 256 points
template <typename R> bool tma_pass_available(int n);
template <typename R>
cudaError_t launch_xypass(const StepArgs<R>& a, const DftArgs<R>* dx, const DftArgs<R>* dy, int batch, cudaStream_t s,
                          int mode);

// ---------------------------------------------------------------------------------
// surface-equivalence transform
// ---------------------------------------------------------------------------------
struct FaceGeom {
    int axis, b, c;           // normal axis, fast and slow in-plane axes
    double sigma;             // -1 low face, +1 high face
    double plane;             // coordinate of the plane along `axis`
    double db, dc;            // in-plane spacings
    double cb0, cc0;          // centre coordinates of the first surface cell along b, c
    int L, M;                 // surface cells along b, c
    int Nb, Nc;               // plane size
    int lo_b, lo_c;           // first surface-cell node index along b, c
    long long cell0;          // index of the face's first cell in the global cell order
};

// Far field from the plane spectra (see farfield_kernel): per face, the 2-D DFT of the
// scaled psi and d psi/d a planes, transposed to [q][i'][j'] and divided by N_b N_c.
template <typename R> struct FarArgs {
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const C* ct;              // spectra, faces back to back
    long long ct_off[6];
    FaceGeom face[6];
    const double* theta;
    const double* phi;
    long long M;
    double k;
    int face_split;           // 1: every block sums all faces; 6: blockIdx.y selects the face
    double2* partial;         // [face_split][M]
};

template <typename R> cudaError_t launch_farfield(const FarArgs<R>& a, cudaStream_t s);
// Ct[q][m][j] = scale * C[q][j][m] in the working precision (C from double2, [Nc][Nb] per quantity)
template <typename R> cudaError_t launch_spectrum_pack(const typename std::conditional<sizeof(R) == 4, float2, double2>::type* c_psi,
                                                       const typename std::conditional<sizeof(R) == 4, float2, double2>::type* c_dpsi,
                                                       int Nb, int Nc, double scale,
                                                       typename std::conditional<sizeof(R) == 4, float2, double2>::type* ct,
                                                       cudaStream_t s);

// members per launch of the multi-member surface transform (bounds its record buffer)
constexpr int kTransformLaunchMembers = 16;

template <typename R> struct TransformArgs {
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const C* rec;             // per cell: G*G psi node values then G*G dpsi node values (weights folded in)
    int members;              // > 0: members in one launch (records [member][cell], wavenumbers km)
    double km[kTransformLaunchMembers];
    long long ncells;
    FaceGeom face[6];
    const double* pts;        // M x 3 points
    long long M;
    double k;
    double gl_node[16];       // Gauss-Legendre nodes on [-1, 1]
    long long cells_per_split;
    double2* partial;         // [split][member][M]
};

// points per thread of the surface transform (CTAs of 128 threads): two points share each
// cell record read from shared memory
#ifndef PSTD_TRANSFORM_PT
#define PSTD_TRANSFORM_PT 2
#endif
template <typename R> cudaError_t launch_transform(const TransformArgs<R>& a, int G, int splits, cudaStream_t s);


// ---------------------------------------------------------------------------------
// discrete adjoint (see adjoint_kernels.cuh)
// ---------------------------------------------------------------------------------
// J = scale * E^T conj(g): g = gradient with respect to one frequency's scaled phasors
// (six faces, psi plane then dpsi plane each, [c][b], faces at face_off)
template <typename R> struct InjectionArgs {
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const double2* g;
    long long face_off[6], face_size[6];
    const C* dw[3];           // [2][N_axis] spectral-derivative weights of the two planes per axis
    int h[3][2];              // plane node indices per axis (low, high)
    int n[3];
    long long ncell;
    double2 scale;            // 1 / S_f
    C* J;
};

// grad[box] += c2 Im[nu (u + s phase)] over the box [lo, hi), x fastest
template <typename R> struct GradArgs {
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const C* nu;              // nu^{n+1}, every member ([member][z][y][x])
    const C* u;               // u^n, every member
    const C* phase[3];        // incident phase tables [member][n_axis]
    C s[PSTD_MAX_BATCH];      // per member a(t_n) e^{-i w0 t_n}
    int with_inc;             // EXACT form: add psi_inc^n
    int batch;                // members summed into the gradient (V is shared)
    int nx, ny, nz;
    long long ncell;          // nodes of one member
    int lo[3], hi[3];
    double c2;                // 2 dt / hbar
    double* grad;
};

template <typename R> struct AdjPoint {
    R d0a, d0b, d0c, R0;      // point minus face centre (normal, b, c) and its length
    R ax, ay;                 // pref conj(e^{ik R0}) dL/dPsi_p
};

template <typename R> struct AdjointTransformArgs {
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    FaceGeom face[6];
    const double* pts;        // M x 3
    const double2* gpts;      // dL/dPsi per point
    long long M;
    double k;
    double gl_node[16];
    AdjPoint<R>* table;       // [6][M]
    long long ncells;
    long long points_per_split;
    C* partial;               // [split][ncells][2 G G]
};

template <typename R> cudaError_t launch_injection(const InjectionArgs<R>& a, cudaStream_t s);
template <typename R>
cudaError_t launch_inject(typename std::conditional<sizeof(R) == 4, float2, double2>::type* prev,
                          const typename std::conditional<sizeof(R) == 4, float2, double2>::type* J,
                          typename std::conditional<sizeof(R) == 4, float2, double2>::type coef, long long n, cudaStream_t s);
template <typename R> cudaError_t launch_grad(const GradArgs<R>& a, cudaStream_t s);
template <typename R> cudaError_t launch_adj_points(const AdjointTransformArgs<R>& a, cudaStream_t s);
template <typename R> cudaError_t launch_transform_adjoint(const AdjointTransformArgs<R>& a, int G, int splits, cudaStream_t s);
template <typename R>
cudaError_t launch_sum_splits(const typename std::conditional<sizeof(R) == 4, float2, double2>::type* partial, int splits,
                              long long n, typename std::conditional<sizeof(R) == 4, float2, double2>::type* rec,
                              cudaStream_t s);
template <typename R>
cudaError_t launch_unpack_records(const typename std::conditional<sizeof(R) == 4, float2, double2>::type* rec, int L, int M,
                                  int G, const double* glw, double cw, long long cell0,
                                  typename std::conditional<sizeof(R) == 4, float2, double2>::type* op,
                                  typename std::conditional<sizeof(R) == 4, float2, double2>::type* od, cudaStream_t s);
template <typename R>
cudaError_t launch_widen(const typename std::conditional<sizeof(R) == 4, float2, double2>::type* in, double2* out,
                         long long n, cudaStream_t s);
cudaError_t launch_reduce_partials(const double2* partial, int splits, long long M, double2* out,
                                   double* dsdo, cudaStream_t s);
// complex GEMM C[MxN] = alpha * A[MxK] B[KxN] (row-major, leading dims given), C = float2 or double2
template <typename C> cudaError_t launch_cgemm(int M, int N, int K, const C* A, int lda, const C* B, int ldb, C* Cm,
                                              int ldc, double2 alpha, cudaStream_t s);
template <typename C> cudaError_t launch_convert(const double2* in, C* out, long long n, cudaStream_t s);
// gather node values into cell records (mirrored-node combinations, see ntdf_kernels.cuh)
template <typename R> cudaError_t launch_pack_records(const typename std::conditional<sizeof(R) == 4, float2, double2>::type* out_psi,
                                                     const typename std::conditional<sizeof(R) == 4, float2, double2>::type* out_dpsi,
                                                     int L, int M, int G, const double* glw, double cw, long long cell0,
                                                     typename std::conditional<sizeof(R) == 4, float2, double2>::type* rec,
                                                     cudaStream_t s);

// used by the allocation-free far-field entry point (noalloc.cu)
int grid_device(const pstd_grid* g);
pstd_status grid_error(pstd_grid* g, pstd_status s, const char* msg);
pstd_status far_field_into_scratch(pstd_grid* g, int b, int f, const double* theta, const double* phi, long M,
                                   double* out_dsdo, double2* out_f, double2* scratch, long long scratch_elems);

}  // namespace pstd
