// C ABI of the PSTD library (include/pstd.h): grid objects, host-side tables in double
// precision, the step loop, the running-DFT bookkeeping and the transform drivers.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>

#include "pstd_internal.h"

using namespace pstd;
using cd = std::complex<double>;

namespace {

thread_local std::string g_create_error;
constexpr double kPi = 3.14159265358979323846;
constexpr int kSizes[] = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384};
constexpr int kKernelIds = 9;

bool supported_size(int n)
{
    for (int s : kSizes)
        if (s == n) return true;
    return false;
}

struct MemberHost {
    bool has_inc = false;
    double khat[3] = {0, 0, 1};
    double k = 0, E = 0, w0 = 0, eta = 1, ramp = 0;
    double rO[3] = {0, 0, 0};
    int nfreq = 0;
    double omega[PSTD_MAX_FREQ] = {};
    long long first = 0, len = 0;
    long long accumulated = 0;
    cd inc_phasor[PSTD_MAX_FREQ];
    bool packet = false;         // Gaussian wave packet (pstd_set_incidence_packet)
    double sigma = 1.0, d0 = 0.0;
    cd chi = cd(1.0, 0.0);       // spinor component's incident amplitude (pstd_set_incidence_spinor)
    // 1-D auxiliary incident wave (pstd_set_incidence_aux): its Fourier modes l0 .. l0 + G0.size() - 1,
    // psi_inc^n(d) = sum_m G0_m e^{i (q_m d - theta_m n)}
    bool aux = false;
    double aux_dt = 0, aux_dq = 0;
    std::vector<cd> aux_G0;
    std::vector<double> aux_theta, aux_q;
};

// The incident wave of member m at the first-contact corner r_O at time t (Eq. incpsiphasor's
// integrand): the CW wave a(t) e^{-i w0 t}, or the packet at d = 0
cd incident_at_origin(const MemberHost& m, double t, double hbar, double mass)
{
    if (m.aux) {   // d = 0 (Eq. pstd_psiinc)
        const double n = std::nearbyint(t / m.aux_dt);
        cd s(0.0, 0.0);
        for (size_t i = 0; i < m.aux_G0.size(); ++i) s += m.aux_G0[i] * std::exp(cd(0.0, -m.aux_theta[i] * n));
        return s;
    }
    if (m.packet) {
        const double tau = hbar * t / (2.0 * mass * m.sigma * m.sigma);
        const double v = hbar * m.k / mass;
        const cd q(1.0, tau);
        const double x = -m.d0;
        return std::pow(q, -0.5) * std::exp(-(x - v * t) * (x - v * t) / (4.0 * m.sigma * m.sigma * q) +
                                            cd(0.0, m.k * x - m.w0 * t));
    }
    const double env = (m.ramp <= 0 || t >= m.ramp) ? 1.0 : (t <= 0 ? 0.0 : 0.5 * (1.0 - std::cos(kPi * t / m.ramp)));
    return env * std::exp(cd(0.0, -m.w0 * t));
}

struct GraphKey {
    bool valid = false;
    long long n0 = 0, nsteps = 0;
    int cur = 0;
    long long version = 0;
    const void* tfac = nullptr;
    const void* tenv = nullptr;
    const void* aux[4] = {};                // auxiliary-wave table, derivative table, value and derivative buffers
    bool operator==(const GraphKey& o) const
    {
        return valid && o.valid && n0 == o.n0 && nsteps == o.nsteps && cur == o.cur && version == o.version &&
               tfac == o.tfac && tenv == o.tenv && aux[0] == o.aux[0] && aux[1] == o.aux[1] && aux[2] == o.aux[2] &&
               aux[3] == o.aux[3];
    }
};

struct TimedLaunch {
    int kernel;
    cudaEvent_t a, b;
};

}  // namespace

struct pstd_grid {
    pstd_grid_desc desc{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    int prec = PSTD_F32;
    size_t csize = 8, rsize = 4;
    long long ncell = 0;
    int batch = 1;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    long long n = 0;
    void* tw[3] = {};
    void* kin[3] = {};
    void* mask[3] = {};
    void* zeta[3] = {};
    void* zeta1[3] = {};
    void* zeta2[3] = {};
    void* phase[3] = {};
    void* dw[3] = {};
    void* V = nullptr;
    // spinor grids (pstd_set_magnetic_field): gamma B on its support box, components = member pairs
    bool spinor = false;
    void* B[3] = {};
    int blo[3] = {0, 0, 0}, bhi[3] = {0, 0, 0};
    double gamma_b = 0, bmax = 0;
    int vlo[3] = {0, 0, 0}, vhi[3] = {0, 0, 0};
    double vmax = 0;
    bool mask_ready = false;
    MemberDev* mem_dev = nullptr;
    std::vector<MemberHost> mem;
    // running DFT accumulators [member][freq][face: psi plane, dpsi plane]
    double2* acc = nullptr;
    int acc_freq_cap = 0;
    long long face_off[6] = {}, face_size[6] = {};
    long long acc_freq_stride = 0;
    long long phasor_version = 0;
    void* tfac = nullptr;                  // [step of the call][member] a(t_n) e^{-i w0 t_n}, working precision
    void* tenv = nullptr;                  // [step of the call][member][3] wave-packet envelope coefficients
    size_t tenv_cap = 0;
    void* proj[3] = {};                    // [member][i] khat_a (x_a - r_O,a), working precision
    unsigned long long packet_mask = 0;
    // 1-D auxiliary incident waves (slots = aux members in member order)
    unsigned long long aux_mask = 0;
    int aux_nslot = 0, aux_nm = 0;          // slots; modes per slot (a multiple of 32, zero padded)
    void* aux_t0[3] = {};                   // [slot][i] e^{i q_0 khat_a (x_a - r_O,a)}, working precision
    void* aux_t1[3] = {};                   // ... e^{i dq ...}
    void* aux_t32[3] = {};                  // ... e^{i 32 dq ...}
    double2* aux_G0 = nullptr;              // [slot][m]
    double* aux_theta = nullptr;
    double* aux_q = nullptr;
    void* aux_tab = nullptr;                // [slot][step of the call][m] G_m^n, working precision
    size_t aux_tab_cap = 0;
    void* aux_dtab = nullptr;               // i q_m G_m^n (PAPER form)
    size_t aux_dtab_cap = 0;
    void* aux_inc = nullptr;                // [slot][box node] psi_inc of the current step
    size_t aux_inc_cap = 0;
    void* aux_dinc = nullptr;               // d psi_inc / d d (PAPER form)
    size_t aux_dinc_cap = 0;
    long aux_call_steps = 0;                // steps of the call the table holds
    size_t tfac_cap = 0;
    double2* dft_phase = nullptr;          // [member][freq][window step] e^{+i omega t_n}
    size_t dft_phase_cap = 0;
    long long dft_phase_len = 0;           // window steps per frequency (max over members)
    long long* window_first_dev = nullptr; // per member
    int* flag = nullptr;
    // transform
    int G = 8;
    int G_order = 0;                        // quadrature nodes a cell edge chosen by the caller (0: default)
    std::vector<double> gl_x, gl_w;
    double* gl_w_dev = nullptr;
    FaceGeom faces[6];
    long long ncells = 0;
    // record / spectrum preparation operands, all in the working precision (float2 or double2)
    void* MbT[6] = {};
    void* Mc[6] = {};
    void* T1 = nullptr;
    void* OutP = nullptr;
    void* OutD = nullptr;
    void* Pw = nullptr;                     // one accumulator plane converted to the working precision (FP32 only)
    void* MbTH[6] = {};                     // conj(MbT)^T [L G][Nb] and conj(Mc)^T [Nc][M G]: the adjoint transform
    void* McH[6] = {};
    // adjoint buffers (allocated on first use)
    void* adj_table = nullptr;              // [6][M] AdjPoint
    size_t adj_table_cap = 0;
    void* adj_partial = nullptr;            // [split][ncells][2 G G]
    size_t adj_partial_cap = 0;
    void* adj_rec = nullptr;                // record gradients [ncells][2 G G]
    void* adj_PA = nullptr;                 // one plane gradient, working precision
    double2* adj_gpts = nullptr;            // dL/dPsi per point (device copy)
    size_t adj_gpts_cap = 0;
    double2* adj_out = nullptr;             // phasor-layout gradient (device copy)
    size_t adj_out_cap = 0;
    void* adj_J = nullptr;                  // injection volumes, one per frequency
    size_t adj_J_cap = 0;
    void* adj_ckpt = nullptr;               // checkpoints (psi^{n-1}, psi^n)
    size_t adj_ckpt_cap = 0;
    void* adj_seg = nullptr;                // forward states of one segment
    size_t adj_seg_cap = 0;
    void* adj_nu = nullptr;                 // two adjoint levels
    size_t adj_nu_cap = 0;
    void* adj_zero = nullptr;               // one zero complex: the adjoint run's incident time factor
    double* adj_grad = nullptr;             // gradient accumulators on the box
    size_t adj_grad_cap = 0;
    // checkpoints in adj_ckpt: segment s holds (psi^{sK-1}, psi^{sK}) of the run from rest;
    // valid for s K < ckpt_upto and s < ckpt_slots (ckpt_upto = -1: none valid)
    bool ckpt_record = false;               // pstd_step records them (pstd_set_checkpointing)
    bool ckpt_contig = true;                // the state is the run from rest at step n (V, incidence unchanged)
    long ckpt_K = 0;
    long ckpt_slots = 0;
    long long ckpt_upto = -1;
    void* rec = nullptr;
    void* rec_group = nullptr;              // records of a member group ([member][cell][2 G G])
    size_t rec_group_cap = 0;
    int rec_member = -1, rec_freq = -1;
    long long rec_version = -1;
    void* Fdft[6][2] = {};                  // per face: DFT matrices along b (Nb x Nb) and c (Nc x Nc)
    void* specP = nullptr;                  // per-face 2-D spectra (scratch for the preparation)
    void* specD = nullptr;
    void* ct = nullptr;                     // far-field spectra, working precision, faces back to back
    long long ct_off[6] = {};
    int ct_member = -1, ct_freq = -1;
    long long ct_version = -1;
    double2* partial = nullptr;
    size_t partial_cap = 0;
    double* pts_dev = nullptr;
    size_t pts_cap = 0;
    double2* out_dev = nullptr;
    size_t out_cap = 0;
    double* dsdo_dev = nullptr;
    size_t dsdo_cap = 0;
    // instrumentation
    bool timing = false;
    int xy_mode = PSTD_XY_SEPARATE;         // fused x + y pass (every step; with the plane DFT on window steps)
    int y_mode = PSTD_LINE_PLAIN;           // y pass form (192/256-point lines: pipelined; 128-256: TMA-fed)
    bool tma_z = false;                     // TMA-fed z pass (128/192/256-point lines, steps without the DFT)
    int plans = 0;                          // bit a: axis a uses the alternative FFT plan of its size
    void* tmaps = nullptr;                  // tensor maps [level buffer][y, z] (device memory, 4 x 128 B)
    bool tma_y_ok = false, tma_z_ok = false;
    // CUDA-graph replay of repeated runs (see run_steps)
    bool graphs = true;
    long long config_version = 0;           // bumped by every call that changes kernel arguments
    GraphKey seen_key, graph_key;
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_launches = 0;
    long long graph_replays = 0;            // pstd_step calls run as one graph launch
    cudaStream_t cap_stream = nullptr;      // private stream for graph capture
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> event_pool;
    long long launches = 0;
    std::string err;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

pstd_status fail(pstd_grid* g, pstd_status s, const std::string& msg)
{
    if (g) g->err = msg;
    else g_create_error = msg;
    return s;
}

pstd_status cuda_fail(pstd_grid* g, cudaError_t e, const char* where)
{
    return fail(g, PSTD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(g, call)                                             \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail((g), e_, #call); \
    } while (0)

template <typename T> cudaError_t dalloc(T** p, size_t bytes)
{
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

double coord(const pstd_grid_desc& d, int axis, int i) { return (i - d.n[axis] / 2) * d.d[axis]; }

double wavenumber(int n, double d, int m)
{
    const int ms = m < (n + 1) / 2 ? m : m - n;   // -N/2..N/2-1 (note after Eq. PSTDupdating)
    return 2.0 * kPi * ms / (n * d);
}

// upload a host vector of doubles as the grid precision (real) or as complex
pstd_status upload_real(pstd_grid* g, void** dst, const std::vector<double>& h)
{
    if (!*dst) CK(g, dalloc(dst, h.size() * g->rsize));
    if (g->prec == PSTD_F64) {
        CK(g, cudaMemcpy(*dst, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(h.begin(), h.end());
        CK(g, cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    return PSTD_OK;
}

pstd_status upload_complex(pstd_grid* g, void** dst, const std::vector<cd>& h, size_t offset_elems = 0,
                           size_t total_elems = 0)
{
    if (!*dst) CK(g, dalloc(dst, (total_elems ? total_elems : h.size()) * g->csize));
    if (g->prec == PSTD_F64) {
        CK(g, cudaMemcpy(static_cast<char*>(*dst) + offset_elems * 16, h.data(), h.size() * 16, cudaMemcpyHostToDevice));
    } else {
        std::vector<float2> f(h.size());
        for (size_t i = 0; i < h.size(); ++i) f[i] = make_float2((float)h[i].real(), (float)h[i].imag());
        CK(g, cudaMemcpy(static_cast<char*>(*dst) + offset_elems * 8, f.data(), f.size() * 8, cudaMemcpyHostToDevice));
    }
    return PSTD_OK;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_G.
void gauss_legendre(int G, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(G, 0.0);
    w.assign(G, 0.0);
    for (int i = 0; i < G; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (G + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= G; ++l) {
                const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            dp = G * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int l = 2; l <= G; ++l) {
            const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
            p0 = p1;
            p1 = p2;
        }
        dp = G * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;   // ascending; x[G-1-i] = -x[i]
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// absorption rate per node along one axis (Eq. Poshcl-Teller or the graded polynomial)
std::vector<double> absorber_gamma(const pstd_grid_desc& d, int axis, double E0)
{
    const int n = d.n[axis], w = d.abc_cells[axis];
    std::vector<double> g(n, 0.0);
    if (w <= 0) return g;
    const double unit = E0 / d.hbar;
    for (int i = 0; i < n; ++i) {
        if (d.abc_profile == PSTD_ABC_POLY) {
            const int depth = std::max(std::max(w - i, i - (n - 1 - w)), 0);
            g[i] = d.abc_param[1] * unit * std::pow((double)depth / w, d.abc_param[0]);
        } else {
            const int dist = std::min(i, n - 1 - i);
            if (dist < w) {
                const double ch = std::cosh(d.abc_param[1] * dist);
                g[i] = d.abc_param[0] * unit / (ch * ch);
            }
        }
    }
    return g;
}

double xi(double r) { return r - 2.0 / (3.0 * kPi) * std::sin(2 * kPi * r) + 1.0 / (12.0 * kPi) * std::sin(4 * kPi * r); }
double dxi(double r) { return 1.0 - 4.0 / 3.0 * std::cos(2 * kPi * r) + 1.0 / 3.0 * std::cos(4 * kPi * r); }
double d2xi(double r) { return 8.0 * kPi / 3.0 * std::sin(2 * kPi * r) - 4.0 * kPi / 3.0 * std::sin(4 * kPi * r); }

void zeta_tables(const pstd_grid_desc& d, int axis, std::vector<double>& z, std::vector<double>& z1, std::vector<double>& z2)
{
    const int n = d.n[axis], lo = d.tfsf_lo[axis], hi = d.tfsf_hi[axis], t = d.taper_cells;
    const double w = t * d.d[axis];
    z.assign(n, 0.0);
    z1.assign(n, 0.0);
    z2.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        if (i > lo && i < lo + t) {
            const double r = double(i - lo) / t;
            z[i] = xi(r); z1[i] = dxi(r) / w; z2[i] = d2xi(r) / (w * w);
        } else if (i >= lo + t && i <= hi - t) {
            z[i] = 1.0;
        } else if (i > hi - t && i < hi) {
            const double r = double(i - (hi - t)) / t;
            z[i] = 1.0 - xi(r); z1[i] = -dxi(r) / w; z2[i] = -d2xi(r) / (w * w);
        }
    }
}

cudaEvent_t take_event(pstd_grid* g)
{
    if (!g->event_pool.empty()) {
        cudaEvent_t e = g->event_pool.back();
        g->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct Timer {
    pstd_grid* g;
    int id;
    cudaEvent_t a = nullptr;
    Timer(pstd_grid* g_, int id_) : g(g_), id(id_)
    {
        if (g->timing) {
            a = take_event(g);
            cudaEventRecord(a, g->stream);
        }
    }
    ~Timer()
    {
        ++g->launches;
        if (g->timing && a) {
            cudaEvent_t b = take_event(g);
            cudaEventRecord(b, g->stream);
            g->timed.push_back({id, a, b});
        }
    }
};

pstd_status check_member(pstd_grid* g, int b)
{
    if (b < 0 || b >= g->batch) return fail(g, PSTD_EINVAL, "batch member out of range");
    return PSTD_OK;
}

pstd_status copy_in(pstd_grid* g, void* dst, const void* src, size_t bytes, int mem)
{
    if (mem == PSTD_MEM_HOST) CK(g, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, g->stream));
    else if (mem == PSTD_MEM_DEVICE) CK(g, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, g->stream));
    else return fail(g, PSTD_EINVAL, "mem must be PSTD_MEM_HOST or PSTD_MEM_DEVICE");
    return PSTD_OK;
}

pstd_status copy_out(pstd_grid* g, void* dst, const void* src, size_t bytes, int mem)
{
    if (mem == PSTD_MEM_HOST) {
        CK(g, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, g->stream));
        CK(g, cudaStreamSynchronize(g->stream));
    } else if (mem == PSTD_MEM_DEVICE) {
        CK(g, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, g->stream));
    } else {
        return fail(g, PSTD_EINVAL, "mem must be PSTD_MEM_HOST or PSTD_MEM_DEVICE");
    }
    return PSTD_OK;
}

template <typename T> pstd_status ensure(pstd_grid* g, T** p, size_t& cap, size_t bytes)
{
    if (cap >= bytes && *p) return PSTD_OK;
    if (*p) {
        CK(g, cudaStreamSynchronize(g->stream));
        cudaFree(*p);
        *p = nullptr;
        cap = 0;
    }
    cudaError_t e = dalloc(p, bytes);
    if (e != cudaSuccess) return fail(g, PSTD_ENOMEM, "device allocation failed");
    cap = bytes;
    return PSTD_OK;
}

pstd_status validate(const pstd_grid_desc* d)
{
    if (!d) return fail(nullptr, PSTD_EINVAL, "null descriptor");
    for (int a = 0; a < 3; ++a) {
        if (!supported_size(d->n[a])) return fail(nullptr, PSTD_EINVAL, "n must be one of 8,12,16,24,32,48,64,96,128,192,256,384");
        if (!(d->d[a] > 0)) return fail(nullptr, PSTD_EINVAL, "spacing must be positive");
        const int n = d->n[a], w = d->abc_cells[a];
        if (w < 0 || 2 * w >= n) return fail(nullptr, PSTD_EINVAL, "absorber wider than the grid");
        if (d->taper_cells < 1) return fail(nullptr, PSTD_EINVAL, "taper_cells must be >= 1");
        if (!(d->huygens_lo[a] >= w && d->huygens_lo[a] <= d->tfsf_lo[a] &&
              d->tfsf_lo[a] + d->taper_cells <= d->tfsf_hi[a] - d->taper_cells && d->tfsf_hi[a] <= d->huygens_hi[a] &&
              d->huygens_hi[a] <= n - 1 - w && d->huygens_lo[a] < d->huygens_hi[a]))
            return fail(nullptr, PSTD_EINVAL,
                        "need abc <= huygens_lo <= tfsf_lo, tfsf_lo + taper <= tfsf_hi - taper, tfsf_hi <= huygens_hi <= n-1-abc");
    }
    if (!(d->dt > 0) || !(d->hbar > 0) || !(d->mass > 0)) return fail(nullptr, PSTD_EINVAL, "dt, hbar, mass must be positive");
    if (d->precision != PSTD_F32 && d->precision != PSTD_F64) return fail(nullptr, PSTD_EINVAL, "precision");
    if (d->batch < 1 || d->batch > PSTD_MAX_BATCH) return fail(nullptr, PSTD_EINVAL, "batch out of range");
    if (d->abc_profile != PSTD_ABC_POLY && d->abc_profile != PSTD_ABC_POSCHL_TELLER) return fail(nullptr, PSTD_EINVAL, "abc_profile");
    if (d->tfsf_mode != PSTD_TFSF_EXACT && d->tfsf_mode != PSTD_TFSF_PAPER) return fail(nullptr, PSTD_EINVAL, "tfsf_mode");
    return PSTD_OK;
}

double dt_bound(const pstd_grid_desc& d, double vmax)
{
    double s = 0;
    for (int a = 0; a < 3; ++a) s += 1.0 / (d.d[a] * d.d[a]);
    return d.hbar / (d.hbar * d.hbar * kPi * kPi / (2.0 * d.mass) * s + std::fabs(vmax));
}

pstd_status upload_members(pstd_grid* g)
{
    std::vector<MemberDev> h(g->batch);
    for (int b = 0; b < g->batch; ++b) {
        const MemberHost& m = g->mem[b];
        MemberDev& o = h[b];
        std::memset(&o, 0, sizeof(o));
        o.w0 = m.w0;
        o.ramp = m.ramp;
        o.eta = m.eta;
        for (int a = 0; a < 3; ++a) o.k[a] = m.k * m.khat[a];
        o.nfreq = m.nfreq;
        for (int f = 0; f < PSTD_MAX_FREQ; ++f) o.omega[f] = m.omega[f];
        o.packet = m.packet ? 1 : 0;
        for (int a = 0; a < 3; ++a) o.khat[a] = m.khat[a];
    }
    CK(g, cudaMemcpyAsync(g->mem_dev, h.data(), sizeof(MemberDev) * g->batch, cudaMemcpyHostToDevice, g->stream));
    CK(g, cudaStreamSynchronize(g->stream));
    return PSTD_OK;
}

// the node box on which aux members need psi_inc: the V box (EXACT form) or the interior of
// the TF/SF box, where the taper's derivatives live (PAPER form); n[] = 0 when empty
void aux_box(const pstd_grid* g, int lo[3], int n[3])
{
    for (int a = 0; a < 3; ++a) {
        if (g->desc.tfsf_mode == PSTD_TFSF_PAPER) { lo[a] = g->desc.tfsf_lo[a] + 1; n[a] = g->desc.tfsf_hi[a] - lo[a]; }
        else { lo[a] = g->vlo[a]; n[a] = g->vhi[a] - g->vlo[a]; }
    }
    if (n[0] <= 0 || n[1] <= 0 || n[2] <= 0) n[0] = n[1] = n[2] = 0;
}

// Tensor maps for the TMA-fed y and z passes: the state buffer as a 3-D tensor of 8-byte
// elements [member * nz + z][y][x] (x innermost), one map per level buffer and axis, with
// boxes of 32 x ny x 1 (y lines) and 32 x 1 x nz (z lines).  Built once per grid (the buffers
// never move) and kept in device memory; FP32 grids whose y or z lines have 128, 192 or 256
// points only.  The driver's encoder is reached through the runtime's entry-point query, so
// the library links no driver library.
pstd_status make_tensor_maps(pstd_grid* g)
{
    const int nx = g->desc.n[0], ny = g->desc.n[1], nz = g->desc.n[2];
    const bool ty = g->prec == PSTD_F32 && tma_pass_available<float>(ny);
    const bool tz = g->prec == PSTD_F32 && tma_pass_available<float>(nz);
    if (!ty && !tz) return PSTD_OK;
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                                const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return PSTD_OK;   // no encoder: the grid keeps the register-fed passes
        encode = reinterpret_cast<Encode>(fn);
    }
    CUtensorMap maps[4];
    std::memset(maps, 0, sizeof(maps));
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz * g->batch};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 8, (cuuint64_t)nx * ny * 8};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int lvl = 0; lvl < 2; ++lvl)
        for (int ax = 1; ax <= 2; ++ax) {
            if ((ax == 1 && !ty) || (ax == 2 && !tz)) continue;
            const cuuint32_t box[3] = {32, ax == 1 ? (cuuint32_t)ny : 1u, ax == 1 ? 1u : (cuuint32_t)nz};
            const CUresult r = encode(&maps[2 * lvl + ax - 1], CU_TENSOR_MAP_DATA_TYPE_INT64, 3, g->buf[lvl], dims, strides, box,
                                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return PSTD_OK;   // the grid keeps the register-fed passes
        }
    CK(g, dalloc(&g->tmaps, sizeof(maps)));
    CK(g, cudaMemcpy(g->tmaps, maps, sizeof(maps), cudaMemcpyHostToDevice));
    g->tma_y_ok = ty;
    g->tma_z_ok = tz;
    return PSTD_OK;
}

template <typename R> StepArgs<R> step_args(pstd_grid* g)
{
    using C = typename StepArgs<R>::C;
    StepArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.cur = static_cast<const C*>(g->buf[g->cur]);
    a.prev = static_cast<C*>(g->buf[g->cur ^ 1]);
    a.nx = g->desc.n[0]; a.ny = g->desc.n[1]; a.nz = g->desc.n[2];
    a.ncell = g->ncell;
    for (int ax = 0; ax < 3; ++ax) {
        a.tw[ax] = static_cast<const C*>(g->tw[ax]);
        a.kin[ax] = static_cast<const R*>(g->kin[ax]);
        a.mask[ax] = static_cast<const R*>(g->mask[ax]);
        a.phase[ax] = static_cast<const C*>(g->phase[ax]);
        a.zeta[ax] = static_cast<const R*>(g->zeta[ax]);
        a.zeta1[ax] = static_cast<const R*>(g->zeta1[ax]);
        a.zeta2[ax] = static_cast<const R*>(g->zeta2[ax]);
        a.tf_lo[ax] = g->desc.tfsf_lo[ax];
        a.tf_hi[ax] = g->desc.tfsf_hi[ax];
        a.vlo[ax] = g->vlo[ax];
        a.vhi[ax] = g->vhi[ax];
    }
    a.V = static_cast<const R*>(g->V);
    a.mem = g->mem_dev;
    a.step = g->n;
    a.dt = g->desc.dt; a.hbar = g->desc.hbar; a.mass = g->desc.mass;
    a.c2 = R(2.0 * g->desc.dt / g->desc.hbar);
    a.h2m = R(g->desc.hbar * g->desc.hbar / (2.0 * g->desc.mass));
    a.mode = g->desc.tfsf_mode;
    a.flag = g->flag;
    a.packet_mask = g->packet_mask;
    a.pipe_y = g->y_mode;
    a.tma_z = g->tma_z ? 1 : 0;
    for (int ax = 0; ax < 3; ++ax) a.plan[ax] = (g->plans >> ax) & 1;
    if (g->tmaps) {
        a.tmap_y = static_cast<const char*>(g->tmaps) + (size_t)(2 * g->cur + 0) * sizeof(CUtensorMap);
        a.tmap_z = static_cast<const char*>(g->tmaps) + (size_t)(2 * g->cur + 1) * sizeof(CUtensorMap);
    }
    // two levels of the whole batch against the 129 MB L2 (with room for the tables and the DFT)
    a.pf_l1 = 2.0 * (double)g->batch * (double)g->ncell * (double)g->csize > 96e6 ? 1 : 0;
    a.spinor = g->spinor ? 1 : 0;
    for (int ax = 0; ax < 3; ++ax) {
        a.B[ax] = static_cast<const R*>(g->B[ax]);
        a.blo[ax] = g->blo[ax];
        a.bhi[ax] = g->bhi[ax];
    }
    a.gamma = R(g->gamma_b);
    for (int ax = 0; ax < 3; ++ax) a.proj[ax] = static_cast<const R*>(g->proj[ax]);
    a.tenv = static_cast<const R*>(g->tenv);
    a.aux_mask = g->aux_mask;
    a.aux_inc = static_cast<const C*>(g->aux_inc);
    a.aux_dinc = static_cast<const C*>(g->aux_dinc);
    aux_box(g, a.abox_lo, a.abox_n);
    return a;
}

template <typename R> DftArgs<R> dft_args(pstd_grid* g, unsigned long long mask, int axis)
{
    using C = typename DftArgs<R>::C;
    DftArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.cur = static_cast<const C*>(g->buf[g->cur]);
    a.nx = g->desc.n[0]; a.ny = g->desc.n[1]; a.nz = g->desc.n[2];
    a.ncell = g->ncell;
    a.acc = g->acc;
    a.acc_freq_stride = g->acc_freq_stride;
    a.acc_member_stride = g->acc_freq_stride * g->acc_freq_cap;
    for (int f = 0; f < 6; ++f) { a.face_off[f] = g->face_off[f]; a.face_size[f] = g->face_size[f]; }
    a.mem = g->mem_dev;
    a.member_mask = mask;
    a.step = g->n;
    a.dt = g->desc.dt;
    a.phase = g->dft_phase;
    a.phase_len = g->dft_phase_len;
    a.phase_member_stride = g->dft_phase_len * PSTD_MAX_FREQ;
    a.window_first = g->window_first_dev;
    a.axis = axis;
    a.h[0] = g->desc.huygens_lo[axis];
    a.h[1] = g->desc.huygens_hi[axis];
    a.dw = static_cast<const C*>(g->dw[axis]);
    return a;
}

// incident time factors a(t_n) e^{-i w0 t_n} for steps [n0, n0 + nsteps) of every member,
// evaluated in double precision and rounded once to the working precision; uploaded in
// stream order (the previous call's kernels finish first)
pstd_status upload_time_factors(pstd_grid* g, long long n0, long nsteps)
{
    std::vector<cd> tab((size_t)std::max(1L, nsteps) * g->batch);
    std::vector<double> env((size_t)std::max(1L, nsteps) * g->batch * 3, 0.0);
    bool any_packet = false;
    for (long s = 0; s < nsteps; ++s) {
        const double t = (n0 + s) * g->desc.dt;
        for (int b = 0; b < g->batch; ++b) {
            const MemberHost& m = g->mem[b];
            if (m.packet) {
                // psi_inc = [q^{-1/2} e^{-i w0 t} e^{-i k d0}] e^{i k d} exp(-alpha (d - c)^2),
                // q = 1 + i tau, alpha = 1 / (4 sigma^2 q), c = d0 + v t
                any_packet = true;
                const double tau = g->desc.hbar * t / (2.0 * g->desc.mass * m.sigma * m.sigma);
                const cd q(1.0, tau);
                tab[(size_t)s * g->batch + b] = m.chi * std::pow(q, -0.5) * std::exp(cd(0.0, -m.w0 * t - m.k * m.d0));
                const cd alpha = 1.0 / (4.0 * m.sigma * m.sigma * q);
                double* e = &env[3 * ((size_t)s * g->batch + b)];
                e[0] = alpha.real();
                e[1] = alpha.imag();
                e[2] = m.d0 + g->desc.hbar * m.k / g->desc.mass * t;
            } else if (m.aux) {
                tab[(size_t)s * g->batch + b] = m.chi;   // psi_inc itself comes from aux_eval_kernel
            } else {
                tab[(size_t)s * g->batch + b] = m.chi * incident_at_origin(m, t, g->desc.hbar, g->desc.mass);
            }
        }
    }
    if (any_packet) {
        pstd_status st = ensure(g, &g->tenv, g->tenv_cap, env.size() * g->rsize);
        if (st != PSTD_OK) return st;
        if (g->prec == PSTD_F64) {
            CK(g, cudaMemcpyAsync(g->tenv, env.data(), env.size() * 8, cudaMemcpyHostToDevice, g->stream));
        } else {
            std::vector<float> f(env.begin(), env.end());
            CK(g, cudaMemcpyAsync(g->tenv, f.data(), f.size() * 4, cudaMemcpyHostToDevice, g->stream));
        }
    }
    pstd_status st = ensure(g, &g->tfac, g->tfac_cap, tab.size() * g->csize);
    if (st != PSTD_OK) return st;
    if (g->prec == PSTD_F64) {
        CK(g, cudaMemcpyAsync(g->tfac, tab.data(), tab.size() * 16, cudaMemcpyHostToDevice, g->stream));
    } else {
        std::vector<float2> f(tab.size());
        for (size_t i = 0; i < tab.size(); ++i) f[i] = make_float2((float)tab[i].real(), (float)tab[i].imag());
        CK(g, cudaMemcpyAsync(g->tfac, f.data(), f.size() * 8, cudaMemcpyHostToDevice, g->stream));
    }
    return PSTD_OK;
}

// Enqueue the kernels of one leapfrog step on the state pair in `a` (all batch members);
// `mask` selects the members whose running DFT accumulates this step (d* their arguments).
template <typename R>
pstd_status enqueue_step(pstd_grid* g, const StepArgs<R>& a, unsigned long long mask, const DftArgs<R>* dx,
                         const DftArgs<R>* dy, const DftArgs<R>* dz, bool need_src)
{
    // the V-term and source: folded into the z pass when x and y run fused; their own kernel
    // ahead of the separate x and y passes otherwise (where the DFT variants are heavier)
    const bool src_in_z = need_src && (g->xy_mode != PSTD_XY_SEPARATE || !mask);
    if (g->aux_mask && need_src) {
        // psi_inc of the aux members on the source box for this step (Eqs. pstd_psiinc, pstd_dpsiinc)
        AuxEvalArgs<R> x;
        std::memset(&x, 0, sizeof(x));
        using C = typename StepArgs<R>::C;
        for (int ax = 0; ax < 3; ++ax) {
            x.t0[ax] = static_cast<const C*>(g->aux_t0[ax]);
            x.t1[ax] = static_cast<const C*>(g->aux_t1[ax]);
            x.t32[ax] = static_cast<const C*>(g->aux_t32[ax]);
            x.n[ax] = g->desc.n[ax];
            x.lo[ax] = a.abox_lo[ax];
            x.bn[ax] = a.abox_n[ax];
        }
        const bool paper = g->desc.tfsf_mode == PSTD_TFSF_PAPER;
        x.G = static_cast<const C*>(g->aux_tab);
        x.dG = paper ? static_cast<const C*>(g->aux_dtab) : nullptr;
        x.nm = g->aux_nm;
        x.step_off = a.step - a.tfac_base;
        x.slot_stride = (long long)g->aux_nm * g->aux_call_steps;
        x.nslot = g->aux_nslot;
        x.out = static_cast<C*>(g->aux_inc);
        x.dout = paper ? static_cast<C*>(g->aux_dinc) : nullptr;
        Timer t(g, 8);
        CK(g, launch_aux_eval<R>(x, g->stream));
    }
    if (need_src && !src_in_z) {
        Timer t(g, 7);
        CK(g, launch_source<R>(a, g->batch, g->stream));
    }
    if (g->xy_mode != PSTD_XY_SEPARATE) {
        // x and y together, one CTA per z plane (with the x and y plane DFT on window steps)
        Timer t(g, 3);
        CK(g, launch_xypass<R>(a, mask ? dx : nullptr, mask ? dy : nullptr, g->batch, g->stream, g->xy_mode));
    } else {
        {
            Timer t(g, 0);
            CK(g, launch_xpass<R>(a, mask ? dx : nullptr, g->batch, g->stream));
        }
        {
            Timer t(g, 1);
            CK(g, launch_ypass<R>(a, mask ? dy : nullptr, g->batch, g->stream));
        }
    }
    {
        Timer t(g, 2);
        const int kind = (g->spinor || (g->aux_mask && g->packet_mask)) ? 2 : g->packet_mask ? 3 : g->aux_mask ? 4 : 1;
        CK(g, launch_zpass<R>(a, mask ? dz : nullptr, src_in_z ? kind : 0, g->batch, g->stream));
    }
    return PSTD_OK;
}

// One planned leapfrog step: its kernel arguments and which members accumulate the DFT.
template <typename R> struct PlannedStep {
    StepArgs<R> a;
    DftArgs<R> d[3];
    unsigned long long mask;
};

// Host side of nsteps steps from the grid's current state: kernel arguments per step, and the
// host bookkeeping of the running DFT (incident phasors at r_O, Eq. incpsiphasor), the step
// counter and the level parity.  dft = false leaves the running DFT untouched.
template <typename R> void plan_steps(pstd_grid* g, long nsteps, bool dft, long long n0, std::vector<PlannedStep<R>>* out)
{
    for (long s = 0; s < nsteps; ++s) {
        unsigned long long mask = 0;
        for (int b = 0; b < g->batch && dft; ++b) {
            const MemberHost& m = g->mem[b];
            if (m.nfreq > 0 && g->n >= m.first && g->n < m.first + m.len) mask |= 1ull << b;
        }
        PlannedStep<R> p;
        p.mask = mask;
        if (mask && out) {
            for (int ax = 0; ax < 3; ++ax) p.d[ax] = dft_args<R>(g, mask, ax);
        }
        if (mask) {
            const double t = g->n * g->desc.dt;
            for (int b = 0; b < g->batch; ++b) {
                if (!((mask >> b) & 1ull)) continue;
                MemberHost& m = g->mem[b];
                const cd inc = incident_at_origin(m, t, g->desc.hbar, g->desc.mass);   // Eq. incpsiphasor
                for (int f = 0; f < m.nfreq; ++f) m.inc_phasor[f] += inc * std::exp(cd(0.0, m.omega[f] * t));
                ++m.accumulated;
            }
            ++g->phasor_version;
        }
        if (out) {
            p.a = step_args<R>(g);
            p.a.tfac = static_cast<const typename StepArgs<R>::C*>(g->tfac);
            p.a.tfac_base = n0;
            p.a.batch = g->batch;
            out->push_back(p);
        }
        g->cur ^= 1;
        ++g->n;
    }
}

// Enqueue planned steps.  With `record` the checkpoints of the run from rest are copied aside
// before steps n = s K; with `save` the state after each step goes to save + (s + 1) * the
// size of one state of every member.
template <typename R>
pstd_status enqueue_steps(pstd_grid* g, const std::vector<PlannedStep<R>>& plan, bool record, void* save)
{
    const bool need_src = g->desc.tfsf_mode == PSTD_TFSF_PAPER || g->vhi[0] > g->vlo[0] || (g->spinor && g->bhi[0] > g->blo[0]);
    const size_t sb = (size_t)g->batch * g->ncell * g->csize;
    if (g->aux_mask && need_src && !plan.empty()) {
        // the aux members' Fourier coefficients for every step of this call
        using C = typename StepArgs<R>::C;
        Timer t(g, 8);
        CK(g, launch_aux_table<R>(g->aux_G0, g->aux_theta, g->aux_q, g->aux_nslot, g->aux_nm, plan[0].a.step, (long)plan.size(),
                                  g->desc.tfsf_mode == PSTD_TFSF_PAPER, static_cast<C*>(g->aux_tab),
                                  static_cast<C*>(g->aux_dtab), g->stream));
    }
    for (size_t s = 0; s < plan.size(); ++s) {
        const PlannedStep<R>& p = plan[s];
        const long long n = p.a.step;
        if (record && n % g->ckpt_K == 0 && n / g->ckpt_K < g->ckpt_slots) {
            char* ck = static_cast<char*>(g->adj_ckpt);
            const size_t slot = (size_t)(n / g->ckpt_K);
            CK(g, cudaMemcpyAsync(ck + 2 * slot * sb, p.a.prev, sb, cudaMemcpyDeviceToDevice, g->stream));
            CK(g, cudaMemcpyAsync(ck + (2 * slot + 1) * sb, p.a.cur, sb, cudaMemcpyDeviceToDevice, g->stream));
        }
        pstd_status st = enqueue_step<R>(g, p.a, p.mask, &p.d[0], &p.d[1], &p.d[2], need_src);
        if (st != PSTD_OK) return st;
        if (save) CK(g, cudaMemcpyAsync(static_cast<char*>(save) + (s + 1) * sb, p.a.prev, sb, cudaMemcpyDeviceToDevice, g->stream));
    }
    return PSTD_OK;
}

void drop_graph(pstd_grid* g)
{
    if (g->graph_exec) cudaGraphExecDestroy(g->graph_exec);
    g->graph_exec = nullptr;
    g->graph_key.valid = false;
}

// nsteps leapfrog steps from the grid's current state.  dft = false leaves the running DFT
// (device sums and host incident phasors) untouched; a non-null `save` receives, in stream
// order, the state after each step: save + (s + 1) * batch * ncell for step s.
//
// A run that repeats the previous run's key (first step, count, level parity, table pointers
// and configuration version: everything the kernel arguments hold) is captured once into a
// CUDA graph and replayed from then on; the host bookkeeping still runs step by step.
template <typename R> pstd_status run_steps(pstd_grid* g, long nsteps, bool dft = true, void* save = nullptr)
{
    const long long n0 = g->n;
    pstd_status st0 = upload_time_factors(g, n0, nsteps);
    if (st0 != PSTD_OK) return st0;
    if (g->aux_mask) {
        int lo[3], bn[3];
        aux_box(g, lo, bn);
        const size_t nb = (size_t)bn[0] * bn[1] * bn[2];
        const size_t tab = (size_t)g->aux_nslot * std::max(1L, nsteps) * g->aux_nm * g->csize;
        const size_t inc = (size_t)g->aux_nslot * std::max<size_t>(1, nb) * g->csize;
        const bool paper = g->desc.tfsf_mode == PSTD_TFSF_PAPER;
        st0 = ensure(g, &g->aux_tab, g->aux_tab_cap, tab);
        if (st0 == PSTD_OK) st0 = ensure(g, &g->aux_inc, g->aux_inc_cap, inc);
        if (st0 == PSTD_OK && paper) st0 = ensure(g, &g->aux_dtab, g->aux_dtab_cap, tab);
        if (st0 == PSTD_OK && paper) st0 = ensure(g, &g->aux_dinc, g->aux_dinc_cap, inc);
        if (st0 != PSTD_OK) return st0;
        g->aux_call_steps = std::max(1L, nsteps);
    }
    // checkpoint recording for the adjoint: steps of the run from rest, recorded from step 0 on
    if (dft && !save && g->ckpt_record && g->ckpt_contig && g->n == 0) g->ckpt_upto = 0;
    const bool record = dft && !save && g->ckpt_record && g->ckpt_contig && g->ckpt_upto == g->n;
    GraphKey key;
    key.valid = true;
    key.n0 = n0;
    key.nsteps = nsteps;
    key.cur = g->cur;
    key.version = g->config_version;
    key.tfac = g->tfac;
    key.tenv = g->tenv;
    key.aux[0] = g->aux_tab;
    key.aux[1] = g->aux_dtab;
    key.aux[2] = g->aux_inc;
    key.aux[3] = g->aux_dinc;
    const bool graphable = g->graphs && dft && !save && !record && !g->timing && nsteps >= 2;
    if (graphable && g->graph_exec && g->graph_key == key) {
        plan_steps<R>(g, nsteps, dft, n0, nullptr);
        CK(g, cudaGraphLaunch(g->graph_exec, g->stream));
        g->launches += g->graph_launches;
        ++g->graph_replays;
        return PSTD_OK;
    }
    std::vector<PlannedStep<R>> plan;
    plan.reserve(nsteps);
    plan_steps<R>(g, nsteps, dft, n0, &plan);
    if (record) g->ckpt_upto = g->n;
    if (graphable && g->seen_key == key) {
        // second run with this key: capture it
        // (captured on a private stream: the grid's stream may be the legacy default stream,
        // which cannot be captured; nothing executes during capture)
        drop_graph(g);
        const long long launches0 = g->launches;
        cudaGraph_t graph = nullptr;
        bool ok = g->cap_stream || cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
        cudaStream_t real = g->stream;
        if (ok) ok = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            g->stream = g->cap_stream;
            const pstd_status st = enqueue_steps<R>(g, plan, false, nullptr);
            g->stream = real;
            ok = cudaStreamEndCapture(g->cap_stream, &graph) == cudaSuccess && st == PSTD_OK && graph;
        }
        cudaGraphExec_t exec = nullptr;
        if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (ok) {
            g->graph_exec = exec;
            g->graph_key = key;
            g->graph_launches = g->launches - launches0;
            CK(g, cudaGraphLaunch(exec, g->stream));
            ++g->graph_replays;
            return PSTD_OK;
        }
        // capture is not available here: launch directly from now on
        cudaGetLastError();
        g->launches = launches0;
        g->graphs = false;
    }
    g->seen_key = key;
    return enqueue_steps<R>(g, plan, record, save);
}

// -------------------------------------------------------------------------------------
// transform preparation
// -------------------------------------------------------------------------------------
// Wavenumber of the free wave at DFT frequency f of member b, k = sqrt(2 m omega_f / hbar): the
// Green's function of the transform (Eq. NTDF) at the energy hbar omega_f of those phasors
// (the carrier k when omega_f = E / hbar)
double wavenumber_of(const pstd_grid* g, int b, int f)
{
    const MemberHost& m = g->mem[b];
    const double w = (f >= 0 && f < m.nfreq) ? m.omega[f] : m.w0;
    return std::sqrt(2.0 * g->desc.mass * w / g->desc.hbar);
}

pstd_status setup_transform(pstd_grid* g)
{
    if (g->MbT[0]) return PSTD_OK;
    const pstd_grid_desc& d = g->desc;
    // default cell quadrature: G = 8 in FP64 (exact to round-off against the literal mode sum);
    // G = 4 in FP32, whose worst case (an interpolant mode at the plane's Nyquist limit) is
    // 1.2e-4 of that mode, inside the FP32 transform target of 1e-3 and, on the workloads' fields,
    // far below FP32 rounding
    g->G = g->G_order ? g->G_order : (g->prec == PSTD_F64 ? 8 : 4);
    gauss_legendre(g->G, g->gl_x, g->gl_w);
    const int G = g->G;
    CK(g, dalloc(&g->gl_w_dev, sizeof(double) * G));
    CK(g, cudaMemcpy(g->gl_w_dev, g->gl_w.data(), sizeof(double) * G, cudaMemcpyHostToDevice));
    long long cell0 = 0;
    size_t t1max = 0, outmax = 0, specmax = 0;
    for (int f = 0; f < 6; ++f) {
        const int a = f / 2, s = f % 2;
        FaceGeom& F = g->faces[f];
        F.axis = a;
        F.b = a == 0 ? 1 : 0;
        F.c = a == 2 ? 1 : 2;
        F.sigma = s == 0 ? -1.0 : 1.0;
        F.plane = coord(d, a, s == 0 ? d.huygens_lo[a] : d.huygens_hi[a]);
        F.db = d.d[F.b];
        F.dc = d.d[F.c];
        F.cb0 = coord(d, F.b, d.huygens_lo[F.b]) + 0.5 * F.db;
        F.cc0 = coord(d, F.c, d.huygens_lo[F.c]) + 0.5 * F.dc;
        F.L = d.huygens_hi[F.b] - d.huygens_lo[F.b];
        F.M = d.huygens_hi[F.c] - d.huygens_lo[F.c];
        F.Nb = d.n[F.b];
        F.Nc = d.n[F.c];
        F.lo_b = d.huygens_lo[F.b];
        F.lo_c = d.huygens_lo[F.c];
        F.cell0 = cell0;
        cell0 += (long long)F.L * F.M;
        // trigonometric interpolation weights w(xi - i) = (1/N) sum_{i'=-N/2}^{N/2-1} e^{2 pi i i' (xi - i)/N}
        auto interp = [&](int N, int lo, int cells, bool transposed, std::vector<cd>& out) {
            out.assign((size_t)N * cells * G, cd(0, 0));
            for (int l = 0; l < cells; ++l)
                for (int gq = 0; gq < G; ++gq) {
                    const double xi_ = lo + l + 0.5 + 0.5 * g->gl_x[gq];
                    for (int i = 0; i < N; ++i) {
                        const double th = 2.0 * kPi * (xi_ - i) / N;
                        // geometric sum e^{-i th N/2} (e^{i th N} - 1) / (e^{i th} - 1)
                        const cd num = std::exp(cd(0, th * N)) - 1.0;
                        const cd den = std::exp(cd(0, th)) - 1.0;
                        const cd v = std::exp(cd(0, -th * (N / 2))) * num / den / double(N);
                        const size_t row = (size_t)l * G + gq;
                        if (transposed) out[(size_t)i * cells * G + row] = v;
                        else out[row * N + i] = v;
                    }
                }
        };
        std::vector<cd> mb, mc;
        interp(F.Nb, d.huygens_lo[F.b], F.L, true, mb);    // [Nb][L G]
        interp(F.Nc, d.huygens_lo[F.c], F.M, false, mc);   // [M G][Nc]
        if (upload_complex(g, &g->MbT[f], mb) != PSTD_OK || upload_complex(g, &g->Mc[f], mc) != PSTD_OK)
            return PSTD_ECUDA;
        {
            // conjugate transposes for the adjoint transform
            const int LG = F.L * G, MG = F.M * G;
            std::vector<cd> mbh((size_t)LG * F.Nb), mch((size_t)F.Nc * MG);
            for (int i = 0; i < F.Nb; ++i)
                for (int r = 0; r < LG; ++r) mbh[(size_t)r * F.Nb + i] = std::conj(mb[(size_t)i * LG + r]);
            for (int r = 0; r < MG; ++r)
                for (int j = 0; j < F.Nc; ++j) mch[(size_t)j * MG + r] = std::conj(mc[(size_t)r * F.Nc + j]);
            if (upload_complex(g, &g->MbTH[f], mbh) != PSTD_OK || upload_complex(g, &g->McH[f], mch) != PSTD_OK)
                return PSTD_ECUDA;
        }
        t1max = std::max(t1max, (size_t)F.Nc * std::max(F.L * G, F.Nb));
        t1max = std::max(t1max, (size_t)F.M * G * F.Nb);   // adjoint: [M G][Nb]
        outmax = std::max(outmax, (size_t)F.M * G * F.L * G);
        // DFT matrices e^{-2 pi i u v / N} for the plane spectra of the far field
        for (int q = 0; q < 2; ++q) {
            const int N = q == 0 ? F.Nb : F.Nc;
            std::vector<cd> fm((size_t)N * N);
            for (int u = 0; u < N; ++u)
                for (int v = 0; v < N; ++v) fm[(size_t)u * N + v] = std::exp(cd(0.0, -2.0 * kPi * (double)((long long)u * v % N) / N));
            if (upload_complex(g, &g->Fdft[f][q], fm) != PSTD_OK) return PSTD_ECUDA;
        }
        g->ct_off[f] = f == 0 ? 0 : g->ct_off[f - 1] + 2LL * g->faces[f - 1].Nb * g->faces[f - 1].Nc;
        specmax = std::max(specmax, (size_t)F.Nb * F.Nc);
    }
    g->ncells = cell0;
    CK(g, dalloc(&g->specP, specmax * g->csize));
    CK(g, dalloc(&g->specD, specmax * g->csize));
    if (g->prec != PSTD_F64) CK(g, dalloc(&g->Pw, specmax * g->csize));
    CK(g, dalloc(&g->adj_PA, specmax * g->csize));
    {
        const long long ctn = g->ct_off[5] + 2LL * g->faces[5].Nb * g->faces[5].Nc;
        if (dalloc(&g->ct, (size_t)ctn * g->csize) != cudaSuccess) return fail(g, PSTD_ENOMEM, "far-field spectra");
    }
    CK(g, dalloc(&g->T1, t1max * g->csize));
    CK(g, dalloc(&g->OutP, outmax * g->csize));
    CK(g, dalloc(&g->OutD, outmax * g->csize));
    if (dalloc(&g->rec, (size_t)g->ncells * 2 * G * G * g->csize) != cudaSuccess)
        return fail(g, PSTD_ENOMEM, "transform records");
    return PSTD_OK;
}

// the accumulators stay FP64 (Eqs. psiphasor, dpsiphasor); the preparation GEMMs run in the working
// precision, so an FP32 grid converts one [Nc][Nb] plane at a time
template <typename C> const C* plane_in_working_precision(pstd_grid* g, const double2* plane, const FaceGeom& F)
{
    if (std::is_same<C, double2>::value) return reinterpret_cast<const C*>(plane);
    const cudaError_t e = launch_convert<C>(plane, static_cast<C*>(g->Pw), (long long)F.Nb * F.Nc, g->stream);
    if (e != cudaSuccess) {
        cuda_fail(g, e, "plane conversion");
        return nullptr;
    }
    return static_cast<const C*>(g->Pw);
}

pstd_status check_window(pstd_grid* g, int b, int f)
{
    pstd_status st = check_member(g, b);
    if (st != PSTD_OK) return st;
    const MemberHost& m = g->mem[b];
    if (f < 0 || f >= m.nfreq) return fail(g, PSTD_EINVAL, "frequency index out of range");
    if (m.len <= 0 || m.accumulated < m.len) return fail(g, PSTD_ESTATE, "the DFT window has not completed");
    if (std::abs(m.inc_phasor[f]) == 0.0) return fail(g, PSTD_ESTATE, "incident phasor at r_O is zero");
    return PSTD_OK;
}

// the cell records of member b, frequency f, into dst (ncells * 2 G^2 values): the grid's
// own record buffer (cached per member, frequency and phasor version) when dst is null
template <typename R> pstd_status prepare_records(pstd_grid* g, int b, int f, void* dst = nullptr)
{
    pstd_status st = setup_transform(g);
    if (st != PSTD_OK) return st;
    if (!dst && g->rec_member == b && g->rec_freq == f && g->rec_version == g->phasor_version) return PSTD_OK;
    const MemberHost& m = g->mem[b];
    const cd scale = 1.0 / m.inc_phasor[f];   // Eqs. scaledphsiphasor, scaleddpsiphasor
    const int G = g->G;
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const double2* base = g->acc + (long long)b * g->acc_freq_stride * g->acc_freq_cap + (long long)f * g->acc_freq_stride;
    C* T1 = static_cast<C*>(g->T1);
    for (int fi = 0; fi < 6; ++fi) {
        const FaceGeom& F = g->faces[fi];
        const int LG = F.L * G, MG = F.M * G;
        for (int q = 0; q < 2; ++q) {
            Timer t(g, 4);
            const C* P = plane_in_working_precision<C>(g, base + g->face_off[fi] + q * g->face_size[fi], F);   // [Nc][Nb]
            if (!P) return PSTD_ECUDA;
            C* out = static_cast<C*>(q == 0 ? g->OutP : g->OutD);
            CK(g, launch_cgemm<C>(F.Nc, LG, F.Nb, P, F.Nb, static_cast<const C*>(g->MbT[fi]), LG, T1, LG,
                                  make_double2(scale.real(), scale.imag()), g->stream));
            CK(g, launch_cgemm<C>(MG, LG, F.Nc, static_cast<const C*>(g->Mc[fi]), F.Nc, T1, LG, out, LG,
                                  make_double2(1.0, 0.0), g->stream));
        }
        Timer t(g, 4);
        CK(g, launch_pack_records<R>(static_cast<const C*>(g->OutP), static_cast<const C*>(g->OutD), F.L, F.M, G,
                                     g->gl_w_dev, 0.25 * F.db * F.dc, F.cell0, static_cast<C*>(dst ? dst : g->rec),
                                     g->stream));
    }
    if (!dst) {
        g->rec_member = b;
        g->rec_freq = f;
        g->rec_version = g->phasor_version;
    }
    return PSTD_OK;
}

// far field: per face, the 2-D DFT of the scaled plane phasors, C = F_c P F_b, transposed into
// the working precision with 1/(N_b N_c) folded in
template <typename R> pstd_status prepare_far(pstd_grid* g, int b, int f)
{
    pstd_status st = setup_transform(g);
    if (st != PSTD_OK) return st;
    if (g->ct_member == b && g->ct_freq == f && g->ct_version == g->phasor_version) return PSTD_OK;
    const cd scale = 1.0 / g->mem[b].inc_phasor[f];   // Eqs. scaledphsiphasor, scaleddpsiphasor
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const double2* base = g->acc + (long long)b * g->acc_freq_stride * g->acc_freq_cap + (long long)f * g->acc_freq_stride;
    C* T1 = static_cast<C*>(g->T1);
    for (int fi = 0; fi < 6; ++fi) {
        const FaceGeom& F = g->faces[fi];
        for (int q = 0; q < 2; ++q) {
            Timer t(g, 4);
            const C* P = plane_in_working_precision<C>(g, base + g->face_off[fi] + q * g->face_size[fi], F);   // [Nc][Nb]
            if (!P) return PSTD_ECUDA;
            C* spec = static_cast<C*>(q == 0 ? g->specP : g->specD);
            CK(g, launch_cgemm<C>(F.Nc, F.Nb, F.Nb, P, F.Nb, static_cast<const C*>(g->Fdft[fi][0]), F.Nb, T1, F.Nb,
                                  make_double2(scale.real(), scale.imag()), g->stream));
            CK(g, launch_cgemm<C>(F.Nc, F.Nb, F.Nc, static_cast<const C*>(g->Fdft[fi][1]), F.Nc, T1, F.Nb, spec, F.Nb,
                                  make_double2(1.0, 0.0), g->stream));
        }
        Timer t(g, 4);
        CK(g, launch_spectrum_pack<R>(static_cast<const C*>(g->specP), static_cast<const C*>(g->specD), F.Nb, F.Nc,
                                      1.0 / ((double)F.Nb * F.Nc), static_cast<C*>(g->ct) + g->ct_off[fi], g->stream));
    }
    g->ct_member = b;
    g->ct_freq = f;
    g->ct_version = g->phasor_version;
    return PSTD_OK;
}

template <typename R>
pstd_status run_far(pstd_grid* g, int b, int f, const double* theta, const double* phi, long M, double2* out, double* dsdo,
                    double2* scratch, long long scratch_elems)
{
    pstd_status st = prepare_far<R>(g, b, f);
    if (st != PSTD_OK) return st;
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    FarArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.ct = static_cast<const C*>(g->ct);
    for (int fi = 0; fi < 6; ++fi) { a.ct_off[fi] = g->ct_off[fi]; a.face[fi] = g->faces[fi]; }
    a.theta = theta;
    a.phi = phi;
    a.M = M;
    a.k = wavenumber_of(g, b, f);
    // one CTA per (direction block, face) where the scratch holds six partial sums a direction:
    // six times the CTAs of the faces-summed form, so the last wave of the grid is a small
    // share of it (64980 directions: 20.1 waves of two CTAs an SM instead of 3.3); otherwise
    // each CTA sums all six faces
    a.face_split = 6LL * M <= scratch_elems ? 6 : 1;
    if ((long long)a.face_split * M > scratch_elems) return fail(g, PSTD_EINVAL, "directions exceed the scratch capacity");
    a.partial = scratch;
    {
        Timer t(g, 6);
        CK(g, launch_farfield<R>(a, g->stream));
    }
    {
        Timer t(g, 6);
        CK(g, launch_reduce_partials(scratch, a.face_split, M, out, dsdo, g->stream));
    }
    return PSTD_OK;
}

template <typename R>
pstd_status run_transform(pstd_grid* g, int b, int f, const double* pts, long M, double2* out)
{
    pstd_status st = prepare_records<R>(g, b, f);
    if (st != PSTD_OK) return st;
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    TransformArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.rec = static_cast<const C*>(g->rec);
    a.ncells = g->ncells;
    for (int fi = 0; fi < 6; ++fi) a.face[fi] = g->faces[fi];
    a.pts = pts;
    a.M = M;
    a.k = wavenumber_of(g, b, f);
    for (int q = 0; q < g->G; ++q) a.gl_node[q] = g->gl_x[q];
    const long long per_block = 128 * PSTD_TRANSFORM_PT;
    const long long blocks = (M + per_block - 1) / per_block;
    const int CH = sizeof(R) == 4 ? 32 : 16;
    const long long chunks = (g->ncells + CH - 1) / CH;
    // split the surface cells so that about four waves of resident CTAs (7 per SM) run
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->dev);
    const long long target = 4LL * 7 * nsm;
    long long splits = std::max(1LL, std::min(chunks, (target + blocks - 1) / blocks));
    splits = std::min(splits, 4096LL);
    long long cps = ((g->ncells + splits - 1) / splits + CH - 1) / CH * CH;
    splits = (g->ncells + cps - 1) / cps;
    a.cells_per_split = cps;
    st = ensure(g, &g->partial, g->partial_cap, (size_t)splits * M * sizeof(double2));
    if (st != PSTD_OK) return st;
    a.partial = g->partial;
    {
        Timer t(g, 5);
        CK(g, launch_transform<R>(a, g->G, (int)splits, g->stream));
    }
    {
        Timer t(g, 5);
        CK(g, launch_reduce_partials(g->partial, (int)splits, M, out, nullptr, g->stream));
    }
    return PSTD_OK;
}

// Several members at once: their records side by side, one transform launch whose grid's z
// extent indexes the member (each with its own wavenumber).  out: [member][M].
template <typename R>
pstd_status run_transform_group(pstd_grid* g, const int* members, const int* freqs, int count, const double* pts, long M,
                                double2* out)
{
    pstd_status st = setup_transform(g);
    if (st != PSTD_OK) return st;
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const size_t rec_elems = (size_t)g->ncells * 2 * g->G * g->G;
    st = ensure(g, &g->rec_group, g->rec_group_cap, (size_t)count * rec_elems * sizeof(C));
    if (st != PSTD_OK) return st;
    TransformArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    for (int i = 0; i < count; ++i) {
        st = prepare_records<R>(g, members[i], freqs[i], static_cast<C*>(g->rec_group) + (size_t)i * rec_elems);
        if (st != PSTD_OK) return st;
        a.km[i] = wavenumber_of(g, members[i], freqs[i]);
    }
    a.rec = static_cast<const C*>(g->rec_group);
    a.members = count;
    a.ncells = g->ncells;
    for (int fi = 0; fi < 6; ++fi) a.face[fi] = g->faces[fi];
    a.pts = pts;
    a.M = M;
    a.k = a.km[0];
    for (int q = 0; q < g->G; ++q) a.gl_node[q] = g->gl_x[q];
    const long long per_block = 128 * PSTD_TRANSFORM_PT;
    const long long blocks = (M + per_block - 1) / per_block * count;
    const int CH = sizeof(R) == 4 ? 32 : 16;
    const long long chunks = (g->ncells + CH - 1) / CH;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->dev);
    const long long target = 4LL * 7 * nsm;
    long long splits = std::max(1LL, std::min(chunks, (target + blocks - 1) / blocks));
    splits = std::min(splits, 4096LL);
    long long cps = ((g->ncells + splits - 1) / splits + CH - 1) / CH * CH;
    splits = (g->ncells + cps - 1) / cps;
    a.cells_per_split = cps;
    st = ensure(g, &g->partial, g->partial_cap, (size_t)splits * count * M * sizeof(double2));
    if (st != PSTD_OK) return st;
    a.partial = g->partial;
    {
        Timer t(g, 5);
        CK(g, launch_transform<R>(a, g->G, (int)splits, g->stream));
    }
    {
        Timer t(g, 5);
        CK(g, launch_reduce_partials(g->partial, (int)splits, (long long)count * M, out, nullptr, g->stream));
    }
    return PSTD_OK;
}

// -------------------------------------------------------------------------------------
// discrete adjoint (the transposes of the forward path; no counterpart in the paper)
// -------------------------------------------------------------------------------------
template <typename C, typename R> C make_c(R x, R y)
{
    C v;
    v.x = x;
    v.y = y;
    return v;
}

double envelope_at(const MemberHost& m, double t)
{
    return (m.ramp <= 0 || t >= m.ramp) ? 1.0 : (t <= 0 ? 0.0 : 0.5 * (1.0 - std::cos(kPi * t / m.ramp)));
}

// gradient with respect to member b's scaled phasors (phasor layout, one frequency) of a
// real loss of the transformed field at M points, given dL/dPsi there (device arrays)
template <typename R>
pstd_status run_transform_adjoint(pstd_grid* g, int b, int f, const double* pts, const double2* gpts, long M, double2* out)
{
    pstd_status st = setup_transform(g);
    if (st != PSTD_OK) return st;
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const int G = g->G, H = G / 2, REC = 2 * G * G;
    AdjointTransformArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    for (int fi = 0; fi < 6; ++fi) a.face[fi] = g->faces[fi];
    a.pts = pts;
    a.gpts = gpts;
    a.M = M;
    a.k = wavenumber_of(g, b, f);
    for (int q = 0; q < G; ++q) a.gl_node[q] = g->gl_x[q];
    a.ncells = g->ncells;
    st = ensure(g, &g->adj_table, g->adj_table_cap, (size_t)6 * M * sizeof(AdjPoint<R>));
    if (st != PSTD_OK) return st;
    a.table = static_cast<AdjPoint<R>*>(g->adj_table);
    // split the points so that about four waves of CTAs (five resident per SM) run
    long long maxitems = 0;
    for (int f = 0; f < 6; ++f) maxitems = std::max(maxitems, (long long)g->faces[f].L * g->faces[f].M * H);
    const long long ctas = 6 * ((maxitems + 127) / 128);
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->dev);
    long long splits = std::max(1LL, std::min((4LL * 5 * nsm + ctas - 1) / ctas, ((long long)M + 127) / 128));
    a.points_per_split = ((M + splits - 1) / splits + 127) / 128 * 128;
    splits = (M + a.points_per_split - 1) / a.points_per_split;
    const size_t nrec = (size_t)g->ncells * REC;
    if (!g->adj_rec && dalloc(&g->adj_rec, nrec * g->csize) != cudaSuccess) return fail(g, PSTD_ENOMEM, "adjoint records");
    if (splits > 1) {
        st = ensure(g, &g->adj_partial, g->adj_partial_cap, (size_t)splits * nrec * g->csize);
        if (st != PSTD_OK) return st;
        a.partial = static_cast<C*>(g->adj_partial);
    } else {
        a.partial = static_cast<C*>(g->adj_rec);
    }
    {
        Timer t(g, 5);
        CK(g, launch_adj_points<R>(a, g->stream));
        CK(g, launch_transform_adjoint<R>(a, G, (int)splits, g->stream));
        if (splits > 1) CK(g, launch_sum_splits<R>(a.partial, (int)splits, (long long)nrec, static_cast<C*>(g->adj_rec), g->stream));
    }
    // records -> node values -> plane gradients: P_adj = Mc^H out_adj MbT^H
    C* T1 = static_cast<C*>(g->T1);
    for (int fi = 0; fi < 6; ++fi) {
        const FaceGeom& F = g->faces[fi];
        const int LG = F.L * G, MG = F.M * G;
        Timer t(g, 4);
        CK(g, launch_unpack_records<R>(static_cast<const C*>(g->adj_rec), F.L, F.M, G, g->gl_w_dev, 0.25 * F.db * F.dc,
                                       F.cell0, static_cast<C*>(g->OutP), static_cast<C*>(g->OutD), g->stream));
        for (int q = 0; q < 2; ++q) {
            const C* oa = static_cast<const C*>(q == 0 ? g->OutP : g->OutD);
            CK(g, launch_cgemm<C>(MG, F.Nb, LG, oa, LG, static_cast<const C*>(g->MbTH[fi]), F.Nb, T1, F.Nb,
                                  make_double2(1.0, 0.0), g->stream));
            CK(g, launch_cgemm<C>(F.Nc, F.Nb, MG, static_cast<const C*>(g->McH[fi]), MG, T1, F.Nb,
                                  static_cast<C*>(g->adj_PA), F.Nb, make_double2(1.0, 0.0), g->stream));
            CK(g, launch_widen<R>(static_cast<const C*>(g->adj_PA), out + g->face_off[fi] + q * g->face_size[fi],
                                  (long long)F.Nb * F.Nc, g->stream));
        }
    }
    return PSTD_OK;
}

// dL/dV on the box [lo, hi) by the discrete adjoint of an nsteps run from rest, given gph
// (device) = dL/d(scaled phasors): for each member in order, one block per frequency of its
// window, each in the phasor layout.  The members share V, so the gradient sums their
// contributions.  The forward run is repeated with checkpoints of (psi^{n-1}, psi^n) of every
// member every K steps; each segment is then recomputed, and the adjoint levels nu of every
// member are stepped backward together with the forward kernels.
template <typename R>
pstd_status run_adjoint(pstd_grid* g, long nsteps, const double2* gph, const int lo[3], const int hi[3], long K, double* grad_out)
{
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const int B = g->batch;
    const size_t mbytes = (size_t)g->ncell * g->csize;   // one member's state
    const size_t sbytes = (size_t)B * mbytes;             // every member's state
    // incident phasors at r_O over each member's window (Eq. incpsiphasor): S[b][f]; blk[b]:
    // index of member b's first block in gph and in the injection volumes
    std::vector<std::vector<cd>> S(B);
    std::vector<int> blk(B + 1, 0);
    for (int b = 0; b < B; ++b) {
        const MemberHost& m = g->mem[b];
        S[b].assign(m.nfreq, cd(0, 0));
        for (long long n = m.first; n < m.first + m.len; ++n) {
            const double t = n * g->desc.dt;
            const cd inc = incident_at_origin(m, t, g->desc.hbar, g->desc.mass);
            for (int f = 0; f < m.nfreq; ++f) S[b][f] += inc * std::exp(cd(0.0, m.omega[f] * t));
        }
        for (int f = 0; f < m.nfreq; ++f)
            if (std::abs(S[b][f]) == 0.0) return fail(g, PSTD_ESTATE, "incident phasor at r_O is zero");
        blk[b + 1] = blk[b] + m.nfreq;
    }
    // injection volumes J_bf = (1 / S_bf) E^T conj(g_bf), one member's size each
    pstd_status st = ensure(g, &g->adj_J, g->adj_J_cap, (size_t)blk[B] * mbytes);
    if (st != PSTD_OK) return st;
    for (int b = 0; b < B; ++b)
        for (int f = 0; f < g->mem[b].nfreq; ++f) {
            InjectionArgs<R> ia;
            std::memset(&ia, 0, sizeof(ia));
            ia.g = gph + (size_t)(blk[b] + f) * g->acc_freq_stride;
            for (int i = 0; i < 6; ++i) { ia.face_off[i] = g->face_off[i]; ia.face_size[i] = g->face_size[i]; }
            for (int ax = 0; ax < 3; ++ax) {
                ia.dw[ax] = static_cast<const C*>(g->dw[ax]);
                ia.h[ax][0] = g->desc.huygens_lo[ax];
                ia.h[ax][1] = g->desc.huygens_hi[ax];
                ia.n[ax] = g->desc.n[ax];
            }
            ia.ncell = g->ncell;
            const cd sc = 1.0 / S[b][f];
            ia.scale = make_double2(sc.real(), sc.imag());
            ia.J = reinterpret_cast<C*>(static_cast<char*>(g->adj_J) + (size_t)(blk[b] + f) * mbytes);
            CK(g, launch_injection<R>(ia, g->stream));
        }
    // buffers
    if (K <= 0) K = std::max(1L, (long)std::ceil(std::sqrt((double)nsteps)));
    const long nseg = (nsteps + K - 1) / K;
    st = ensure(g, &g->adj_seg, g->adj_seg_cap, (size_t)K * sbytes);
    if (st != PSTD_OK) return st;
    st = ensure(g, &g->adj_nu, g->adj_nu_cap, 2 * sbytes);
    if (st != PSTD_OK) return st;
    const long long box = (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    st = ensure(g, &g->adj_grad, g->adj_grad_cap, (size_t)box * sizeof(double));
    if (st != PSTD_OK) return st;
    if (!g->adj_zero) {
        // zero incident time factors of every member for the adjoint steps
        CK(g, dalloc(&g->adj_zero, sizeof(double2) * PSTD_MAX_BATCH));
        CK(g, cudaMemsetAsync(g->adj_zero, 0, sizeof(double2) * PSTD_MAX_BATCH, g->stream));
    }
    char* seg = static_cast<char*>(g->adj_seg);
    // checkpoints: those pstd_step recorded for this run if they cover it, else a forward run
    // that takes them (the running DFT is left as it is)
    const bool recorded = g->ckpt_upto >= nsteps && g->ckpt_K == K && nseg <= g->ckpt_slots;
    if (!recorded) {
        st = ensure(g, &g->adj_ckpt, g->adj_ckpt_cap, (size_t)nseg * 2 * sbytes);
        if (st != PSTD_OK) return st;
        char* ck = static_cast<char*>(g->adj_ckpt);
        CK(g, cudaMemsetAsync(g->buf[0], 0, sbytes, g->stream));
        CK(g, cudaMemsetAsync(g->buf[1], 0, sbytes, g->stream));
        g->n = 0;
        g->cur = 0;
        for (long s = 0; s < nseg; ++s) {
            CK(g, cudaMemcpyAsync(ck + (size_t)(2 * s) * sbytes, g->buf[g->cur ^ 1], sbytes, cudaMemcpyDeviceToDevice, g->stream));
            CK(g, cudaMemcpyAsync(ck + (size_t)(2 * s + 1) * sbytes, g->buf[g->cur], sbytes, cudaMemcpyDeviceToDevice, g->stream));
            st = run_steps<R>(g, std::min(K, nsteps - s * K), false);
            if (st != PSTD_OK) return st;
        }
        g->ckpt_K = K;
        g->ckpt_slots = (long)(g->adj_ckpt_cap / (2 * sbytes));
        g->ckpt_upto = nsteps;
    }
    char* ckpt = static_cast<char*>(g->adj_ckpt);
    // backward
    C* nu[2] = {static_cast<C*>(g->adj_nu), reinterpret_cast<C*>(static_cast<char*>(g->adj_nu) + sbytes)};
    int nc = 0;   // nu[nc] = nu^{n+1} (current), nu[nc ^ 1] = nu^{n+2} (previous)
    CK(g, cudaMemsetAsync(g->adj_nu, 0, 2 * sbytes, g->stream));
    CK(g, cudaMemsetAsync(g->adj_grad, 0, (size_t)box * sizeof(double), g->stream));
    const bool need_src = g->vhi[0] > g->vlo[0];
    const bool exact = g->desc.tfsf_mode == PSTD_TFSF_EXACT;
    for (long s = nseg - 1; s >= 0; --s) {
        const long n0 = s * K, n1 = std::min(nsteps, n0 + K);
        // recompute u^{n0} .. u^{n1-1} into the segment buffer
        g->cur = 0;
        CK(g, cudaMemcpyAsync(g->buf[1], ckpt + (size_t)(2 * s) * sbytes, sbytes, cudaMemcpyDeviceToDevice, g->stream));
        CK(g, cudaMemcpyAsync(g->buf[0], ckpt + (size_t)(2 * s + 1) * sbytes, sbytes, cudaMemcpyDeviceToDevice, g->stream));
        CK(g, cudaMemcpyAsync(seg, g->buf[0], sbytes, cudaMemcpyDeviceToDevice, g->stream));
        g->n = n0;
        if (n1 - n0 > 1) {
            st = run_steps<R>(g, n1 - n0 - 1, false, seg);
            if (st != PSTD_OK) return st;
        }
        for (long n = n1 - 1; n >= n0; --n) {
            const double t = n * g->desc.dt;
            // dL/dV += (2 dt / hbar) Im[nu^{n+1} (u^n + psi_inc^n)]
            GradArgs<R> ga;
            std::memset(&ga, 0, sizeof(ga));
            ga.nu = nu[nc];
            ga.u = reinterpret_cast<const C*>(seg + (size_t)(n - n0) * sbytes);
            for (int ax = 0; ax < 3; ++ax) {
                ga.phase[ax] = static_cast<const C*>(g->phase[ax]);
                ga.lo[ax] = lo[ax];
                ga.hi[ax] = hi[ax];
            }
            for (int b = 0; b < B; ++b) {
                const MemberHost& m = g->mem[b];
                const cd sf = envelope_at(m, t) * std::exp(cd(0.0, -m.w0 * t));
                ga.s[b] = make_c<C>(R(sf.real()), R(sf.imag()));
            }
            ga.with_inc = exact ? 1 : 0;
            ga.batch = B;
            ga.nx = g->desc.n[0];
            ga.ny = g->desc.n[1];
            ga.nz = g->desc.n[2];
            ga.ncell = g->ncell;
            ga.c2 = 2.0 * g->desc.dt / g->desc.hbar;
            ga.grad = g->adj_grad;
            CK(g, launch_grad<R>(ga, g->stream));
            // observation term on each member's DFT-window steps: nu_b^{n+2} += sum_f e^{i w_f t_n} J_bf
            for (int b = 0; b < B; ++b) {
                const MemberHost& m = g->mem[b];
                if (n < m.first || n >= m.first + m.len) continue;
                for (int f = 0; f < m.nfreq; ++f) {
                    const cd e = std::exp(cd(0.0, m.omega[f] * t));
                    CK(g, launch_inject<R>(nu[nc ^ 1] + (size_t)b * g->ncell,
                                           reinterpret_cast<const C*>(static_cast<char*>(g->adj_J) + (size_t)(blk[b] + f) * mbytes),
                                           make_c<C>(R(e.real()), R(e.imag())), g->ncell, g->stream));
                }
            }
            // nu^n = Gamma [nu^{n+2} - (2 i dt / hbar)(eta hbar^2/2m K + V) nu^{n+1}]: the forward
            // step of every member with the EXACT V-term and no incident wave
            StepArgs<R> a = step_args<R>(g);
            a.cur = nu[nc];
            a.prev = nu[nc ^ 1];
            a.mode = PSTD_TFSF_EXACT;
            a.tfac = static_cast<const C*>(g->adj_zero);
            a.tfac_base = 0;
            a.step = 0;
            a.batch = B;
            // the tensor-copy line feeds read through maps of the grid's own level buffers, not
            // of nu: the adjoint levels take the register-fed forms
            a.tma_z = 0;
            if (a.pipe_y == PSTD_LINE_TMA) a.pipe_y = PSTD_LINE_PLAIN;
            st = enqueue_step<R>(g, a, 0, nullptr, nullptr, nullptr, need_src);
            if (st != PSTD_OK) return st;
            nc ^= 1;
        }
    }
    CK(g, cudaMemcpyAsync(grad_out, g->adj_grad, (size_t)box * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    // leave the grid at rest: state zero, step 0 (the running DFT is untouched)
    CK(g, cudaMemsetAsync(g->buf[0], 0, sbytes, g->stream));
    CK(g, cudaMemsetAsync(g->buf[1], 0, sbytes, g->stream));
    g->n = 0;
    g->cur = 0;
    g->ckpt_contig = true;
    return PSTD_OK;
}

}  // namespace

namespace pstd {

int grid_device(const pstd_grid* g) { return g->dev; }

pstd_status grid_error(pstd_grid* g, pstd_status s, const char* msg) { return fail(g, s, msg); }

// Far field of member b, frequency f, with the per-face partial sums written to a
// caller-provided device buffer of `scratch_elems` double2 entries instead of the grid's
// own: nothing is allocated.  The grid's transform buffers must already exist (they are
// created by the first pstd_transform_to_points / pstd_cross_section call on the grid).
template <typename R>
pstd_status far_field_into_scratch_r(pstd_grid* g, int b, int f, const double* theta, const double* phi, long M,
                                     double* out_dsdo, double2* out_f, double2* scratch, long long scratch_elems)
{
    if (!g->MbT[0] || !g->rec || !g->ct)
        return fail(g, PSTD_ESTATE, "surface records not set up: call pstd_cross_section or pstd_transform_to_points once first");
    return run_far<R>(g, b, f, theta, phi, M, out_f, out_dsdo, scratch, scratch_elems);
}

pstd_status far_field_into_scratch(pstd_grid* g, int b, int f, const double* theta, const double* phi, long M,
                                   double* out_dsdo, double2* out_f, double2* scratch, long long scratch_elems)
{
    DeviceGuard dg(g->dev);
    pstd_status st = check_window(g, b, f);
    if (st != PSTD_OK) return st;
    return g->prec == PSTD_F64 ? far_field_into_scratch_r<double>(g, b, f, theta, phi, M, out_dsdo, out_f, scratch, scratch_elems)
                               : far_field_into_scratch_r<float>(g, b, f, theta, phi, M, out_dsdo, out_f, scratch, scratch_elems);
}

}  // namespace pstd

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

pstd_status pstd_create_grid(const pstd_grid_desc* desc, pstd_grid** out)
{
    if (!out) return fail(nullptr, PSTD_EINVAL, "null output pointer");
    *out = nullptr;
    pstd_status st = validate(desc);
    if (st != PSTD_OK) return st;
    if (desc->dt > dt_bound(*desc, 0.0)) return fail(nullptr, PSTD_EUNSTABLE, "dt above the stability bound (Eq. PSTDstability)");
    pstd_grid* g = new pstd_grid();
    g->desc = *desc;
    if (cudaGetDevice(&g->dev) != cudaSuccess) {
        delete g;
        return fail(nullptr, PSTD_ECUDA, "no CUDA device");
    }
    g->stream = static_cast<cudaStream_t>(desc->stream);
    g->prec = desc->precision;
    // the fused x + y pass by default: one CTA per plane up to 128 points, a cluster per plane above
    if (g->prec == PSTD_F32 && xypass_available<float>(desc->n[0], desc->n[1], PSTD_XY_PLANE)) g->xy_mode = PSTD_XY_PLANE;
    else if (g->prec == PSTD_F32 && xypass_available<float>(desc->n[0], desc->n[1], PSTD_XY_CLUSTER)) g->xy_mode = PSTD_XY_CLUSTER;
    else g->xy_mode = PSTD_XY_SEPARATE;
    g->y_mode = g->prec == PSTD_F32 && pipe_y_available<float>(desc->n[1]) ? PSTD_LINE_PIPELINED : PSTD_LINE_PLAIN;
    g->rsize = g->prec == PSTD_F64 ? 8 : 4;
    g->csize = 2 * g->rsize;
    g->ncell = (long long)desc->n[0] * desc->n[1] * desc->n[2];
    g->batch = desc->batch;
    g->mem.assign(g->batch, MemberHost());
    const size_t sbytes = (size_t)g->batch * g->ncell * g->csize;
    auto cleanup_fail = [&](pstd_status s, const char* msg) {
        g_create_error = g->err.empty() ? msg : g->err;
        pstd_destroy_grid(g);
        return s;
    };
    for (int i = 0; i < 2; ++i)
        if (dalloc(&g->buf[i], sbytes) != cudaSuccess) return cleanup_fail(PSTD_ENOMEM, "state allocation failed");
    if (dalloc(&g->flag, sizeof(int)) != cudaSuccess || dalloc(&g->mem_dev, sizeof(MemberDev) * g->batch) != cudaSuccess)
        return cleanup_fail(PSTD_ENOMEM, "allocation failed");
    {
        const pstd_status ts = make_tensor_maps(g);
        if (ts != PSTD_OK) return cleanup_fail(ts, "tensor maps");
    }
    // 1-D tables (double precision on the host, rounded once to the grid precision)
    for (int a = 0; a < 3; ++a) {
        const int n = desc->n[a];
        std::vector<cd> tw(n);
        std::vector<double> kin(n), ones(n, 1.0), z, z1, z2;
        for (int m = 0; m < n; ++m) {
            tw[m] = std::exp(cd(0.0, -2.0 * kPi * m / n));
            const double km = wavenumber(n, desc->d[a], m);
            kin[m] = desc->dt * desc->hbar / desc->mass * km * km / n;
        }
        zeta_tables(*desc, a, z, z1, z2);
        // spectral-derivative weights for the two virtual planes normal to this axis
        std::vector<cd> dw(2 * (size_t)n);
        for (int s = 0; s < 2; ++s) {
            const int h = s == 0 ? desc->huygens_lo[a] : desc->huygens_hi[a];
            for (int q = 0; q < n; ++q) {
                cd acc(0, 0);
                for (int m = 0; m < n; ++m) {
                    const double km = wavenumber(n, desc->d[a], m);
                    acc += cd(0.0, km) * std::exp(cd(0.0, 2.0 * kPi * (double)m * (h - q) / n));
                }
                dw[(size_t)s * n + q] = acc / double(n);
            }
        }
        if (upload_complex(g, &g->tw[a], tw) || upload_real(g, &g->kin[a], kin) || upload_real(g, &g->mask[a], ones) ||
            upload_real(g, &g->zeta[a], z) || upload_real(g, &g->zeta1[a], z1) || upload_real(g, &g->zeta2[a], z2) ||
            upload_complex(g, &g->dw[a], dw) ||
            upload_complex(g, &g->phase[a], std::vector<cd>((size_t)n * g->batch, cd(1.0, 0.0))))
            return cleanup_fail(PSTD_ENOMEM, "table allocation failed");
    }
    // one dummy potential element so the pointer is never null
    if (upload_real(g, &g->V, std::vector<double>(1, 0.0)) != PSTD_OK) return cleanup_fail(PSTD_ENOMEM, "allocation failed");
    // face geometry for the DFT accumulators: plane sizes in face order
    long long off = 0;
    for (int f = 0; f < 6; ++f) {
        const int a = f / 2;
        const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
        g->face_size[f] = (long long)desc->n[b] * desc->n[c];
        g->face_off[f] = off;
        off += 2 * g->face_size[f];
    }
    g->acc_freq_stride = off;
    if (upload_members(g) != PSTD_OK) return cleanup_fail(PSTD_ECUDA, "member upload failed");
    pstd_status r = pstd_reset(g);
    if (r != PSTD_OK) return cleanup_fail(r, "reset failed");
    *out = g;
    return PSTD_OK;
}

pstd_status pstd_destroy_grid(pstd_grid* g)
{
    if (!g) return PSTD_OK;
    DeviceGuard dg(g->dev);
    cudaStreamSynchronize(g->stream);
    for (void* p : {g->buf[0], g->buf[1], g->V, (void*)g->mem_dev, (void*)g->acc, (void*)g->flag, (void*)g->gl_w_dev,
                    (void*)g->dft_phase, (void*)g->window_first_dev, g->tfac,
                    g->T1, g->OutP, g->OutD, g->Pw, g->rec, (void*)g->partial, (void*)g->pts_dev,
                    (void*)g->out_dev, (void*)g->dsdo_dev, g->tmaps, g->rec_group})
        if (p) cudaFree(p);
    for (int a = 0; a < 3; ++a)
        for (void* p : {g->tw[a], g->kin[a], g->mask[a], g->zeta[a], g->zeta1[a], g->zeta2[a], g->phase[a], g->dw[a]})
            if (p) cudaFree(p);
    drop_graph(g);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    for (void* p : {g->B[0], g->B[1], g->B[2]})
        if (p) cudaFree(p);
    for (int a = 0; a < 3; ++a)
        for (void* p : {g->aux_t0[a], g->aux_t1[a], g->aux_t32[a]})
            if (p) cudaFree(p);
    for (void* p : {(void*)g->aux_G0, (void*)g->aux_theta, (void*)g->aux_q, g->aux_tab, g->aux_dtab, g->aux_inc, g->aux_dinc})
        if (p) cudaFree(p);
    for (void* p : {g->tenv, g->proj[0], g->proj[1], g->proj[2]})
        if (p) cudaFree(p);
    for (void* p : {g->adj_table, g->adj_partial, g->adj_rec, g->adj_PA, (void*)g->adj_gpts, (void*)g->adj_out, g->adj_J,
                    g->adj_ckpt, g->adj_seg, g->adj_nu, g->adj_zero, (void*)g->adj_grad})
        if (p) cudaFree(p);
    for (int f = 0; f < 6; ++f) {
        if (g->MbT[f]) cudaFree(g->MbT[f]);
        if (g->Mc[f]) cudaFree(g->Mc[f]);
        if (g->MbTH[f]) cudaFree(g->MbTH[f]);
        if (g->McH[f]) cudaFree(g->McH[f]);
        for (int q = 0; q < 2; ++q)
            if (g->Fdft[f][q]) cudaFree(g->Fdft[f][q]);
    }
    for (void* p : {(void*)g->specP, (void*)g->specD, g->ct})
        if (p) cudaFree(p);
    for (auto& t : g->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    for (auto e : g->event_pool) cudaEventDestroy(e);
    delete g;
    return PSTD_OK;
}

pstd_status pstd_set_transform_order(pstd_grid* g, int G)
{
    if (!g) return fail(nullptr, PSTD_EINVAL, "null grid");
    if (G != 0 && G != 4 && G != 6 && G != 8) return fail(g, PSTD_EINVAL, "quadrature order must be 0, 4, 6 or 8");
    DeviceGuard dg(g->dev);
    const int want = G ? G : (g->prec == PSTD_F64 ? 8 : 4);
    g->G_order = G;
    if (!g->MbT[0] || want == g->G) return PSTD_OK;
    // the interpolation matrices, records and their adjoint buffers depend on G: drop them, and
    // the next transform sets them up again
    CK(g, cudaStreamSynchronize(g->stream));
    for (int f = 0; f < 6; ++f) {
        for (void** p : {&g->MbT[f], &g->Mc[f], &g->MbTH[f], &g->McH[f], &g->Fdft[f][0], &g->Fdft[f][1]}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
    }
    for (void** p : {(void**)&g->specP, (void**)&g->specD, &g->ct, &g->T1, &g->OutP, &g->OutD, &g->Pw, &g->rec, &g->adj_PA,
                     &g->adj_rec, (void**)&g->gl_w_dev, &g->rec_group}) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    g->rec_group_cap = 0;
    g->rec_member = g->ct_member = -1;
    return PSTD_OK;
}

pstd_status pstd_reset(pstd_grid* g)
{
    if (!g) return fail(nullptr, PSTD_EINVAL, "null grid");
    DeviceGuard dg(g->dev);
    const size_t sbytes = (size_t)g->batch * g->ncell * g->csize;
    CK(g, cudaMemsetAsync(g->buf[0], 0, sbytes, g->stream));
    CK(g, cudaMemsetAsync(g->buf[1], 0, sbytes, g->stream));
    CK(g, cudaMemsetAsync(g->flag, 0, sizeof(int), g->stream));
    if (g->acc) CK(g, cudaMemsetAsync(g->acc, 0, sizeof(double2) * g->acc_freq_stride * g->acc_freq_cap * g->batch, g->stream));
    for (auto& m : g->mem) {
        m.accumulated = 0;
        for (auto& p : m.inc_phasor) p = cd(0, 0);
    }
    g->n = 0;
    g->cur = 0;
    g->ckpt_contig = true;
    ++g->phasor_version;
    return PSTD_OK;
}

pstd_status pstd_set_potential(pstd_grid* g, const void* V, int mem, int dtype)
{
    if (!g || !V) return fail(g, PSTD_EINVAL, "null argument");
    DeviceGuard dg(g->dev);
    ++g->config_version;      // kernel arguments change: no graph replay of earlier runs
    g->ckpt_upto = -1;        // recorded checkpoints belong to the previous potential
    g->ckpt_contig = false;
    if (dtype != PSTD_DTYPE_F32 && dtype != PSTD_DTYPE_F64) return fail(g, PSTD_EINVAL, "dtype");
    const pstd_grid_desc& d = g->desc;
    const size_t n = (size_t)g->ncell;
    std::vector<double> h(n);
    if (mem == PSTD_MEM_HOST) {
        if (dtype == PSTD_DTYPE_F64) std::memcpy(h.data(), V, n * 8);
        else for (size_t i = 0; i < n; ++i) h[i] = static_cast<const float*>(V)[i];
    } else if (mem == PSTD_MEM_DEVICE) {
        CK(g, cudaStreamSynchronize(g->stream));
        if (dtype == PSTD_DTYPE_F64) CK(g, cudaMemcpy(h.data(), V, n * 8, cudaMemcpyDeviceToHost));
        else {
            std::vector<float> f(n);
            CK(g, cudaMemcpy(f.data(), V, n * 4, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < n; ++i) h[i] = f[i];
        }
    } else {
        return fail(g, PSTD_EINVAL, "mem");
    }
    int lo[3] = {d.n[0], d.n[1], d.n[2]}, hi[3] = {-1, -1, -1};
    double vmax = 0;
    int core_lo[3], core_hi[3];
    for (int a = 0; a < 3; ++a) {
        core_lo[a] = d.tfsf_lo[a] + d.taper_cells;
        core_hi[a] = d.tfsf_hi[a] - d.taper_cells;
    }
    for (int k = 0; k < d.n[2]; ++k)
        for (int j = 0; j < d.n[1]; ++j)
            for (int i = 0; i < d.n[0]; ++i) {
                const double v = h[((size_t)k * d.n[1] + j) * d.n[0] + i];
                if (!std::isfinite(v)) return fail(g, PSTD_EINVAL, "V is not finite");
                if (v == 0.0) continue;
                if (i < core_lo[0] || i > core_hi[0] || j < core_lo[1] || j > core_hi[1] || k < core_lo[2] || k > core_hi[2])
                    return fail(g, PSTD_EINVAL, "V must vanish outside the zeta == 1 core ((zeta - 1) V = 0)");
                lo[0] = std::min(lo[0], i); hi[0] = std::max(hi[0], i);
                lo[1] = std::min(lo[1], j); hi[1] = std::max(hi[1], j);
                lo[2] = std::min(lo[2], k); hi[2] = std::max(hi[2], k);
                vmax = std::max(vmax, std::fabs(v));
            }
    if (d.dt > dt_bound(d, vmax + std::fabs(g->gamma_b) * g->bmax))
        return fail(g, PSTD_EUNSTABLE, "dt above the stability bound with this |V|max (Eq. PSTDstability)");
    std::vector<double> box;
    if (hi[0] < 0) {   // V == 0 everywhere
        for (int a = 0; a < 3; ++a) { g->vlo[a] = 0; g->vhi[a] = 0; }
        box.assign(1, 0.0);
    } else {
        for (int a = 0; a < 3; ++a) { g->vlo[a] = lo[a]; g->vhi[a] = hi[a] + 1; }
        const int bx = g->vhi[0] - g->vlo[0], by = g->vhi[1] - g->vlo[1], bz = g->vhi[2] - g->vlo[2];
        box.resize((size_t)bx * by * bz);
        for (int k = 0; k < bz; ++k)
            for (int j = 0; j < by; ++j)
                for (int i = 0; i < bx; ++i)
                    box[((size_t)k * by + j) * bx + i] = h[((size_t)(k + lo[2]) * d.n[1] + (j + lo[1])) * d.n[0] + (i + lo[0])];
    }
    CK(g, cudaStreamSynchronize(g->stream));
    if (g->V) { cudaFree(g->V); g->V = nullptr; }
    pstd_status st = upload_real(g, &g->V, box);
    if (st != PSTD_OK) return st;
    g->vmax = vmax;
    return PSTD_OK;
}

namespace {
// direction, carrier, r_O, phase and projection tables, eta and (member 0) the absorber of an
// incident wave of member b; the envelope is set by the caller
pstd_status set_incidence_common(pstd_grid* g, int b, const double khat[3], double k)
{
    const double nrm = std::sqrt(khat[0] * khat[0] + khat[1] * khat[1] + khat[2] * khat[2]);
    if (!(k > 0) || !(nrm > 0)) return fail(g, PSTD_EINVAL, "k or khat");
    const pstd_grid_desc& d = g->desc;
    MemberHost& m = g->mem[b];
    m.has_inc = true;
    for (int a = 0; a < 3; ++a) m.khat[a] = khat[a] / nrm;
    m.k = k;
    m.E = d.hbar * d.hbar * k * k / (2.0 * d.mass);
    m.w0 = m.E / d.hbar;
    const double x = m.E * d.dt / d.hbar;
    m.eta = x == 0 ? 1.0 : std::sin(x) / x;   // Eq. numdis2
    // first-contact corner: the TF/SF box corner minimising khat . r (Eq. Oinc)
    double best = 0;
    bool first = true;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                const double c[3] = {coord(d, 0, cx ? d.tfsf_hi[0] : d.tfsf_lo[0]), coord(d, 1, cy ? d.tfsf_hi[1] : d.tfsf_lo[1]),
                                     coord(d, 2, cz ? d.tfsf_hi[2] : d.tfsf_lo[2])};
                const double v = m.khat[0] * c[0] + m.khat[1] * c[1] + m.khat[2] * c[2];
                if (first || v < best - 1e-12) {
                    best = v;
                    first = false;
                    for (int a = 0; a < 3; ++a) m.rO[a] = c[a];
                }
            }
    pstd_status st = PSTD_OK;
    for (int a = 0; a < 3; ++a) {
        const int n = d.n[a];
        std::vector<cd> ph(n);
        std::vector<double> pr(n);
        for (int i = 0; i < n; ++i) {
            pr[i] = m.khat[a] * (coord(d, a, i) - m.rO[a]);   // Eq. inc_d, one axis
            ph[i] = std::exp(cd(0.0, k * pr[i]));
        }
        st = upload_complex(g, &g->phase[a], ph, (size_t)b * n, (size_t)n * g->batch);
        if (st != PSTD_OK) return st;
        if (!g->proj[a]) CK(g, dalloc(&g->proj[a], (size_t)n * g->batch * g->rsize));
        if (g->prec == PSTD_F64) {
            CK(g, cudaMemcpy(static_cast<char*>(g->proj[a]) + (size_t)b * n * 8, pr.data(), (size_t)n * 8, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> f(pr.begin(), pr.end());
            CK(g, cudaMemcpy(static_cast<char*>(g->proj[a]) + (size_t)b * n * 4, f.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
        }
    }
    if (b == 0) {   // absorber strength is expressed in units of member 0's E / hbar
        for (int a = 0; a < 3; ++a) {
            std::vector<double> gam = absorber_gamma(d, a, m.E), msk(d.n[a]);
            for (int i = 0; i < d.n[a]; ++i) msk[i] = std::exp(-gam[i] * d.dt);
            st = upload_real(g, &g->mask[a], msk);
            if (st != PSTD_OK) return st;
        }
        g->mask_ready = true;
    }
    return PSTD_OK;
}
}  // namespace

namespace {
// Forward DFT in place, X_l = sum_j x_j e^{-2 pi i j l / n} (n a power of two; radix 2).
void fft_pow2(std::vector<cd>& a)
{
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        for (size_t i = 0; i < n; i += len)
            for (size_t j = 0; j < len / 2; ++j) {
                const cd w = std::exp(cd(0.0, -2.0 * kPi * (double)j / (double)len));
                const cd u = a[i + j], v = a[i + j + len / 2] * w;
                a[i + j] = u + v;
                a[i + j + len / 2] = u - v;
            }
    }
}

// Device tables of every aux member (slots in member order), rebuilt whenever one changes.
pstd_status rebuild_aux(pstd_grid* g)
{
    CK(g, cudaStreamSynchronize(g->stream));
    for (int a = 0; a < 3; ++a)
        for (void** p : {&g->aux_t0[a], &g->aux_t1[a], &g->aux_t32[a]}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
    for (void* p : {(void*)g->aux_G0, (void*)g->aux_theta, (void*)g->aux_q})
        if (p) cudaFree(p);
    g->aux_G0 = nullptr;
    g->aux_theta = g->aux_q = nullptr;
    g->aux_mask = 0;
    g->aux_nslot = g->aux_nm = 0;
    std::vector<int> slots;
    unsigned long long mask = 0;
    size_t nm = 0;
    for (int b = 0; b < g->batch; ++b)
        if (g->mem[b].aux) {
            mask |= 1ull << b;
            slots.push_back(b);
            nm = std::max(nm, g->mem[b].aux_G0.size());
        }
    if (slots.empty()) return PSTD_OK;
    nm = (nm + 31) / 32 * 32;
    const int ns = (int)slots.size();
    std::vector<double2> G0(ns * nm, make_double2(0.0, 0.0));
    std::vector<double> th(ns * nm, 0.0), q(ns * nm, 0.0);
    const pstd_grid_desc& d = g->desc;
    std::vector<cd> t0[3], t1[3], t32[3];
    for (int a = 0; a < 3; ++a) { t0[a].resize((size_t)ns * d.n[a]); t1[a] = t0[a]; t32[a] = t0[a]; }
    for (int s = 0; s < ns; ++s) {
        const MemberHost& m = g->mem[slots[s]];
        const size_t cnt = m.aux_G0.size();
        const double q0 = m.aux_q[0], dq = cnt > 1 ? m.aux_q[1] - m.aux_q[0] : m.aux_dq;
        for (size_t i = 0; i < nm; ++i) {
            const size_t k = (size_t)s * nm + i;
            if (i < cnt) {
                G0[k] = make_double2(m.aux_G0[i].real(), m.aux_G0[i].imag());
                th[k] = m.aux_theta[i];
                q[k] = m.aux_q[i];
            } else {
                q[k] = q0 + (double)i * dq;   // padding: G0 = 0
            }
        }
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < d.n[a]; ++i) {
                const double pr = m.khat[a] * (coord(d, a, i) - m.rO[a]);   // Eq. inc_d, one axis
                t0[a][(size_t)s * d.n[a] + i] = std::exp(cd(0.0, q0 * pr));
                t1[a][(size_t)s * d.n[a] + i] = std::exp(cd(0.0, dq * pr));
                t32[a][(size_t)s * d.n[a] + i] = std::exp(cd(0.0, 32.0 * dq * pr));
            }
    }
    for (int a = 0; a < 3; ++a) {
        pstd_status st = upload_complex(g, &g->aux_t0[a], t0[a]);
        if (st == PSTD_OK) st = upload_complex(g, &g->aux_t1[a], t1[a]);
        if (st == PSTD_OK) st = upload_complex(g, &g->aux_t32[a], t32[a]);
        if (st != PSTD_OK) return st;
    }
    CK(g, dalloc(&g->aux_G0, G0.size() * sizeof(double2)));
    CK(g, dalloc(&g->aux_theta, th.size() * sizeof(double)));
    CK(g, dalloc(&g->aux_q, q.size() * sizeof(double)));
    CK(g, cudaMemcpy(g->aux_G0, G0.data(), G0.size() * sizeof(double2), cudaMemcpyHostToDevice));
    CK(g, cudaMemcpy(g->aux_theta, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(g, cudaMemcpy(g->aux_q, q.data(), q.size() * sizeof(double), cudaMemcpyHostToDevice));
    g->aux_nslot = ns;
    g->aux_nm = (int)nm;
    g->aux_mask = mask;   // only now: a failure above leaves no member marked for the kernels
    return PSTD_OK;
}

// member b no longer uses the auxiliary wave
pstd_status drop_aux(pstd_grid* g, int b)
{
    if (!g->mem[b].aux) return PSTD_OK;
    g->mem[b].aux = false;
    const pstd_status st = rebuild_aux(g);
    if (st != PSTD_OK)   // no tables for the others: they are left without an incidence
        for (auto& m : g->mem)
            if (m.aux) { m.aux = false; m.has_inc = false; }
    return st;
}
}  // namespace

pstd_status pstd_set_incidence_aux(pstd_grid* g, int b, const double khat[3], double k, double d_lo, double dd, long n1,
                                   const double* psi0)
{
    if (!g || !khat || !psi0) return fail(g, PSTD_EINVAL, "null argument");
    DeviceGuard dg(g->dev);
    ++g->config_version;
    g->ckpt_upto = -1;
    g->ckpt_contig = false;
    pstd_status st = check_member(g, b);
    if (st != PSTD_OK) return st;
    if (g->spinor) return fail(g, PSTD_EINVAL, "spinor grids take pstd_set_incidence_spinor");
    if (n1 < 8 || n1 > (1L << 16) || (n1 & (n1 - 1))) return fail(g, PSTD_EINVAL, "n1 must be a power of two in [8, 65536]");
    if (!(dd > 0) || !std::isfinite(d_lo)) return fail(g, PSTD_EINVAL, "d_lo or dd");
    for (long i = 0; i < 2 * n1; ++i)
        if (!std::isfinite(psi0[i])) return fail(g, PSTD_EINVAL, "the profile is not finite");
    st = set_incidence_common(g, b, khat, k);
    if (st != PSTD_OK) return st;
    MemberHost& m = g->mem[b];
    const pstd_grid_desc& d = g->desc;
    // the axis must hold every node of the TF/SF box: d in [0, dmax] from the first-contact corner
    double dmax = 0;
    for (int c = 0; c < 8; ++c) {
        double v = 0;
        for (int a = 0; a < 3; ++a) v += m.khat[a] * (coord(d, a, (c >> a) & 1 ? d.tfsf_hi[a] : d.tfsf_lo[a]) - m.rO[a]);
        dmax = std::max(dmax, v);
    }
    if (d_lo > 0 || d_lo + (double)n1 * dd < dmax)
        return fail(g, PSTD_EINVAL, "the 1-D axis [d_lo, d_lo + n1 dd) must cover the TF/SF box, d in [0, khat . diagonal]");
    // every mode of the 1-D leapfrog must be stable: dt eta hbar q^2 / 2m <= 1 (Eq. PSTDstability, 1-D)
    const double qn = kPi / dd;
    if (d.dt * m.eta * d.hbar * qn * qn / (2.0 * d.mass) > 1.0)
        return fail(g, PSTD_EUNSTABLE, "the 1-D auxiliary axis is too fine for dt (dt eta hbar (pi/dd)^2 / 2m > 1)");
    std::vector<cd> F(n1);
    for (long i = 0; i < n1; ++i) F[i] = cd(psi0[2 * i], psi0[2 * i + 1]);
    fft_pow2(F);
    double fmax = 0;
    for (const cd& v : F) fmax = std::max(fmax, std::abs(v));
    // modes in signed order l = -n1/2 .. n1/2 - 1 (FFT index (l + n1) mod n1); keep the span of
    // those above 1e-15 (FP64) or 1e-10 (FP32) of the largest: the n1 <= 65536 dropped ones sum
    // below the working precision's rounding of psi_inc
    const double cut = (g->prec == PSTD_F64 ? 1e-15 : 1e-10) * fmax;
    long lo = n1, hi = -n1;
    for (long l = -n1 / 2; l < n1 / 2; ++l)
        if (std::abs(F[(l + n1) % n1]) > cut) { lo = std::min(lo, l); hi = std::max(hi, l); }
    if (hi < lo) lo = hi = 0;
    m.aux_G0.clear();
    m.aux_theta.clear();
    m.aux_q.clear();
    for (long l = lo; l <= hi; ++l) {
        const double ql = 2.0 * kPi * (double)l / ((double)n1 * dd);
        const double al = d.dt * m.eta * d.hbar * ql * ql / (2.0 * d.mass);
        // F_l^n = F_l^0 z^n, z = -i a + sqrt(1 - a^2) = e^{-i asin a} (the scheme's physical root;
        // psi1^{-1} is its exact backward step); the phase at d: e^{i q_l (d - d_lo)}
        m.aux_G0.push_back(F[(l + n1) % n1] / (double)n1 * std::exp(cd(0.0, -ql * d_lo)));
        m.aux_theta.push_back(std::asin(al));
        m.aux_q.push_back(ql);
    }
    m.aux_dq = 2.0 * kPi / ((double)n1 * dd);
    m.aux_dt = d.dt;
    m.aux = true;
    m.ramp = 0.0;
    m.packet = false;
    m.chi = cd(1.0, 0.0);
    g->packet_mask &= ~(1ull << b);
    st = rebuild_aux(g);
    if (st != PSTD_OK) {
        // no tables: every aux member is left without an incidence (pstd_step reports ESTATE)
        for (auto& mm : g->mem)
            if (mm.aux) { mm.aux = false; mm.has_inc = false; }
        return st;
    }
    return upload_members(g);
}

pstd_status pstd_set_incidence(pstd_grid* g, int b, const double khat[3], double k, int envelope, double ramp_time)
{
    if (!g || !khat) return fail(g, PSTD_EINVAL, "null argument");
    DeviceGuard dg(g->dev);
    ++g->config_version;      // kernel arguments change: no graph replay of earlier runs
    g->ckpt_upto = -1;        // recorded checkpoints belong to the previous incidence
    g->ckpt_contig = false;
    pstd_status st = check_member(g, b);
    if (st != PSTD_OK) return st;
    if (envelope != PSTD_ENV_CW_RAMP) return fail(g, PSTD_EINVAL, "envelope");
    if (!(ramp_time >= 0)) return fail(g, PSTD_EINVAL, "ramp_time");
    if (g->spinor) return fail(g, PSTD_EINVAL, "spinor grids take pstd_set_incidence_spinor");
    st = set_incidence_common(g, b, khat, k);
    if (st != PSTD_OK) return st;
    MemberHost& m = g->mem[b];
    m.ramp = ramp_time;
    m.packet = false;
    m.chi = cd(1.0, 0.0);
    g->packet_mask &= ~(1ull << b);
    st = drop_aux(g, b);
    if (st != PSTD_OK) return st;
    return upload_members(g);
}

pstd_status pstd_set_incidence_packet(pstd_grid* g, int b, const double khat[3], double k, double sigma, double d0)
{
    if (!g || !khat) return fail(g, PSTD_EINVAL, "null argument");
    DeviceGuard dg(g->dev);
    ++g->config_version;      // kernel arguments change: no graph replay of earlier runs
    g->ckpt_upto = -1;
    g->ckpt_contig = false;
    pstd_status st = check_member(g, b);
    if (st != PSTD_OK) return st;
    if (!(sigma > 0) || !std::isfinite(d0)) return fail(g, PSTD_EINVAL, "sigma or d0");
    if (g->desc.tfsf_mode != PSTD_TFSF_EXACT)
        return fail(g, PSTD_EINVAL, "wave-packet incidence needs the EXACT TF/SF form (V (psi + psi_inc))");
    if (g->spinor) return fail(g, PSTD_EINVAL, "spinor grids take pstd_set_incidence_spinor");
    st = set_incidence_common(g, b, khat, k);
    if (st != PSTD_OK) return st;
    MemberHost& m = g->mem[b];
    m.ramp = 0.0;
    m.packet = true;
    m.chi = cd(1.0, 0.0);
    m.sigma = sigma;
    m.d0 = d0;
    g->packet_mask |= 1ull << b;
    st = drop_aux(g, b);
    if (st != PSTD_OK) return st;
    return upload_members(g);
}

pstd_status pstd_huygens_dft(pstd_grid* g, int b, const double* omega, int nfreq, long first_step, long n_steps)
{
    if (!g) return fail(nullptr, PSTD_EINVAL, "null grid");
    DeviceGuard dg(g->dev);
    ++g->config_version;      // kernel arguments change: no graph replay of earlier runs
    if (nfreq < 0 || nfreq > PSTD_MAX_FREQ || (nfreq > 0 && !omega)) return fail(g, PSTD_EINVAL, "nfreq");
    if (first_step < 0 || n_steps < 0) return fail(g, PSTD_EINVAL, "window");
    if (b < -1 || b >= g->batch) return fail(g, PSTD_EINVAL, "batch member out of range");
    if (nfreq > g->acc_freq_cap) {
        CK(g, cudaStreamSynchronize(g->stream));
        if (g->acc) cudaFree(g->acc);
        g->acc = nullptr;
        const size_t bytes = sizeof(double2) * g->acc_freq_stride * nfreq * g->batch;
        if (dalloc(&g->acc, bytes) != cudaSuccess) return fail(g, PSTD_ENOMEM, "DFT accumulators");
        CK(g, cudaMemsetAsync(g->acc, 0, bytes, g->stream));
        g->acc_freq_cap = nfreq;
        for (auto& m : g->mem) { m.accumulated = 0; for (auto& p : m.inc_phasor) p = cd(0, 0); }
    }
    for (int mb = 0; mb < g->batch; ++mb) {
        if (b >= 0 && mb != b) continue;
        MemberHost& m = g->mem[mb];
        m.nfreq = nfreq;
        for (int f = 0; f < PSTD_MAX_FREQ; ++f) m.omega[f] = f < nfreq ? omega[f] : 0.0;
        m.first = first_step;
        m.len = n_steps;
        m.accumulated = 0;
        for (auto& p : m.inc_phasor) p = cd(0, 0);
        if (g->acc)
            CK(g, cudaMemsetAsync(g->acc + (size_t)mb * g->acc_freq_stride * g->acc_freq_cap, 0,
                                  sizeof(double2) * g->acc_freq_stride * g->acc_freq_cap, g->stream));
    }
    ++g->phasor_version;
    // e^{+i omega_f t_n} for every member, frequency and window step, in double precision
    long long len = 1;
    for (const auto& m : g->mem) len = std::max(len, m.len);
    const size_t entries = (size_t)g->batch * PSTD_MAX_FREQ * len;
    std::vector<double2> tab(entries, make_double2(0.0, 0.0));
    std::vector<long long> first(g->batch, 0);
    for (int mb = 0; mb < g->batch; ++mb) {
        const MemberHost& m = g->mem[mb];
        first[mb] = m.first;
        for (int f = 0; f < m.nfreq; ++f)
            for (long long s2 = 0; s2 < m.len; ++s2) {
                const double t = (m.first + s2) * g->desc.dt;
                tab[((size_t)mb * PSTD_MAX_FREQ + f) * len + s2] = make_double2(std::cos(m.omega[f] * t), std::sin(m.omega[f] * t));
            }
    }
    CK(g, cudaStreamSynchronize(g->stream));
    pstd_status st = ensure(g, &g->dft_phase, g->dft_phase_cap, entries * sizeof(double2));
    if (st != PSTD_OK) return st;
    if (!g->window_first_dev && dalloc(&g->window_first_dev, sizeof(long long) * g->batch) != cudaSuccess)
        return fail(g, PSTD_ENOMEM, "window table");
    CK(g, cudaMemcpy(g->dft_phase, tab.data(), entries * sizeof(double2), cudaMemcpyHostToDevice));
    CK(g, cudaMemcpy(g->window_first_dev, first.data(), sizeof(long long) * g->batch, cudaMemcpyHostToDevice));
    g->dft_phase_len = len;
    return upload_members(g);
}

pstd_status pstd_step(pstd_grid* g, long nsteps)
{
    if (!g) return fail(nullptr, PSTD_EINVAL, "null grid");
    if (nsteps < 0) return fail(g, PSTD_EINVAL, "nsteps");
    DeviceGuard dg(g->dev);
    for (int b = 0; b < g->batch; ++b)
        if (!g->mem[b].has_inc) return fail(g, PSTD_ESTATE, "every batch member needs pstd_set_incidence before stepping");
    return g->prec == PSTD_F64 ? run_steps<double>(g, nsteps) : run_steps<float>(g, nsteps);
}

pstd_status pstd_transform_to_points(pstd_grid* g, int b, int f, const double* xyz, long M, void* out_psi, int mem)
{
    if (!g || (M > 0 && (!xyz || !out_psi))) return fail(g, PSTD_EINVAL, "null argument");
    if (M < 0) return fail(g, PSTD_EINVAL, "M");
    DeviceGuard dg(g->dev);
    pstd_status st = check_window(g, b, f);
    if (st != PSTD_OK) return st;
    if (M == 0) return PSTD_OK;
    if (mem != PSTD_MEM_HOST && mem != PSTD_MEM_DEVICE) return fail(g, PSTD_EINVAL, "mem");
    const double* pts = xyz;
    double2* out = static_cast<double2*>(out_psi);
    if (mem == PSTD_MEM_HOST) {
        st = ensure(g, &g->pts_dev, g->pts_cap, sizeof(double) * 3 * M);
        if (st != PSTD_OK) return st;
        st = ensure(g, &g->out_dev, g->out_cap, sizeof(double2) * M);
        if (st != PSTD_OK) return st;
        CK(g, cudaMemcpyAsync(g->pts_dev, xyz, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, g->stream));
        pts = g->pts_dev;
        out = g->out_dev;
    }
    st = g->prec == PSTD_F64 ? run_transform<double>(g, b, f, pts, M, out) : run_transform<float>(g, b, f, pts, M, out);
    if (st != PSTD_OK) return st;
    if (mem == PSTD_MEM_HOST) return copy_out(g, out_psi, g->out_dev, sizeof(double2) * M, PSTD_MEM_HOST);
    return PSTD_OK;
}

pstd_status pstd_transform_members(pstd_grid* g, int count, const int* members, const int* freqs, const double* xyz,
                                   long M, void* out_psi, int mem)
{
    if (!g || count < 0 || (count > 0 && (!members || !freqs)) || (M > 0 && count > 0 && (!xyz || !out_psi)))
        return fail(g, PSTD_EINVAL, "null argument");
    if (M < 0) return fail(g, PSTD_EINVAL, "M");
    DeviceGuard dg(g->dev);
    for (int i = 0; i < count; ++i) {
        pstd_status st = check_window(g, members[i], freqs[i]);
        if (st != PSTD_OK) return st;
    }
    if (M == 0 || count == 0) return PSTD_OK;
    if (mem != PSTD_MEM_HOST && mem != PSTD_MEM_DEVICE) return fail(g, PSTD_EINVAL, "mem");
    const double* pts = xyz;
    double2* out = static_cast<double2*>(out_psi);
    pstd_status st;
    if (mem == PSTD_MEM_HOST) {
        st = ensure(g, &g->pts_dev, g->pts_cap, sizeof(double) * 3 * M);
        if (st != PSTD_OK) return st;
        st = ensure(g, &g->out_dev, g->out_cap, sizeof(double2) * M * count);
        if (st != PSTD_OK) return st;
        CK(g, cudaMemcpyAsync(g->pts_dev, xyz, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, g->stream));
        pts = g->pts_dev;
        out = g->out_dev;
    }
    // up to kTransformLaunchMembers members a launch, in the given order
    for (int i0 = 0; i0 < count; i0 += kTransformLaunchMembers) {
        const int n = std::min(kTransformLaunchMembers, count - i0);
        st = g->prec == PSTD_F64 ? run_transform_group<double>(g, members + i0, freqs + i0, n, pts, M, out + (size_t)i0 * M)
                                 : run_transform_group<float>(g, members + i0, freqs + i0, n, pts, M, out + (size_t)i0 * M);
        if (st != PSTD_OK) return st;
    }
    if (mem == PSTD_MEM_HOST) return copy_out(g, out_psi, g->out_dev, sizeof(double2) * M * count, PSTD_MEM_HOST);
    return PSTD_OK;
}

pstd_status pstd_cross_section(pstd_grid* g, int b, int f, const double* theta, const double* phi, long M, double* out_dsdo,
                               void* out_f, int mem)
{
    if (!g || (M > 0 && (!theta || !phi || !out_dsdo))) return fail(g, PSTD_EINVAL, "null argument");
    if (M < 0) return fail(g, PSTD_EINVAL, "M");
    DeviceGuard dg(g->dev);
    pstd_status st = check_window(g, b, f);
    if (st != PSTD_OK) return st;
    if (M == 0) return PSTD_OK;
    if (mem != PSTD_MEM_HOST && mem != PSTD_MEM_DEVICE) return fail(g, PSTD_EINVAL, "mem");
    const double *th = theta, *ph = phi;
    double2* fo = static_cast<double2*>(out_f);
    double* ds = out_dsdo;
    if (mem == PSTD_MEM_HOST) {
        st = ensure(g, &g->pts_dev, g->pts_cap, sizeof(double) * 2 * M);
        if (st != PSTD_OK) return st;
        st = ensure(g, &g->out_dev, g->out_cap, sizeof(double2) * M);
        if (st != PSTD_OK) return st;
        st = ensure(g, &g->dsdo_dev, g->dsdo_cap, sizeof(double) * M);
        if (st != PSTD_OK) return st;
        CK(g, cudaMemcpyAsync(g->pts_dev, theta, sizeof(double) * M, cudaMemcpyHostToDevice, g->stream));
        CK(g, cudaMemcpyAsync(g->pts_dev + M, phi, sizeof(double) * M, cudaMemcpyHostToDevice, g->stream));
        th = g->pts_dev;
        ph = g->pts_dev + M;
        fo = g->out_dev;
        ds = g->dsdo_dev;
    } else if (!fo) {
        st = ensure(g, &g->out_dev, g->out_cap, sizeof(double2) * M);
        if (st != PSTD_OK) return st;
        fo = g->out_dev;
    }
    st = ensure(g, &g->partial, g->partial_cap, sizeof(double2) * 6 * (size_t)M);
    if (st != PSTD_OK) return st;
    st = g->prec == PSTD_F64 ? run_far<double>(g, b, f, th, ph, M, fo, ds, g->partial, 6LL * M)
                             : run_far<float>(g, b, f, th, ph, M, fo, ds, g->partial, 6LL * M);
    if (st != PSTD_OK) return st;
    if (mem == PSTD_MEM_HOST) {
        CK(g, cudaMemcpyAsync(out_dsdo, g->dsdo_dev, sizeof(double) * M, cudaMemcpyDeviceToHost, g->stream));
        if (out_f) CK(g, cudaMemcpyAsync(out_f, g->out_dev, sizeof(double2) * M, cudaMemcpyDeviceToHost, g->stream));
        CK(g, cudaStreamSynchronize(g->stream));
    }
    return PSTD_OK;
}

pstd_status pstd_get_field(pstd_grid* g, int b, int which, void* out, int mem)
{
    if (!g || !out) return fail(g, PSTD_EINVAL, "null argument");
    DeviceGuard dg(g->dev);
    pstd_status st = check_member(g, b);
    if (st != PSTD_OK) return st;
    const size_t bytes = (size_t)g->ncell * g->csize;
    if (which == PSTD_FIELD_CURRENT || which == PSTD_FIELD_SCATTERED) {
        const char* src = static_cast<const char*>(g->buf[g->cur]) + (size_t)b * bytes;
        st = copy_out(g, out, src, bytes, mem);
        if (st != PSTD_OK || which == PSTD_FIELD_CURRENT || g->desc.tfsf_mode == PSTD_TFSF_EXACT) return st;
        // PAPER form: subtract zeta psi_inc^n on the host copy
        if (mem != PSTD_MEM_HOST) return fail(g, PSTD_EINVAL, "PSTD_FIELD_SCATTERED of the PAPER form needs host memory");
        const pstd_grid_desc& d = g->desc;
        const MemberHost& m = g->mem[b];
        std::vector<double> z[3], z1, z2;
        for (int a = 0; a < 3; ++a) zeta_tables(d, a, z[a], z1, z2);
        const double t = g->n * d.dt;
        const double env = (m.ramp <= 0 || t >= m.ramp) ? 1.0 : (t <= 0 ? 0.0 : 0.5 * (1.0 - std::cos(kPi * t / m.ramp)));
        const cd s = env * std::exp(cd(0.0, -m.w0 * t));
        std::vector<cd> Gn;   // aux members: the step's coefficients, psi_inc(d) = sum Gn_m e^{i q_m d}
        if (m.aux)
            for (size_t i = 0; i < m.aux_G0.size(); ++i) Gn.push_back(m.aux_G0[i] * std::exp(cd(0.0, -m.aux_theta[i] * (double)g->n)));
        for (int k = 0; k < d.n[2]; ++k)
            for (int j = 0; j < d.n[1]; ++j)
                for (int i = 0; i < d.n[0]; ++i) {
                    const double zz = z[0][i] * z[1][j] * z[2][k];
                    if (zz == 0.0) continue;
                    const double r[3] = {coord(d, 0, i), coord(d, 1, j), coord(d, 2, k)};
                    double dd = 0;
                    for (int a = 0; a < 3; ++a) dd += m.khat[a] * (r[a] - m.rO[a]);
                    cd v;
                    if (m.aux) {
                        cd w(0.0, 0.0);
                        for (size_t q = 0; q < Gn.size(); ++q) w += Gn[q] * std::exp(cd(0.0, m.aux_q[q] * dd));
                        v = zz * w;
                    } else {
                        v = zz * s * std::exp(cd(0.0, m.k * dd));
                    }
                    const size_t idx = ((size_t)k * d.n[1] + j) * d.n[0] + i;
                    if (g->prec == PSTD_F64) {
                        double* o = static_cast<double*>(out) + 2 * idx;
                        o[0] -= v.real(); o[1] -= v.imag();
                    } else {
                        float* o = static_cast<float*>(out) + 2 * idx;
                        o[0] -= (float)v.real(); o[1] -= (float)v.imag();
                    }
                }
        return PSTD_OK;
    }
    if (which == PSTD_FIELD_PREVIOUS) {
        const char* src = static_cast<const char*>(g->buf[g->cur ^ 1]) + (size_t)b * bytes;
        return copy_out(g, out, src, bytes, mem);
    }
    return fail(g, PSTD_EINVAL, "which");
}

pstd_status pstd_set_field(pstd_grid* g, int b, const void* prev, const void* cur, long n, int mem)
{
    if (!g || !prev || !cur) return fail(g, PSTD_EINVAL, "null argument");
    DeviceGuard dg(g->dev);
    pstd_status st = check_member(g, b);
    if (st != PSTD_OK) return st;
    if (n < 0) return fail(g, PSTD_EINVAL, "n");
    const size_t bytes = (size_t)g->ncell * g->csize;
    st = copy_in(g, static_cast<char*>(g->buf[g->cur]) + (size_t)b * bytes, cur, bytes, mem);
    if (st != PSTD_OK) return st;
    st = copy_in(g, static_cast<char*>(g->buf[g->cur ^ 1]) + (size_t)b * bytes, prev, bytes, mem);
    if (st != PSTD_OK) return st;
    g->n = n;
    g->ckpt_contig = false;   // no longer the run from rest
    ++g->phasor_version;
    if (mem == PSTD_MEM_HOST) CK(g, cudaStreamSynchronize(g->stream));
    return PSTD_OK;
}

pstd_status pstd_get_phasors(pstd_grid* g, int b, int f, void* out, int mem)
{
    if (!g || !out) return fail(g, PSTD_EINVAL, "null argument");
    DeviceGuard dg(g->dev);
    pstd_status st = check_window(g, b, f);
    if (st != PSTD_OK) return st;
    // scale on the host (small): copy raw, divide by the incident phasor at r_O
    const size_t count = (size_t)g->acc_freq_stride;
    std::vector<cd> h(count);
    const double2* src = g->acc + (size_t)b * g->acc_freq_stride * g->acc_freq_cap + (size_t)f * g->acc_freq_stride;
    CK(g, cudaMemcpyAsync(h.data(), src, count * 16, cudaMemcpyDeviceToHost, g->stream));
    CK(g, cudaStreamSynchronize(g->stream));
    const cd s = 1.0 / g->mem[b].inc_phasor[f];
    for (auto& v : h) v *= s;
    if (mem == PSTD_MEM_HOST) {
        std::memcpy(out, h.data(), count * 16);
        return PSTD_OK;
    }
    if (mem == PSTD_MEM_DEVICE) {
        CK(g, cudaMemcpyAsync(out, h.data(), count * 16, cudaMemcpyHostToDevice, g->stream));
        CK(g, cudaStreamSynchronize(g->stream));
        return PSTD_OK;
    }
    return fail(g, PSTD_EINVAL, "mem");
}

pstd_status pstd_synchronize(pstd_grid* g)
{
    if (!g) return fail(nullptr, PSTD_EINVAL, "null grid");
    DeviceGuard dg(g->dev);
    CK(g, cudaStreamSynchronize(g->stream));
    int flag = 0;
    CK(g, cudaMemcpy(&flag, g->flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag & 2) {
        CK(g, cudaMemset(g->flag, 0, sizeof(int)));
        return fail(g, PSTD_ETIMEOUT, "a step kernel gave up waiting for its tensor copies");
    }
    if (flag & 1) {
        CK(g, cudaMemset(g->flag, 0, sizeof(int)));
        return fail(g, PSTD_ENONFINITE, "the state became non-finite");
    }
    return PSTD_OK;
}

pstd_status pstd_get_step(pstd_grid* g, long* n)
{
    if (!g || !n) return fail(g, PSTD_EINVAL, "null argument");
    *n = (long)g->n;
    return PSTD_OK;
}

pstd_status pstd_get_device(pstd_grid* g, int* device)
{
    if (!g || !device) return fail(g, PSTD_EINVAL, "null argument");
    *device = g->dev;
    return PSTD_OK;
}

pstd_status pstd_stability_dt_max(const pstd_grid_desc* desc, double vmax, double* out_dt)
{
    if (!desc || !out_dt) return fail(nullptr, PSTD_EINVAL, "null argument");
    for (int a = 0; a < 3; ++a)
        if (!(desc->d[a] > 0)) return fail(nullptr, PSTD_EINVAL, "spacing");
    if (!(desc->hbar > 0) || !(desc->mass > 0)) return fail(nullptr, PSTD_EINVAL, "hbar, mass");
    *out_dt = dt_bound(*desc, vmax);
    return PSTD_OK;
}

pstd_status pstd_set_timing(pstd_grid* g, int enable)
{
    if (!g) return fail(nullptr, PSTD_EINVAL, "null grid");
    DeviceGuard dg(g->dev);
    CK(g, cudaStreamSynchronize(g->stream));
    for (auto& t : g->timed) { g->event_pool.push_back(t.a); g->event_pool.push_back(t.b); }
    g->timed.clear();
    g->timing = enable != 0;
    return PSTD_OK;
}

pstd_status pstd_kernel_stats(pstd_grid* g, int kernel_id, long* launches, double* total_ms)
{
    if (!g || !launches || !total_ms) return fail(g, PSTD_EINVAL, "null argument");
    if (kernel_id < 0 || kernel_id >= kKernelIds) return fail(g, PSTD_EINVAL, "kernel id");
    DeviceGuard dg(g->dev);
    CK(g, cudaStreamSynchronize(g->stream));
    long c = 0;
    double ms = 0;
    for (auto& t : g->timed) {
        if (t.kernel != kernel_id) continue;
        float e = 0;
        CK(g, cudaEventElapsedTime(&e, t.a, t.b));
        ms += e;
        ++c;
    }
    *launches = c;
    *total_ms = ms;
    return PSTD_OK;
}

pstd_status pstd_launch_count(pstd_grid* g, long* count)
{
    if (!g || !count) return fail(g, PSTD_EINVAL, "null argument");
    *count = (long)g->launches;
    return PSTD_OK;
}

const char* pstd_last_error(const pstd_grid* g)
{
    return g ? g->err.c_str() : g_create_error.c_str();
}

}  // extern "C"

pstd_status pstd_transform_adjoint(pstd_grid* g, int b, int f, const double* xyz, long M, const void* dl_dpsi, void* out,
                                   int mem)
{
    if (!g || !out || (M > 0 && (!xyz || !dl_dpsi))) return fail(g, PSTD_EINVAL, "null argument");
    if (M < 0) return fail(g, PSTD_EINVAL, "M");
    if (mem != PSTD_MEM_HOST && mem != PSTD_MEM_DEVICE) return fail(g, PSTD_EINVAL, "mem");
    DeviceGuard dg(g->dev);
    pstd_status st = check_member(g, b);
    if (st != PSTD_OK) return st;
    if (!g->mem[b].has_inc) return fail(g, PSTD_ESTATE, "pstd_set_incidence first (the transform needs k)");
    if (f < 0 || f >= std::max(1, g->mem[b].nfreq)) return fail(g, PSTD_EINVAL, "frequency index out of range");
    const size_t count = (size_t)g->acc_freq_stride;
    st = ensure(g, &g->adj_out, g->adj_out_cap, count * sizeof(double2));
    if (st != PSTD_OK) return st;
    CK(g, cudaMemsetAsync(g->adj_out, 0, count * sizeof(double2), g->stream));
    if (M > 0) {
        const double* pts = xyz;
        const double2* gp = static_cast<const double2*>(dl_dpsi);
        if (mem == PSTD_MEM_HOST) {
            st = ensure(g, &g->pts_dev, g->pts_cap, sizeof(double) * 3 * M);
            if (st != PSTD_OK) return st;
            st = ensure(g, &g->adj_gpts, g->adj_gpts_cap, sizeof(double2) * M);
            if (st != PSTD_OK) return st;
            CK(g, cudaMemcpyAsync(g->pts_dev, xyz, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, g->stream));
            CK(g, cudaMemcpyAsync(g->adj_gpts, dl_dpsi, sizeof(double2) * M, cudaMemcpyHostToDevice, g->stream));
            pts = g->pts_dev;
            gp = g->adj_gpts;
        }
        st = g->prec == PSTD_F64 ? run_transform_adjoint<double>(g, b, f, pts, gp, M, g->adj_out)
                                 : run_transform_adjoint<float>(g, b, f, pts, gp, M, g->adj_out);
        if (st != PSTD_OK) return st;
    }
    return copy_out(g, out, g->adj_out, count * sizeof(double2), mem);
}

pstd_status pstd_adjoint_gradient(pstd_grid* g, long nsteps, const void* dl_dphasors, const int box_lo[3],
                                  const int box_hi[3], long checkpoint_interval, double* dl_dv, int mem)
{
    if (!g || !dl_dphasors || !box_lo || !box_hi || !dl_dv) return fail(g, PSTD_EINVAL, "null argument");
    if (mem != PSTD_MEM_HOST && mem != PSTD_MEM_DEVICE) return fail(g, PSTD_EINVAL, "mem");
    if (g->spinor) return fail(g, PSTD_EINVAL, "the adjoint runs on scalar grids (no spinor coupling)");
    if (nsteps <= 0 || checkpoint_interval < 0) return fail(g, PSTD_EINVAL, "nsteps / checkpoint_interval");
    DeviceGuard dg(g->dev);
    size_t blocks = 0;
    for (int b = 0; b < g->batch; ++b) {
        const MemberHost& m = g->mem[b];
        if (!m.has_inc) return fail(g, PSTD_ESTATE, "pstd_set_incidence first (every member)");
        if (m.packet || m.aux) return fail(g, PSTD_EINVAL, "the adjoint supports the CW incidence");
        if (m.nfreq < 1 || m.len < 1)
            return fail(g, PSTD_ESTATE, "pstd_huygens_dft first, for every member (the loss is a function of the phasors)");
        if (m.first + m.len > nsteps) return fail(g, PSTD_EINVAL, "the DFT window must end within nsteps");
        blocks += (size_t)m.nfreq;
    }
    for (int a = 0; a < 3; ++a)
        if (box_lo[a] < 0 || box_hi[a] > g->desc.n[a] || box_lo[a] >= box_hi[a]) return fail(g, PSTD_EINVAL, "box");
    const size_t count = (size_t)g->acc_freq_stride * blocks;
    pstd_status st = ensure(g, &g->adj_out, g->adj_out_cap, count * sizeof(double2));
    if (st != PSTD_OK) return st;
    CK(g, cudaMemcpyAsync(g->adj_out, dl_dphasors, count * sizeof(double2),
                          mem == PSTD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->stream));
    const long long box = (long long)(box_hi[0] - box_lo[0]) * (box_hi[1] - box_lo[1]) * (box_hi[2] - box_lo[2]);
    double* dst = dl_dv;
    if (mem == PSTD_MEM_HOST) {
        st = ensure(g, &g->pts_dev, g->pts_cap, sizeof(double) * box);   // staging
        if (st != PSTD_OK) return st;
        dst = g->pts_dev;
    }
    st = g->prec == PSTD_F64 ? run_adjoint<double>(g, nsteps, g->adj_out, box_lo, box_hi, checkpoint_interval, dst)
                             : run_adjoint<float>(g, nsteps, g->adj_out, box_lo, box_hi, checkpoint_interval, dst);
    if (st != PSTD_OK) return st;
    if (mem == PSTD_MEM_HOST) return copy_out(g, dl_dv, dst, sizeof(double) * box, PSTD_MEM_HOST);
    CK(g, cudaStreamSynchronize(g->stream));
    return PSTD_OK;
}

pstd_status pstd_set_checkpointing(pstd_grid* g, long interval, long max_steps)
{
    if (!g) return fail(nullptr, PSTD_EINVAL, "null grid");
    if (interval < 0 || max_steps < 0) return fail(g, PSTD_EINVAL, "interval / max_steps");
    DeviceGuard dg(g->dev);
    ++g->config_version;      // kernel arguments change: no graph replay of earlier runs
    g->ckpt_upto = -1;
    if (interval == 0) {
        g->ckpt_record = false;
        return PSTD_OK;
    }
    const size_t sbytes = (size_t)g->batch * g->ncell * g->csize;   // both levels of every member
    const long slots = std::max(1L, (max_steps + interval - 1) / interval);
    pstd_status st = ensure(g, &g->adj_ckpt, g->adj_ckpt_cap, (size_t)slots * 2 * sbytes);
    if (st != PSTD_OK) return st;
    g->ckpt_record = true;
    g->ckpt_K = interval;
    g->ckpt_slots = (long)(g->adj_ckpt_cap / (2 * sbytes));
    return PSTD_OK;
}

pstd_status pstd_set_graphs(pstd_grid* g, int enable)
{
    if (!g) return fail(nullptr, PSTD_EINVAL, "null grid");
    DeviceGuard dg(g->dev);
    CK(g, cudaStreamSynchronize(g->stream));
    g->graphs = enable != 0;
    drop_graph(g);
    g->seen_key.valid = false;
    return PSTD_OK;
}

namespace {
bool xy_possible(const pstd_grid* g, int mode)
{
    return mode == PSTD_XY_SEPARATE || (g->prec == PSTD_F32 && xypass_available<float>(g->desc.n[0], g->desc.n[1], mode));
}
bool ymode_possible(const pstd_grid* g, int mode)
{
    if (mode == PSTD_LINE_PLAIN) return true;
    if (mode == PSTD_LINE_PIPELINED) return g->prec == PSTD_F32 && pipe_y_available<float>(g->desc.n[1]);
    if (mode == PSTD_LINE_TMA) return g->tma_y_ok;
    return false;
}
bool zmode_possible(const pstd_grid* g, int mode)
{
    return mode == PSTD_LINE_PLAIN || (mode == PSTD_LINE_TMA && g->tma_z_ok);
}
// the axes whose line length has an alternative FFT plan (FP32 grids, 128 and 256 points)
int alt_plan_axes(const pstd_grid* g)
{
    int m = 0;
    for (int ax = 0; ax < 3; ++ax)
        if (g->prec == PSTD_F32 && (g->desc.n[ax] == 128 || g->desc.n[ax] == 256)) m |= 1 << ax;
    return m;
}
}  // namespace

pstd_status pstd_set_variants(pstd_grid* g, int fused_xy, int y_pass, int z_pass, int plans)
{
    if (!g) return fail(nullptr, PSTD_EINVAL, "null grid");
    if (fused_xy < PSTD_XY_SEPARATE || fused_xy > PSTD_XY_CLUSTER || !xy_possible(g, fused_xy) || !ymode_possible(g, y_pass) ||
        !zmode_possible(g, z_pass) || (plans & ~alt_plan_axes(g)) != 0)
        return fail(g, PSTD_EINVAL, "variant not available for this grid");
    DeviceGuard dg(g->dev);
    ++g->config_version;
    g->xy_mode = fused_xy;
    g->y_mode = y_pass;
    g->tma_z = z_pass == PSTD_LINE_TMA;
    g->plans = plans;
    return PSTD_OK;
}

pstd_status pstd_autotune(pstd_grid* g, long trial_steps, int* out_variants)
{
    if (!g) return fail(nullptr, PSTD_EINVAL, "null grid");
    if (trial_steps < 1) return fail(g, PSTD_EINVAL, "trial_steps");
    DeviceGuard dg(g->dev);
    for (int b = 0; b < g->batch; ++b)
        if (!g->mem[b].has_inc) return fail(g, PSTD_ESTATE, "every batch member needs its incidence before tuning");
    // the trials step a copy of the current state (no DFT); the state is put back afterwards
    const size_t sbytes = (size_t)g->batch * g->ncell * g->csize;
    void* saved = nullptr;
    if (dalloc(&saved, 2 * sbytes) != cudaSuccess) return fail(g, PSTD_ENOMEM, "tuning copy");
    const long long n_saved = g->n;
    const int cur_saved = g->cur;
    const bool timing_saved = g->timing;
    g->timing = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pstd_status st = PSTD_OK;
    float best = -1;
    int best_xy = g->xy_mode, best_y = g->y_mode;
    bool best_z = g->tma_z;
    auto restore = [&]() -> pstd_status {
        CK(g, cudaMemcpyAsync(g->buf[0], saved, sbytes, cudaMemcpyDeviceToDevice, g->stream));
        CK(g, cudaMemcpyAsync(g->buf[1], static_cast<char*>(saved) + sbytes, sbytes, cudaMemcpyDeviceToDevice, g->stream));
        g->n = n_saved;
        g->cur = cur_saved;
        return PSTD_OK;
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = fail(g, PSTD_ECUDA, "events");
    if (st == PSTD_OK) {
        cudaMemcpyAsync(saved, g->buf[0], sbytes, cudaMemcpyDeviceToDevice, g->stream);
        cudaMemcpyAsync(static_cast<char*>(saved) + sbytes, g->buf[1], sbytes, cudaMemcpyDeviceToDevice, g->stream);
    }
    // one trial: steps of the current variants from the saved state, timed
    auto trial = [&](float* ms) -> pstd_status {
        pstd_status t = restore();
        if (t != PSTD_OK) return t;
        t = g->prec == PSTD_F64 ? run_steps<double>(g, 2, false) : run_steps<float>(g, 2, false);   // warm-up
        if (t != PSTD_OK) return t;
        cudaEventRecord(e0, g->stream);
        t = g->prec == PSTD_F64 ? run_steps<double>(g, trial_steps, false) : run_steps<float>(g, trial_steps, false);
        if (t != PSTD_OK) return t;
        cudaEventRecord(e1, g->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return fail(g, PSTD_ECUDA, "tuning events");
        cudaEventElapsedTime(ms, e0, e1);
        return PSTD_OK;
    };
    int best_plans = g->plans;
    // the pass forms with the default plans, then each axis's alternative plan with the best forms
    for (int xy = PSTD_XY_CLUSTER; xy >= PSTD_XY_SEPARATE && st == PSTD_OK; --xy)
        for (int ym = PSTD_LINE_TMA; ym >= PSTD_LINE_PLAIN && st == PSTD_OK; --ym)
        for (int zm = PSTD_LINE_TMA; zm >= PSTD_LINE_PLAIN && st == PSTD_OK; zm -= 2) {
            if (!xy_possible(g, xy) || !ymode_possible(g, ym) || !zmode_possible(g, zm)) continue;
            if (xy != PSTD_XY_SEPARATE && ym != PSTD_LINE_PLAIN) continue;   // no separate y pass to vary
            g->xy_mode = xy;
            g->y_mode = ym;
            g->tma_z = zm == PSTD_LINE_TMA;
            g->plans = 0;
            float ms = 0;
            st = trial(&ms);
            if (st != PSTD_OK) break;
            if (best < 0 || ms < best) { best = ms; best_xy = xy; best_y = ym; best_z = zm == PSTD_LINE_TMA; best_plans = 0; }
        }
    const int axes = alt_plan_axes(g);
    for (int ax = 0; ax < 3 && st == PSTD_OK; ++ax) {
        if (!((axes >> ax) & 1)) continue;
        g->xy_mode = best_xy;
        g->y_mode = best_y;
        g->tma_z = best_z;
        // the fused and register-free forms use the default plan; the x and y axes change together
        // in the cluster form
        int flip = 1 << ax;
        if (ax == 0 && best_xy == PSTD_XY_CLUSTER) flip |= 2;
        if (ax == 1 && best_xy == PSTD_XY_CLUSTER) continue;
        if (best_xy == PSTD_XY_PLANE && ax < 2) continue;
        if (ax == 1 && best_y != PSTD_LINE_PLAIN) continue;
        if (ax == 2 && best_z) continue;
        if ((flip & ~axes) != 0) continue;
        g->plans = best_plans ^ flip;
        float ms = 0;
        st = trial(&ms);
        if (st != PSTD_OK) break;
        if (ms < best) { best = ms; best_plans = g->plans; }
    }
    const pstd_status rs = restore();
    if (st == PSTD_OK) st = rs;
    CK(g, cudaStreamSynchronize(g->stream));
    cudaFree(saved);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    g->timing = timing_saved;
    g->xy_mode = best_xy;
    g->y_mode = best_y;
    g->tma_z = best_z;
    g->plans = best_plans;
    ++g->config_version;
    if (out_variants) {
        out_variants[0] = g->xy_mode;
        out_variants[1] = g->y_mode;
        out_variants[2] = g->tma_z ? PSTD_LINE_TMA : PSTD_LINE_PLAIN;
        out_variants[3] = g->plans;
    }
    return st;
}

pstd_status pstd_graph_replays(pstd_grid* g, long* count)
{
    if (!g || !count) return fail(g, PSTD_EINVAL, "null argument");
    *count = (long)g->graph_replays;
    return PSTD_OK;
}

namespace {
// a real full-grid array ([z][y][x], f32/f64, host or device) into host doubles
pstd_status read_grid_array(pstd_grid* g, const void* src, int mem, int dtype, std::vector<double>& h)
{
    const size_t n = (size_t)g->ncell;
    h.resize(n);
    if (dtype != PSTD_DTYPE_F32 && dtype != PSTD_DTYPE_F64) return fail(g, PSTD_EINVAL, "dtype");
    if (mem == PSTD_MEM_HOST) {
        if (dtype == PSTD_DTYPE_F64) std::memcpy(h.data(), src, n * 8);
        else for (size_t i = 0; i < n; ++i) h[i] = static_cast<const float*>(src)[i];
    } else if (mem == PSTD_MEM_DEVICE) {
        CK(g, cudaStreamSynchronize(g->stream));
        if (dtype == PSTD_DTYPE_F64) {
            CK(g, cudaMemcpy(h.data(), src, n * 8, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f(n);
            CK(g, cudaMemcpy(f.data(), src, n * 4, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < n; ++i) h[i] = f[i];
        }
    } else {
        return fail(g, PSTD_EINVAL, "mem");
    }
    return PSTD_OK;
}
}  // namespace

pstd_status pstd_set_magnetic_field(pstd_grid* g, const void* Bx, const void* By, const void* Bz, double gamma, int mem,
                                    int dtype)
{
    if (!g || !Bx || !By || !Bz) return fail(g, PSTD_EINVAL, "null argument");
    DeviceGuard dg(g->dev);
    ++g->config_version;
    g->ckpt_upto = -1;
    g->ckpt_contig = false;
    if (g->batch % 2) return fail(g, PSTD_EINVAL, "spinor grids pair the batch members: the batch must be even");
    if (g->desc.tfsf_mode != PSTD_TFSF_EXACT) return fail(g, PSTD_EINVAL, "spinor grids use the EXACT TF/SF form");
    if (!std::isfinite(gamma)) return fail(g, PSTD_EINVAL, "gamma");
    if (g->packet_mask || g->aux_mask) return fail(g, PSTD_EINVAL, "spinor grids take pstd_set_incidence_spinor");
    const pstd_grid_desc& d = g->desc;
    std::vector<double> h[3];
    for (int a = 0; a < 3; ++a) {
        pstd_status st = read_grid_array(g, a == 0 ? Bx : a == 1 ? By : Bz, mem, dtype, h[a]);
        if (st != PSTD_OK) return st;
    }
    int lo[3] = {d.n[0], d.n[1], d.n[2]}, hi[3] = {-1, -1, -1};
    double bmax = 0;
    for (int k = 0; k < d.n[2]; ++k)
        for (int j = 0; j < d.n[1]; ++j)
            for (int i = 0; i < d.n[0]; ++i) {
                const size_t e = ((size_t)k * d.n[1] + j) * d.n[0] + i;
                const double bx = h[0][e], by = h[1][e], bz = h[2][e];
                if (!std::isfinite(bx) || !std::isfinite(by) || !std::isfinite(bz)) return fail(g, PSTD_EINVAL, "B is not finite");
                if (bx == 0.0 && by == 0.0 && bz == 0.0) continue;
                if (i < d.tfsf_lo[0] + d.taper_cells || i > d.tfsf_hi[0] - d.taper_cells || j < d.tfsf_lo[1] + d.taper_cells ||
                    j > d.tfsf_hi[1] - d.taper_cells || k < d.tfsf_lo[2] + d.taper_cells || k > d.tfsf_hi[2] - d.taper_cells)
                    return fail(g, PSTD_EINVAL, "B must vanish outside the zeta == 1 core");
                lo[0] = std::min(lo[0], i); hi[0] = std::max(hi[0], i);
                lo[1] = std::min(lo[1], j); hi[1] = std::max(hi[1], j);
                lo[2] = std::min(lo[2], k); hi[2] = std::max(hi[2], k);
                bmax = std::max(bmax, std::sqrt(bx * bx + by * by + bz * bz));
            }
    // the eigenvalues of V + gamma sigma . B lie within |V| + |gamma| |B|
    if (d.dt > dt_bound(d, g->vmax + std::fabs(gamma) * bmax))
        return fail(g, PSTD_EUNSTABLE, "dt above the stability bound with |V|max + |gamma| |B|max (Eq. PSTDstability)");
    CK(g, cudaStreamSynchronize(g->stream));
    g->spinor = false;   // until the new field is in place (a failed upload leaves a scalar grid)
    for (int a = 0; a < 3; ++a) {
        if (g->B[a]) cudaFree(g->B[a]);
        g->B[a] = nullptr;
    }
    std::vector<double> box[3];
    if (hi[0] < 0) {
        for (int a = 0; a < 3; ++a) { g->blo[a] = 0; g->bhi[a] = 0; box[a].assign(1, 0.0); }
    } else {
        for (int a = 0; a < 3; ++a) { g->blo[a] = lo[a]; g->bhi[a] = hi[a] + 1; }
        const int bx = g->bhi[0] - g->blo[0], by = g->bhi[1] - g->blo[1], bz = g->bhi[2] - g->blo[2];
        for (int a = 0; a < 3; ++a) {
            box[a].resize((size_t)bx * by * bz);
            for (int k = 0; k < bz; ++k)
                for (int j = 0; j < by; ++j)
                    for (int i = 0; i < bx; ++i)
                        box[a][((size_t)k * by + j) * bx + i] = h[a][((size_t)(k + lo[2]) * d.n[1] + (j + lo[1])) * d.n[0] + (i + lo[0])];
        }
    }
    for (int a = 0; a < 3; ++a) {
        pstd_status st = upload_real(g, &g->B[a], box[a]);
        if (st != PSTD_OK) return st;
    }
    g->spinor = true;
    g->gamma_b = gamma;
    g->bmax = bmax;
    return PSTD_OK;
}

pstd_status pstd_set_incidence_spinor(pstd_grid* g, int p, const double khat[3], double k, double ramp_time,
                                      const double chi[4])
{
    if (!g || !khat || !chi) return fail(g, PSTD_EINVAL, "null argument");
    DeviceGuard dg(g->dev);
    ++g->config_version;
    g->ckpt_upto = -1;
    g->ckpt_contig = false;
    if (g->batch % 2 || p < 0 || 2 * p + 1 >= g->batch) return fail(g, PSTD_EINVAL, "spinor index out of range");
    if (!(ramp_time >= 0)) return fail(g, PSTD_EINVAL, "ramp_time");
    for (int c = 0; c < 2; ++c) {
        const int b = 2 * p + c;
        pstd_status st = set_incidence_common(g, b, khat, k);
        if (st != PSTD_OK) return st;
        MemberHost& m = g->mem[b];
        m.ramp = ramp_time;
        m.packet = false;
        m.chi = cd(chi[2 * c], chi[2 * c + 1]);
        g->packet_mask &= ~(1ull << b);
        st = drop_aux(g, b);
        if (st != PSTD_OK) return st;
    }
    return upload_members(g);
}
