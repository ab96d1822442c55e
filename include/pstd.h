/*
 * pstd.h -- C ABI of the GB300 PSTD quantum-scattering library.
 *
 * The library advances the time-dependent Schroedinger equation on a 3-D grid with
 * the leapfrog pseudo-spectral time-domain (PSTD) update of Chen, "A General PSTD
 * Method to Solve Quantum Scattering in the Fresnel and Far-Field Regions by A
 * Localized Potential of Arbitrary Form" (arXiv 2403.04053), Eq. PSTDupdating,
 * injects plane waves with total-field/scattered-field sources (Section 2.2),
 * absorbs outgoing waves with a masking layer (Eqs. expmask, Gamma), accumulates
 * the running single-frequency DFT of psi and d psi/dn on six virtual planes
 * (Eqs. psiphasor, dpsiphasor) and carries it to arbitrary exterior points and to
 * the far field with the quantum surface-equivalence transform (Eqs. NTDF,
 * bottomPsi_lm ... Psi).
 *
 * Conventions
 *  - Every call returns a pstd_status.  Nothing aborts or throws across the ABI.
 *    pstd_last_error() gives a message for the most recent failure on a grid (or,
 *    with NULL, for a failed pstd_create_grid on the calling thread).
 *  - The library owns every device buffer of a grid.  The caller owns every array
 *    it passes; `mem` says whether a pointer is host (PSTD_MEM_HOST) or device
 *    (PSTD_MEM_DEVICE) memory.  Device pointers must be on the grid's device.
 *  - Calls are asynchronous on the grid's CUDA stream (pstd_grid_desc.stream,
 *    NULL = the legacy default stream) unless they return host data: calls that
 *    write host memory synchronise the stream before they return.  Device errors
 *    of an asynchronous call surface at the next synchronising call.
 *  - Host scalars and coordinates are double.  Complex arrays are interleaved
 *    (re, im).  Real-space arrays are ordered [z][y][x] (x fastest) with node i at
 *    x_i = (i - n/2) d (the convention of Eq. AnBottomPsi's (x + L/2) shift);
 *    batch members are outermost.
 *  - Units: hbar and mass are given in the descriptor; energies E = hbar^2 k^2 / 2m.
 */
#ifndef PSTD_H
#define PSTD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PSTD_OK = 0,
    PSTD_EINVAL = 1,      /* bad argument, geometry, size or call order detail */
    PSTD_ENOMEM = 2,      /* device allocation failed */
    PSTD_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    PSTD_EUNSTABLE = 4,   /* dt above the PSTD stability bound (Eq. PSTDstability) */
    PSTD_ESTATE = 5,      /* call not valid in the grid's current state */
    PSTD_ENONFINITE = 6,  /* the state became NaN/Inf (detected on the device) */
    PSTD_ETIMEOUT = 7     /* a bounded device wait gave up */
} pstd_status;

enum { PSTD_F32 = 0, PSTD_F64 = 1 };                       /* arithmetic precision of the state */
enum { PSTD_MEM_HOST = 0, PSTD_MEM_DEVICE = 1 };
enum { PSTD_DTYPE_F32 = 0, PSTD_DTYPE_F64 = 1 };
enum { PSTD_ABC_POLY = 0, PSTD_ABC_POSCHL_TELLER = 1 };     /* absorbing-layer profile */
enum { PSTD_TFSF_EXACT = 0, PSTD_TFSF_PAPER = 1 };          /* TF/SF source form */
enum { PSTD_ENV_CW_RAMP = 0 };                              /* incident-wave envelope */
enum { PSTD_FIELD_CURRENT = 0, PSTD_FIELD_PREVIOUS = 1, PSTD_FIELD_SCATTERED = 2 };
enum { PSTD_MAX_FREQ = 16, PSTD_MAX_BATCH = 64 };

typedef struct pstd_grid pstd_grid;   /* opaque */

/* Geometry of one internal model (Section 2, Fig. model-setup).
 *  n[3], d[3]      points and spacing along x, y, z.  Each n must be one of
 *                  8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384.
 *  dt, hbar, mass  leapfrog step and units.
 *  precision       PSTD_F32 (complex64 state) or PSTD_F64 (complex128 state).
 *  batch           number of incident waves advanced together against one V (1..PSTD_MAX_BATCH).
 *  abc_cells[3]    absorbing-layer width per axis (cells, both ends; 0 = periodic axis).
 *  abc_profile     PSTD_ABC_POLY: gamma = abc_param[1] (E0/hbar) * depth^abc_param[0]
 *                  PSTD_ABC_POSCHL_TELLER: gamma = abc_param[0] (E0/hbar) / cosh^2(abc_param[1] d)
 *                  (Eq. Poshcl-Teller, d in cells from the outermost surface).  E0 is the
 *                  energy of the incident wave of batch member 0.
 *  tfsf_lo/hi[3], taper_cells   outer edges of the TF/SF transition layer and its width
 *                  (zeta rises over (lo, lo + taper), Eq. zeta_y); the potential must vanish
 *                  outside the zeta == 1 core.
 *  tfsf_mode       PSTD_TFSF_EXACT: the state is the scattered field, the incident wave
 *                  enters through -2i dt V psi_inc / hbar (zero leakage at V = 0);
 *                  PSTD_TFSF_PAPER: the state is psi~ = psi_scat + zeta psi_inc and the
 *                  source of Eq. tildeSchrodinger acts in the transition layer.
 *  huygens_lo/hi[3] node indices of the six virtual planes (Fig. virtual-surface); they must
 *                  lie outside the TF/SF box and inside the absorbing layer's inner edge.
 *  stream          cudaStream_t for all work of the grid (NULL = default stream).
 */
typedef struct {
    int n[3];
    double d[3];
    double dt, hbar, mass;
    int precision;
    int batch;
    int abc_cells[3];
    int abc_profile;
    double abc_param[2];
    int tfsf_lo[3], tfsf_hi[3];
    int taper_cells;
    int tfsf_mode;
    int huygens_lo[3], huygens_hi[3];
    void* stream;
} pstd_grid_desc;

/* Validate the geometry (sizes, nesting of absorber / virtual planes / TF-SF box),
 * check dt against Eq. PSTDstability with V = 0, allocate the device state (two time
 * levels per batch member) and tables.  *out receives the new grid.
 * EINVAL bad descriptor, EUNSTABLE dt too large, ENOMEM, ECUDA. */
pstd_status pstd_create_grid(const pstd_grid_desc* desc, pstd_grid** out);

/* Free every device buffer of the grid (synchronises its stream).  NULL is accepted. */
pstd_status pstd_destroy_grid(pstd_grid* g);

/* Real potential V on the full grid, [z][y][x], dtype PSTD_DTYPE_F32/F64, host or device.
 * V must be zero where zeta < 1 ((zeta - 1) V = 0, Section 2.2.2), else EINVAL; dt must
 * satisfy Eq. PSTDstability with |V|max, else EUNSTABLE.  The library keeps V on the
 * bounding box of its support, rounded to the grid precision. */
pstd_status pstd_set_potential(pstd_grid* g, const void* V, int mem, int dtype);

/* Incident plane wave of batch member b (Eqs. khat, Oinc, inc_d):
 *   psi_inc(r, t) = a(t) exp(i k khat . (r - r_O) - i E t / hbar),  E = hbar^2 k^2 / 2m,
 * r_O the corner of the TF/SF box first met by the wavefront, a(t) the raised-cosine
 * switch-on (1 - cos(pi t / ramp_time)) / 2 for t < ramp_time (envelope PSTD_ENV_CW_RAMP).
 * Also sets the dispersion factor eta = sinc(E dt / hbar) of member b (Eq. numdis2).
 * khat need not be normalised (it is).  EINVAL for b out of range, k <= 0, khat = 0. */
pstd_status pstd_set_incidence(pstd_grid* g, int b, const double khat[3], double k, int envelope, double ramp_time);

/* Incident Gaussian wave packet of batch member b, one of the incident waves with a closed
 * form that Section 2.2.3 names (the broadband alternative to the CW wave):
 *   psi_inc(r, t) = (1 + i tau)^(-1/2) exp(-(x - v t)^2 / (4 sigma^2 (1 + i tau)) + i (k x - E t / hbar)),
 *   x = d - d0,  d = khat . (r - r_O) (Eq. inc_d),  tau = hbar t / (2 m sigma^2),  v = hbar k / m,
 * i.e. a packet of spatial width sigma whose centre starts at d0 on the incidence axis (d0 < 0:
 * before the first-contact corner r_O) and moves along khat.  The free packet in closed form
 * solves the free Schrodinger equation exactly.  eta, r_O and the phase tables are set as
 * for the CW wave (the carrier k).  Its spectrum covers E(k +- a few / sigma); the running
 * DFT's phasors at each frequency are scaled by that frequency's incident phasor at r_O
 * (Eq. incpsiphasor), so one run gives the scattering at every DFT frequency.
 * EINVAL for b out of range, k <= 0, sigma <= 0, khat = 0. */
pstd_status pstd_set_incidence_packet(pstd_grid* g, int b, const double khat[3], double k, double sigma, double d0);

/* Incidence of member b from the 1-D auxiliary wave of Section 2.2.3: a packet of any shape.
 * The free 1-D Schroedinger equation is solved along the incidence axis d = khat . (r - r_O)
 * (Eq. inc_d) by the 1-D leapfrog of Eq. PSTDupdating with this run's dt and eta(k); each node
 * reads psi_inc and d psi_inc / d d from the 1-D grid's Fourier series (Eqs. pstd_psiinc,
 * pstd_dpsiinc).  EXACT and PAPER forms.
 *   psi0   2 * n1 doubles, interleaved (re, im): the profile psi1(d_lo + m dd, t = 0), m < n1;
 *          copied; the 1-D run starts from it and from its exact backward step.
 *   n1     a power of two in [8, 65536]; the axis is periodic, [d_lo, d_lo + n1 dd).
 *   k      the carrier: eta and the default DFT frequency hbar k^2 / 2m.
 * EINVAL: the axis does not cover the TF/SF box (d_lo > 0 or d_lo + n1 dd below the box's
 * largest d), a non-finite profile, a spinor grid.  EUNSTABLE: dt eta hbar (pi/dd)^2 / 2m > 1.
 * The adjoint rejects such members (EINVAL).  Kernel id 8 times the per-step evaluation. */
pstd_status pstd_set_incidence_aux(pstd_grid* g, int b, const double khat[3], double k, double d_lo, double dd, long n1,
                                   const double* psi0);

/* Spin-dependent scattering (the paper's motivating magnetic case; the paper itself treats a
 * scalar wave function): the grid's batch members pair up as the spin-up and spin-down
 * components (2p, 2p + 1) of spinors p, coupled by W = V I + gamma sigma . B(r),
 *   sigma . B = [[Bz, Bx - i By], [Bx + i By, -Bz]],
 * in the EXACT TF/SF form (W (u + chi psi_inc)).  Bx, By, Bz: real full-grid arrays like V;
 * B must vanish where zeta < 1, and dt must satisfy Eq. PSTDstability with |V|max +
 * |gamma| |B|max (EUNSTABLE).  EINVAL for an odd batch, the PAPER form or packet members. */
pstd_status pstd_set_magnetic_field(pstd_grid* g, const void* Bx, const void* By, const void* Bz, double gamma, int mem,
                                    int dtype);

/* CW incidence of spinor p (members 2p, 2p + 1): the plane wave of pstd_set_incidence times the
 * spin state chi = (chi[0] + i chi[1], chi[2] + i chi[3]) (up, down).  Each component's phasors
 * are scaled by the scalar plane wave's incident phasor at r_O, so that the transforms give the
 * spin-resolved amplitudes (spin flip included) for the incident spin state chi. */
pstd_status pstd_set_incidence_spinor(pstd_grid* g, int p, const double khat[3], double k, double ramp_time,
                                      const double chi[4]);

/* Zero both time levels, the step counter and every DFT accumulator of all members. */
pstd_status pstd_reset(pstd_grid* g);

/* Running DFT window of member b (Eqs. psiphasor, dpsiphasor, incpsiphasor): while the
 * step index n of the current state is in [first_step, first_step + n_steps), each
 * pstd_step adds psi^n e^{i omega t_n} and (d psi^n / d a) e^{i omega t_n} on the six
 * planes to double-precision accumulators (a = the plane's normal axis, spectral
 * derivative), for each of the nfreq (<= PSTD_MAX_FREQ) angular frequencies.  Clears
 * member b's accumulators.  b = -1 configures every member. */
pstd_status pstd_huygens_dft(pstd_grid* g, int b, const double* omega, int nfreq, long first_step, long n_steps);

/* Advance every batch member by nsteps leapfrog steps (Eq. PSTDupdating with the mask
 * of Eq. expmask).  Asynchronous; ESTATE if a member has no incidence. */
pstd_status pstd_step(pstd_grid* g, long nsteps);

/* Scattered wave function at M points xyz[3*i + {0,1,2}] from the DFT of member b at
 * frequency index f, scaled by the incident phasor at r_O (Eqs. scaledphsiphasor,
 * scaleddpsiphasor), with the Green's function of that energy, k = sqrt(2 m omega_f) / hbar
 * (the carrier k at omega_f = E / hbar): the per-cell semi-analytic surface integral of Eqs. bottomPsi_lm,
 * topPsi_lm, backfrontPsi_mn, leftrightPsi_ln summed per Eq. Psi, each cell integral
 * evaluated by tensor Gauss-Legendre quadrature of the trigonometric interpolant
 * (Eq. AnBottomPsi) times the linearised Green's phase.  out_psi: M complex128.
 * `mem` applies to both xyz and out_psi.  ESTATE if the window has not completed. */
pstd_status pstd_transform_to_points(pstd_grid* g, int b, int f, const double* xyz, long M, void* out_psi, int mem);

/* The same transform for several members at once (Eq. Psi for each): out_psi[i * M + p] is
 * Psi of member members[i] at its DFT frequency freqs[i] (and that frequency's wavenumber) at
 * point p.  Up to 16 (member, frequency) pairs go into one launch over their records side by
 * side: the batched incidences of one potential share the surface geometry and the points.
 * members, freqs: count host ints; xyz (M x 3 doubles) and out_psi (count * M complex128) in
 * `mem`.  ESTATE if any member's window has not completed.  The records of a launch take
 * count * ncells * 2 G^2 working-precision values of device memory (2 GB at 256^3 x 16). */
pstd_status pstd_transform_members(pstd_grid* g, int count, const int* members, const int* freqs, const double* xyz, long M,
                                   void* out_psi, int mem);

/* Gauss-Legendre nodes per cell edge of the surface transform's cell quadrature (and of its
 * adjoint): 4, 6 or 8; 0 restores the default (4 for PSTD_F32, 8 for PSTD_F64).  Each cell
 * integral of the trigonometric interpolant times the linearised Green's phase is a G x G sum.
 * G = 8 reproduces the literal mode sum of Eq. bottomPsi_lm to round-off; G = 4 takes 60% of
 * the time of G = 6 and errs by at most 1.2e-4 on an interpolant mode at the plane's Nyquist
 * limit (far less on resolved fields: 2e-11 on the 128^3 Gaussian-sum workload).  The far field
 * (pstd_cross_section) is exact and does not depend on it.  Drops the grid's transform set-up
 * when the order changes; synchronises. */
pstd_status pstd_set_transform_order(pstd_grid* g, int G);

/* Far-field amplitude f(theta, phi) = lim r e^{-ikr} Psi(r rhat) (the r -> infinity limit of
 * the same per-cell integrals) and dsigma/dOmega = |f|^2 at M directions.  out_dsdo: M
 * doubles; out_f: M complex128 or NULL.  `mem` applies to theta, phi, out_dsdo, out_f. */
pstd_status pstd_cross_section(pstd_grid* g, int b, int f, const double* theta, const double* phi, long M,
                               double* out_dsdo, void* out_f, int mem);

/* Allocation-free variant of pstd_cross_section, for callers that cannot allocate device
 * memory once running (a fixed, fully reserved memory budget, or a latency-critical loop
 * that cannot afford an allocation or the synchronisation a free implies).  The paper has
 * no counterpart: this is a deployment convenience.  theta, phi, out_dsdo and out_f (may be
 * NULL) are DEVICE pointers on the grid's device (PSTD_EINVAL for host or other-device
 * memory, checked before any launch); M <= 1048576, else PSTD_EINVAL.  The only scratch,
 * the transform's partial sums, sits in a 16 MiB file-scope device array held until exit.
 * With CUDA's lazy module loading (the default) the array is committed on a device when
 * the first call there looks up its address: that first call can fail with PSTD_ECUDA
 * (out of memory) under a fully reserved budget, so make it at start-up, before memory is
 * reserved and before any stream capture.  Later calls allocate nothing.  All calls on a
 * device share the array and it keeps the last call's contents; calls whose kernels
 * overlap on the GPU race on it and must be serialised.  The grid's surface records must
 * exist: PSTD_ESTATE until pstd_cross_section or pstd_transform_to_points has run once on
 * the grid. */
pstd_status pstd_cross_section_noalloc(pstd_grid* g, int b, int f, const double* theta, const double* phi, long M,
                                       double* out_dsdo, void* out_f);

/* Copy a state of member b out: PSTD_FIELD_CURRENT (psi^n), PSTD_FIELD_PREVIOUS
 * (psi^{n-1}) or PSTD_FIELD_SCATTERED (psi^n minus zeta psi_inc^n in the PAPER form, the
 * state itself in the EXACT form).  out: n[0]*n[1]*n[2] complex values of the grid
 * precision (complex64 for PSTD_F32, complex128 for PSTD_F64). */
pstd_status pstd_get_field(pstd_grid* g, int b, int which, void* out, int mem);

/* Load both time levels of member b (same layout and precision as pstd_get_field) and
 * set the step index to n: checkpoint restore, and one-step parity tests. */
pstd_status pstd_set_field(pstd_grid* g, int b, const void* prev, const void* cur, long n, int mem);

/* The six scaled plane phasor pairs of member b, frequency f, as complex128, in face
 * order 2*axis + side (axis x, y, z; side 0 = low, 1 = high); each face gives its psi
 * plane then its d psi / d axis plane, each [slow][fast] over the two in-plane axes
 * (x-normal: [z][y], y-normal: [z][x], z-normal: [y][x]). */
pstd_status pstd_get_phasors(pstd_grid* g, int b, int f, void* out, int mem);

/* Wait for the grid's stream; ENONFINITE if a step produced NaN/Inf since the last check. */
pstd_status pstd_synchronize(pstd_grid* g);

/* Step index n of the current state. */
pstd_status pstd_get_step(pstd_grid* g, long* n);

/* CUDA device ordinal the grid was created on (its buffers live there). */
pstd_status pstd_get_device(pstd_grid* g, int* device);

/* Sufficient stability bound of Eq. PSTDstability for the descriptor's spacing and units. */
pstd_status pstd_stability_dt_max(const pstd_grid_desc* desc, double vmax, double* out_dt);

/* Per-kernel timing with CUDA events on the grid's stream (off by default).  Kernel ids:
 * 0 x-pass, 1 y-pass, 2 z-pass (on DFT-window steps these also accumulate the running DFT),
 * 3 fused x+y pass (FP32 square planes of 64, 96 or 128, on steps without the DFT),
 * 4 transform/node preparation, 5 point transform, 6 far field, 7 V-term and TF/SF source,
 * 8 the 1-D auxiliary incident wave (per-call coefficient table and per-step evaluation).
 * pstd_kernel_stats returns the launches and summed milliseconds since the last
 * pstd_set_timing(g, 1) (synchronises).  pstd_launch_count counts every kernel the grid
 * launched since creation. */
pstd_status pstd_set_timing(pstd_grid* g, int enable);
pstd_status pstd_kernel_stats(pstd_grid* g, int kernel_id, long* launches, double* total_ms);
pstd_status pstd_launch_count(pstd_grid* g, long* count);

/* ---- Discrete adjoint (gradients for inverse scattering) ----------------------------
 * The paper has no adjoint; these are the exact transposes of the discrete forward path
 * above, for the gradient of a real loss L with respect to the potential.  Gradient
 * convention for complex z: g = dL/dRe z + i dL/dIm z (the convention of PyTorch's
 * complex autograd), complex128 interleaved. */

/* Gradient of L with respect to member b's scaled phasors at frequency index f (the data
 * pstd_get_phasors returns, same layout), given dl_dpsi[i] = gradient of L with respect to
 * the field pstd_transform_to_points computes at xyz[3*i..3*i+2] (M complex128).  The
 * transpose of that transform (Gauss-Legendre quadrature of the trigonometric interpolant,
 * the same discretisation).  Needs only the member's incidence (its k), not a completed
 * window.  `mem` applies to xyz, dl_dpsi and out. */
pstd_status pstd_transform_adjoint(pstd_grid* g, int b, int f, const double* xyz, long M, const void* dl_dpsi, void* out,
                                   int mem);

/* dL/dV on the box [box_lo, box_hi) of grid nodes (x fastest, doubles) for a loss that is
 * a function of the scaled phasors of a run of nsteps leapfrog steps from rest, given
 * dl_dphasors = the gradient of L with respect to them: for member 0, 1, ... in order, one
 * block per frequency of the member's DFT window, each in the layout of pstd_get_phasors.
 * On a batch the members share V, so the result is the sum of their contributions (a loss
 * over several incidences).  Every member needs its CW incidence and its DFT window
 * (ESTATE), each window must end within nsteps (EINVAL); packet, auxiliary-wave and spinor
 * grids are refused (EINVAL).  The discrete adjoint of Eq. PSTDupdating with Eq. expmask:
 * the forward run is repeated with checkpoints of (psi^{n-1}, psi^n) every
 * checkpoint_interval steps (0: ceil(sqrt(nsteps))), each segment is recomputed, and the
 * adjoint levels are stepped backward with the forward kernels (the adjoint of the update
 * is its complex conjugate with no incident wave), accumulating
 * dL/dV = (2 dt/hbar) sum_b sum_n Im[nu_b^{n+1} (psi_b^n + psi_inc,b^n)] (no psi_inc in the
 * PAPER form).  Device memory: 2 ceil(nsteps/K) + K + 2 states of the whole batch plus one
 * member state per (member, frequency).  Leaves the grid at rest (state zero, step 0) with
 * its DFT sums untouched.  `mem` applies to dl_dphasors and dl_dv; synchronises. */
pstd_status pstd_adjoint_gradient(pstd_grid* g, long nsteps, const void* dl_dphasors, const int box_lo[3],
                                  const int box_hi[3], long checkpoint_interval, double* dl_dv, int mem);

/* Record adjoint checkpoints during pstd_step: from the next step taken from rest (after
 * pstd_reset), the state pair (psi^{n-1}, psi^n) is copied aside every `interval` steps, for
 * up to max_steps steps (allocated now: 2 ceil(max_steps/interval) states).  A later
 * pstd_adjoint_gradient over nsteps <= the recorded run with the same checkpoint interval then
 * uses them instead of repeating the forward run.  pstd_set_potential and pstd_set_incidence
 * discard the record; pstd_set_field stops it.  interval 0 stops recording.  A state here holds
 * every member of the batch. */
pstd_status pstd_set_checkpointing(pstd_grid* g, long interval, long max_steps);

/* CUDA-graph replay of pstd_step (on by default).  A pstd_step call that repeats the previous
 * call's first step, step count and level parity with no set-up call in between (e.g. reset +
 * step(N) per pass) is captured into a CUDA graph once and replayed from then on, instead of
 * launching its 2-4 kernels per step one by one.  Not used while per-kernel timing or
 * checkpoint recording is on; if capture is unavailable the grid falls back to direct launches.
 * enable = 0 turns it off (and drops a captured graph); synchronises. */
pstd_status pstd_set_graphs(pstd_grid* g, int enable);
/* Number of pstd_step calls of g that ran as one CUDA-graph launch. */
pstd_status pstd_graph_replays(pstd_grid* g, long* count);

/* Step-kernel variants.  fused_xy selects how the x and y transforms run:
 *   PSTD_XY_SEPARATE  1-D line passes along x, then along y (two launches);
 *   PSTD_XY_PLANE     one CTA applies K_x + K_y to a whole z plane held in shared memory
 *                     (FP32 square 64/96/128 planes);
 *   PSTD_XY_CLUSTER   a thread-block cluster of N/32 CTAs per z plane: each CTA transforms 32
 *                     rows, then, after a cluster barrier, 32 columns, the plane's second
 *                     visit served from L2 (FP32 square 128/192/256 planes).
 * y_pass (the separate y pass) and z_pass select how their lines reach the SMs on steps
 * without the running DFT:
 *   PSTD_LINE_PLAIN      each CTA loads its tile into registers (any size and precision);
 *   PSTD_LINE_PIPELINED  y only, FP32 192/256-point lines: a persistent CTA stages the next
 *                        tile with cp.async while it transforms the current one;
 *   PSTD_LINE_TMA        FP32 128/192/256-point lines: a persistent CTA streams its tiles with
 *                        tensor copies into a ring of shared-memory slots (mbarrier-completed),
 *                        several tiles in flight while one is transformed.
 * plans: bit a set = axis a's register-fed line passes use the alternative FFT plan of their
 * size (FP32, 128 and 256 points: radix 8-4-4 and 8-8-4 with twice the threads a line,
 * instead of 16-8 and 16-16); the cluster form takes one plan for x and y together.
 * All variants compute the same step.  pstd_set_variants forces them (EINVAL where a variant
 * does not exist for the grid); pstd_autotune times trial_steps steps of every available
 * combination of the pass forms from the grid's current state, then each axis's alternative
 * plan with the best forms, keeps the fastest and puts the state back (step counter
 * included; the running DFT is not touched).  out_variants (may be NULL): {fused_xy, y_pass,
 * z_pass, plans} chosen.  Both synchronise. */
enum { PSTD_XY_SEPARATE = 0, PSTD_XY_PLANE = 1, PSTD_XY_CLUSTER = 2 };
enum { PSTD_LINE_PLAIN = 0, PSTD_LINE_PIPELINED = 1, PSTD_LINE_TMA = 2 };
pstd_status pstd_set_variants(pstd_grid* g, int fused_xy, int y_pass, int z_pass, int plans);
pstd_status pstd_autotune(pstd_grid* g, long trial_steps, int* out_variants);

/* Measured fused multiply-add peak of the current device in TFLOP/s (2 flops per FMA) for
 * PSTD_F32 or PSTD_F64: independent FMA chains over every SM, best of five timed launches.
 * The roofline denominator of the library's ALU-bound kernels (the surface transform, the
 * auxiliary-wave evaluation, the FP64 passes).  Not part of the paper's method; synchronises. */
pstd_status pstd_measure_fma_peak(int precision, double* tflops);

/* Self-test of failure detection: one CTA waits, with the time-bounded mbarrier wait of the
 * TMA-fed passes, on a barrier that nothing arrives on, for limit_s seconds (0 < limit_s <= 1).
 * Returns PSTD_ETIMEOUT when the wait gave up as it must (waited_s: how long it waited), and
 * leaves the context usable.  Not part of the paper's method; synchronises. */
pstd_status pstd_selftest_bounded_wait(double limit_s, double* waited_s);

/* Message of the last failure on g (or of the last failed pstd_create_grid when g is NULL). */
const char* pstd_last_error(const pstd_grid* g);

#ifdef __cplusplus
}
#endif
#endif /* PSTD_H */
