"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds workload definitions only (grid geometry, potentials, incident
directions, observation points).  It contains none of the PSTD method's
arithmetic and imports nothing from the CUDA binding or from ``oracle/``, so both
sides of a parity test can take their inputs from here.

Units: hbar = m = 1 throughout, as in the workloads' statement.  Arrays are
indexed [z, y, x] (x fastest in memory); grid node i sits at
x_i = (i - N/2) * dx, the convention fixed by the (x + L/2) shift of the
trigonometric interpolant (Eq. AnBottomPsi).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

HBAR = 1.0
MASS = 1.0


@dataclasses.dataclass
class GridSpec:
    """Geometry and time stepping of one internal model (Section 2, Fig. model-setup).

    n, d        : grid points and spacing per axis (x, y, z)
    dt          : leapfrog time step
    abc_cells   : absorbing-layer width per axis, in cells, on both sides
    abc_profile : "poly" (gamma = gamma_max * depth^p) or "poschl_teller" (Eq. Poshcl-Teller)
    abc_param   : poly -> (p, gamma_max / (E0/hbar)); poschl_teller -> (U0 / (E0/hbar), alpha per cell)
    tfsf_lo/hi  : outer edges (grid indices) of the TF/SF transition layer per axis
    taper_cells : width of the transition layer (zeta rises over it, Eq. zeta_y)
    tfsf_mode   : "exact" (scattered-field state, source -2i dt V psi_inc) or
                  "paper" (state psi~ = psi_scat + zeta psi_inc, Eq. tildeSchrodinger)
    huygens_lo/hi : grid indices of the six virtual planes (Fig. virtual-surface)
    """

    n: tuple
    d: tuple
    dt: float
    abc_cells: tuple = (8, 8, 8)
    abc_profile: str = "poly"
    abc_param: tuple = (3.0, 5.0)
    tfsf_lo: tuple = (14, 14, 14)
    tfsf_hi: tuple = (34, 34, 34)
    taper_cells: int = 4
    tfsf_mode: str = "exact"
    huygens_lo: tuple = (11, 11, 11)
    huygens_hi: tuple = (37, 37, 37)
    hbar: float = HBAR
    mass: float = MASS
    batch: int = 1

    @property
    def shape(self):
        """numpy shape [z, y, x]."""
        return (self.n[2], self.n[1], self.n[0])

    def coords(self, axis: int) -> np.ndarray:
        n, d = self.n[axis], self.d[axis]
        return (np.arange(n) - n // 2) * d

    def core_box(self):
        """Index range [lo, hi] (inclusive) per axis where zeta == 1."""
        return [(self.tfsf_lo[a] + self.taper_cells, self.tfsf_hi[a] - self.taper_cells) for a in range(3)]


@dataclasses.dataclass
class Incidence:
    khat: tuple
    k: float
    ramp_time: float


@dataclasses.dataclass
class Workload:
    """A complete run: grid, potential, incidences, DFT window and outputs."""

    name: str
    spec: GridSpec
    V: np.ndarray
    incidences: list
    nsteps: int
    window_first: int
    window_len: int
    fresnel_points: np.ndarray | None = None   # (M, 3) observation points
    far_theta: np.ndarray | None = None        # radians
    far_phi: np.ndarray | None = None


# ----------------------------------------------------------------------------------
# potentials
# ----------------------------------------------------------------------------------

def sphere_potential(spec: GridSpec, V0: float, radius: float, centre=(0.0, 0.0, 0.0), sub: int = 8) -> np.ndarray:
    """Central square potential (Eq. sphericalV) voxelised by volume fraction.

    The paper does not say how the sphere is put on the lattice; each node gets
    V0 times the fraction of its cell (centred on the node) inside r <= radius,
    estimated on a deterministic sub x sub x sub sub-grid.
    """
    xs = [spec.coords(a) - centre[a] for a in range(3)]
    offs = (np.arange(sub) + 0.5) / sub - 0.5
    V = np.zeros(spec.shape)
    # only cells near the sphere need sub-sampling
    reach = radius + 0.5 * math.sqrt(sum(di * di for di in spec.d))
    idx = [np.nonzero(np.abs(xs[a]) <= reach)[0] for a in range(3)]
    ox, oy, oz = np.meshgrid(offs * spec.d[0], offs * spec.d[1], offs * spec.d[2], indexing="ij")
    for kk in idx[2]:
        for jj in idx[1]:
            for ii in idx[0]:
                r2 = (xs[0][ii] + ox) ** 2 + (xs[1][jj] + oy) ** 2 + (xs[2][kk] + oz) ** 2
                frac = np.count_nonzero(r2 <= radius * radius) / r2.size
                V[kk, jj, ii] = V0 * frac
    return V


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (QR of a Gaussian matrix with sign fix)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def gaussian_sum_potential(spec: GridSpec, E0: float, seed: int, count: int = 8,
                           centre_radius: float = 4.0, sigma_range=(0.3, 1.2),
                           amp_range=(-0.5, 0.5)) -> np.ndarray:
    """Sum of anisotropic Gaussians with seeded centres, widths, rotations, amplitudes.

    V = sum_g A_g exp(-1/2 (r-c_g)^T R_g S_g^-2 R_g^T (r-c_g)); A_g ~ U[amp_range]*E0,
    c_g uniform in a ball of radius centre_radius, per-axis widths ~ U[sigma_range],
    R_g uniform random rotations.  V is zeroed where |V| < 1e-8 max|V| and outside
    the zeta == 1 core, so that (zeta - 1) V = 0 holds exactly.
    """
    rng = np.random.default_rng(seed)
    x, y, z = spec.coords(0), spec.coords(1), spec.coords(2)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    P = np.stack([X, Y, Z], axis=-1)
    V = np.zeros(spec.shape)
    for _ in range(count):
        while True:
            c = rng.uniform(-centre_radius, centre_radius, 3)
            if np.dot(c, c) <= centre_radius ** 2:
                break
        sig = rng.uniform(sigma_range[0], sigma_range[1], 3)
        R = random_rotation(rng)
        A = rng.uniform(amp_range[0], amp_range[1]) * E0
        M = R @ np.diag(1.0 / sig ** 2) @ R.T
        dP = P - c
        q = np.einsum("...i,ij,...j->...", dP, M, dP)
        V += A * np.exp(-0.5 * q)
    vmax = np.max(np.abs(V))
    V[np.abs(V) < 1e-8 * vmax] = 0.0
    core = spec.core_box()
    mask = np.zeros(spec.shape, dtype=bool)
    mask[core[2][0]:core[2][1] + 1, core[1][0]:core[1][1] + 1, core[0][0]:core[0][1] + 1] = True
    V[~mask] = 0.0
    return V


# ----------------------------------------------------------------------------------
# directions and observation points
# ----------------------------------------------------------------------------------

def fibonacci_directions(count: int = 8) -> np.ndarray:
    """Fibonacci-sphere unit vectors: z_i = 1 - (2i+1)/count, phi_i = i*pi*(3 - sqrt 5)."""
    out = []
    for i in range(count):
        zc = 1.0 - (2 * i + 1) / count
        rho = math.sqrt(max(0.0, 1.0 - zc * zc))
        ph = i * math.pi * (3.0 - math.sqrt(5.0))
        out.append((rho * math.cos(ph), rho * math.sin(ph), zc))
    return np.array(out)


def seeded_direction(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def plane_points(normal, distance: float, side: float, count: int, centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """count x count points on a square plane normal to `normal`, at `distance` from `centre`."""
    nrm = np.asarray(normal, dtype=float)
    nrm = nrm / np.linalg.norm(nrm)
    helper = np.array([1.0, 0.0, 0.0]) if abs(nrm[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(nrm, helper)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(nrm, e1)
    s = (np.arange(count) + 0.5) / count * side - side / 2
    A, B = np.meshgrid(s, s, indexing="ij")
    pts = np.asarray(centre) + distance * nrm + A[..., None] * e1 + B[..., None] * e2
    return pts.reshape(-1, 3)


def z_plane_points(z: float, side: float, count: int) -> np.ndarray:
    s = (np.arange(count) + 0.5) / count * side - side / 2
    Y, X = np.meshgrid(s, s, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)


def shell_points(count: int, r_min: float, r_max: float, seed: int) -> np.ndarray:
    """Seeded points with radius uniform in [r_min, r_max] and direction uniform on the sphere."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((count, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = rng.uniform(r_min, r_max, count)
    return v * r[:, None]


def far_field_grid():
    """361 phi values (0..360 deg, 1 deg) x 180 theta values (0.5..179.5 deg)."""
    phi = np.deg2rad(np.arange(361.0))
    theta = np.deg2rad(np.arange(180) + 0.5)
    T, P = np.meshgrid(theta, phi, indexing="ij")
    return T.ravel(), P.ravel()


# ----------------------------------------------------------------------------------
# random fields for parity tests
# ----------------------------------------------------------------------------------

def random_field(shape, seed: int, dtype=np.complex128, scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return (scale * a).astype(dtype)


def random_field_c64(shape, seed: int) -> np.ndarray:
    """complex64 white noise with unit-variance real and imaginary parts, drawn in float32
    (for full-size grids, where a complex128 draw would double the host memory)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((*shape, 2), dtype=np.float32).view(np.complex64)[..., 0]


def smooth_random_field(spec: GridSpec, seed: int, kmax_frac: float = 0.5) -> np.ndarray:
    """Band-limited random complex field (modes with |k_a| <= kmax_frac * Nyquist)."""
    rng = np.random.default_rng(seed)
    shape = spec.shape
    F = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    for ax, a in ((2, 0), (1, 1), (0, 2)):
        m = np.fft.fftfreq(spec.n[a]) * 2.0  # in units of Nyquist
        keep = (np.abs(m) <= kmax_frac).astype(float)
        sh = [1, 1, 1]
        sh[ax] = -1
        F = F * keep.reshape(sh)
    u = np.fft.ifftn(F)
    return u / np.max(np.abs(u))


# ----------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------

def stable_dt(spec_n, spec_d, vmax: float, frac: float = 0.9) -> float:
    """frac times the PSTD stability bound (Eq. PSTDstability) with hbar = m = 1."""
    kin = 0.5 * math.pi ** 2 * sum(1.0 / (d * d) for d in spec_d)
    return frac / (kin + vmax)


def dft_window(E0: float, dt: float, nsteps: int, periods: int = 3):
    """Last `periods` whole carrier periods, rounded to whole steps (the whole run if shorter)."""
    M = min(int(round(periods * 2 * math.pi / (E0 * dt))), nsteps)
    return nsteps - M, M


def square_barrier_workload(n: int = 48, dx: float = 0.25, dt: float = 0.004, nsteps: int = 750,
                            ramp_steps: int = 125, vfrac: float = 0.3, radius: float = 1.5,
                            abc: int = 8, tf=(14, 34), taper: int = 4, hb=(11, 37),
                            khat=(0.0, 0.0, 1.0), with_outputs: bool = True) -> Workload:
    """Plain FP64 PSTD on a central square barrier, 48^3 (the small, fully-checked case).

    k = 2 pi along +z, V0 = 0.3 k^2/2, radius 1.5 at the grid centre, 8-cell graded
    absorber, TF/SF box over cells 14-34, Huygens box over cells 11-37.  The stated
    dt = 0.005 breaks Eq. PSTDstability at dx = 0.25 (bound 0.004119), so the run is
    made at dt = 0.004 for 750 steps with a 125-step raised-cosine ramp (the same
    physical times).
    """
    k = 2 * math.pi
    E0 = 0.5 * k * k
    spec = GridSpec(n=(n, n, n), d=(dx, dx, dx), dt=dt, abc_cells=(abc,) * 3,
                    tfsf_lo=(tf[0],) * 3, tfsf_hi=(tf[1],) * 3, taper_cells=taper,
                    huygens_lo=(hb[0],) * 3, huygens_hi=(hb[1],) * 3)
    V = sphere_potential(spec, vfrac * E0, radius)
    n0, M = dft_window(E0, dt, nsteps)
    wl = Workload(name=f"square-barrier-{n}^3", spec=spec, V=V,
                  incidences=[Incidence(tuple(khat), k, ramp_steps * dt)],
                  nsteps=nsteps, window_first=n0, window_len=M)
    if with_outputs:
        core = (tf[1] - taper - (tf[0] + taper)) * dx
        wl.fresnel_points = z_plane_points(20.0, 1.5 * core, 32)
        wl.far_theta = np.deg2rad(np.arange(181.0))
        wl.far_phi = np.zeros(181)
    return wl


def gaussian_sum_workload(n: int = 128, dx: float = 0.25, nsteps: int = 3000, seed: int = 2404,
                          abc: int = 16, tf=(24, 104), taper: int = 4, hb=(20, 108),
                          fresnel_count: int = 256, with_outputs: bool = True) -> Workload:
    """128^3 run on a seeded non-central Gaussian-sum potential (FP32 vs FP64 comparison case).

    8 anisotropic Gaussians, centres within radius 4, widths U[0.3, 1.2], random
    rotations, amplitudes U[-0.5, 0.5]*E; k = 2 pi along a seeded unit direction;
    dt = 0.9 x the stability bound; outputs: a fresnel_count^2 plane normal to khat at
    distance D^2/(4 lambda) (D = side of the zeta = 1 core), side 1.5 D, plus the
    361 x 180 far-field grid.
    """
    k = 2 * math.pi
    E0 = 0.5 * k * k
    spec = GridSpec(n=(n, n, n), d=(dx, dx, dx), dt=1.0, abc_cells=(abc,) * 3,
                    tfsf_lo=(tf[0],) * 3, tfsf_hi=(tf[1],) * 3, taper_cells=taper,
                    huygens_lo=(hb[0],) * 3, huygens_hi=(hb[1],) * 3)
    V = gaussian_sum_potential(spec, E0, seed)
    spec.dt = stable_dt(spec.n, spec.d, float(np.max(np.abs(V))))
    khat = seeded_direction(seed + 1)
    n0, M = dft_window(E0, spec.dt, nsteps)
    ramp = 0.5
    wl = Workload(name=f"gaussian-sum-{n}^3", spec=spec, V=V,
                  incidences=[Incidence(tuple(khat), k, ramp)],
                  nsteps=nsteps, window_first=n0, window_len=M)
    if with_outputs:
        D = (tf[1] - taper - (tf[0] + taper)) * dx
        lam = 2 * math.pi / k
        wl.fresnel_points = plane_points(khat, D * D / (4 * lam), 1.5 * D, fresnel_count)
        wl.far_theta, wl.far_phi = far_field_grid()
    return wl


def smoothed_noise_potential(spec: GridSpec, seed: int, block: int = 48, sigma_cells: float = 2.0,
                             amplitude: float = 1.0) -> np.ndarray:
    """Seeded Gaussian noise on the central block^3 nodes, smoothed by a Gaussian of
    sigma_cells (separable, truncated at 4 sigma), scaled so that max |V| = amplitude."""
    rng = np.random.default_rng(seed)
    V = np.zeros(spec.shape)
    lo = [spec.n[a] // 2 - block // 2 for a in range(3)]
    noise = rng.standard_normal((block, block, block))
    r = int(math.ceil(4 * sigma_cells))
    x = np.arange(-r, r + 1)
    ker = np.exp(-0.5 * (x / sigma_cells) ** 2)
    ker /= ker.sum()
    for ax in range(3):
        noise = np.apply_along_axis(lambda v: np.convolve(v, ker, mode="same"), ax, noise)
    noise *= amplitude / np.max(np.abs(noise))
    V[lo[2]:lo[2] + block, lo[1]:lo[1] + block, lo[0]:lo[0] + block] = noise
    return V


def adjoint_workload(n: int = 128, dx: float = 0.25, nsteps: int = 2000, seed: int = 2407, block: int = 48,
                     fresnel_count: int = 128, abc: int = 16, tf=(24, 104), taper: int = 4, hb=(20, 108)):
    """Inverse-scattering gradient case: V on the central block^3 from seeded smoothed noise
    (sigma 2 cells, amplitude 0.2 E), k = 2 pi along a seeded direction, dt = 0.9 x the
    stability bound; the loss is the L2 misfit of |Psi| on a fresnel_count^2 plane (normal to
    khat at D^2/(4 lambda), side 1.5 D) against the field of a second seeded potential.
    Returns (Workload, V_target); the workload's window is the last three carrier periods."""
    k = 2 * math.pi
    E0 = 0.5 * k * k
    spec = GridSpec(n=(n, n, n), d=(dx, dx, dx), dt=1.0, abc_cells=(abc,) * 3,
                    tfsf_lo=(tf[0],) * 3, tfsf_hi=(tf[1],) * 3, taper_cells=taper,
                    huygens_lo=(hb[0],) * 3, huygens_hi=(hb[1],) * 3)
    V = smoothed_noise_potential(spec, seed, block, 2.0, 0.2 * E0)
    V_target = smoothed_noise_potential(spec, seed + 100, block, 2.0, 0.2 * E0)
    spec.dt = stable_dt(spec.n, spec.d, 0.2 * E0)
    khat = seeded_direction(seed + 1)
    n0, M = dft_window(E0, spec.dt, nsteps)
    wl = Workload(name=f"adjoint-{n}^3", spec=spec, V=V, incidences=[Incidence(tuple(khat), k, 0.5)],
                  nsteps=nsteps, window_first=n0, window_len=M)
    D = (tf[1] - taper - (tf[0] + taper)) * dx
    wl.fresnel_points = plane_points(khat, D * D / (4 * (2 * math.pi / k)), 1.5 * D, fresnel_count)
    return wl, V_target


def batched_workload(n: int = 256, dx: float = 0.25, nsteps: int = 3000, seed: int = 2408, abc: int = 24,
                     tf=(40, 216), taper: int = 4, hb=(32, 224), directions: int = 8):
    """Many incidences against one potential: one seeded Gaussian-sum potential (as in
    gaussian_sum_workload, amplitudes relative to E at k = 2 pi) on an n^3 grid, and
    `directions` Fibonacci-sphere directions x k in {2 pi, pi} (2 * directions members,
    k = 2 pi first).  Each member's DFT window is the last three periods of its own carrier;
    they are returned as wl.windows = [(first, len), ...] (wl.window_* hold member 0's).

    The potential is evaluated on a 96^3 sub-box around the centre, which holds every
    Gaussian down to the 1e-8 cut, and embedded: the same values as a whole-grid evaluation."""
    k0 = 2 * math.pi
    E = 0.5 * k0 * k0
    spec = GridSpec(n=(n, n, n), d=(dx, dx, dx), dt=1.0, abc_cells=(abc,) * 3,
                    tfsf_lo=(tf[0],) * 3, tfsf_hi=(tf[1],) * 3, taper_cells=taper,
                    huygens_lo=(hb[0],) * 3, huygens_hi=(hb[1],) * 3)
    m = 96
    small = GridSpec(n=(m, m, m), d=(dx, dx, dx), dt=1.0, abc_cells=(1, 1, 1), tfsf_lo=(1, 1, 1),
                     tfsf_hi=(m - 1, m - 1, m - 1), taper_cells=1, huygens_lo=(1, 1, 1), huygens_hi=(m - 1, m - 1, m - 1))
    Vs = gaussian_sum_potential(small, E, seed)
    V = np.zeros(spec.shape)
    o = n // 2 - m // 2
    V[o:o + m, o:o + m, o:o + m] = Vs
    spec.dt = stable_dt(spec.n, spec.d, float(np.max(np.abs(V))))
    incs, windows = [], []
    for k in (k0, 0.5 * k0):
        for d in fibonacci_directions(directions):
            incs.append(Incidence(tuple(d), k, 0.5))
            windows.append(dft_window(0.5 * k * k, spec.dt, nsteps))
    wl = Workload(name=f"batched-{n}^3-x{len(incs)}", spec=spec, V=V, incidences=incs, nsteps=nsteps,
                  window_first=windows[0][0], window_len=windows[0][1])
    wl.windows = windows
    return wl


def smooth_window(r, r_in: float, r_out: float):
    """C1 radial window: 0 for r <= r_in / 2, 1 on [r_in, r_out - 1], 0 for r >= r_out, joined by
    the smoothstep t^2 (3 - 2t) over [r_in / 2, r_in] and [r_out - 1, r_out]."""
    def step(t):
        t = np.clip(t, 0.0, 1.0)
        return t * t * (3.0 - 2.0 * t)
    return step((r - 0.5 * r_in) / (0.5 * r_in)) * (1.0 - step(r - (r_out - 1.0)))


def _dipole_box(spec: GridSpec, mhat, r_in: float, r_out: float):
    """(sub-box slices [z, y, x], (Bx, By, Bz) on that box) of dipole_field."""
    m = np.asarray(mhat, dtype=float)
    m = m / np.linalg.norm(m)
    sl, xs = [], []
    for a in range(3):
        x = spec.coords(a)
        idx = np.nonzero(np.abs(x) <= r_out)[0]
        sl.append(slice(idx[0], idx[-1] + 1))
        xs.append(x[idx])
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    w = smooth_window(r, r_in, r_out)
    rs = np.where(r > 0, r, 1.0)
    mr = (m[0] * X + m[1] * Y + m[2] * Z) / rs
    box = tuple(np.where(r > 0, w * (3.0 * mr * comp / rs - m[a]) / rs ** 3, 0.0) for a, comp in enumerate((X, Y, Z)))
    return (sl[2], sl[1], sl[0]), box


def dipole_field(spec: GridSpec, mhat, r_in: float = 1.0, r_out: float = 12.0, scale: float = 1.0):
    """Point-dipole induction B = scale (3 (m . rhat) rhat - m) / r^3 of a unit moment along mhat
    at the origin, times smooth_window(r, r_in, r_out).  Evaluated on the sub-box |x_a| <= r_out
    and embedded in zeros; returns (Bx, By, Bz) as [z, y, x] float64 arrays."""
    sl, box = _dipole_box(spec, mhat, r_in, r_out)
    out = [np.zeros(spec.shape) for _ in range(3)]
    for o, b in zip(out, box):
        o[sl] = scale * b
    return tuple(out)


def spinor_workload(n: int = 384, dx: float = 0.25, nsteps: int = 6000, seed: int = 2409, abc: int = 24,
                    tf=(128, 256), taper: int = 4, hb=(120, 264), gamma: float = 1.0, strength: float = 0.5,
                    fresnel_count: int = 512, with_outputs: bool = True) -> Workload:
    """Spin-dependent scattering by a point-dipole field: H = -lap/2 + gamma sigma . B(r), V = 0.

    B is dipole_field with a seeded moment direction, cut off smoothly inside r = 1 and outside
    r = 12, scaled so that gamma |B|max = strength * E (E = k^2 / 2 at k = 2 pi).  Unpolarised
    incidence is the pair of spin states up and down along z, run as two spinors (four batch
    members) along one seeded direction; dt = 0.9 x the stability bound with |gamma B|max; the
    DFT window is the last three carrier periods.  Outputs: a fresnel_count^2 plane normal to
    khat at D^2/(4 lambda) (D = side of the zeta = 1 core), side 1.5 D, and the 361 x 180 far
    field.  wl.B, wl.gamma and wl.chis hold the field, the coupling and the spin states."""
    k = 2 * math.pi
    E0 = 0.5 * k * k
    spec = GridSpec(n=(n, n, n), d=(dx, dx, dx), dt=1.0, abc_cells=(abc,) * 3,
                    tfsf_lo=(tf[0],) * 3, tfsf_hi=(tf[1],) * 3, taper_cells=taper,
                    huygens_lo=(hb[0],) * 3, huygens_hi=(hb[1],) * 3)
    mhat = seeded_direction(seed)
    _, box = _dipole_box(spec, mhat, 1.0, 12.0)
    bmax = float(np.max(np.sqrt(box[0] ** 2 + box[1] ** 2 + box[2] ** 2)))
    B = dipole_field(spec, mhat, scale=strength * E0 / (abs(gamma) * bmax))
    spec.dt = stable_dt(spec.n, spec.d, strength * E0)
    khat = seeded_direction(seed + 1)
    n0, M = dft_window(E0, spec.dt, nsteps)
    wl = Workload(name=f"spinor-dipole-{n}^3-x2", spec=spec, V=np.zeros(spec.shape),
                  incidences=[Incidence(tuple(khat), k, 0.5)], nsteps=nsteps, window_first=n0, window_len=M)
    wl.B, wl.gamma, wl.chis = B, gamma, [(1.0, 0.0), (0.0, 1.0)]
    if with_outputs:
        D = (tf[1] - taper - (tf[0] + taper)) * dx
        lam = 2 * math.pi / k
        wl.fresnel_points = plane_points(khat, D * D / (4 * lam), 1.5 * D, fresnel_count)
        wl.far_theta, wl.far_phi = far_field_grid()
    return wl

