"""FP64 CPU oracle: tables, leapfrog PSTD update and virtual-plane DFT.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path, and it imports nothing from it.

Everything here follows the paper's statement step by step, in its order, with
numpy.fft as the FFT primitive and float64/complex128 arithmetic:

  * spectral kinetic operator       Eq. spatialFFTeigen; k index range -N/2..N/2-1
                                    (the note after Eq. PSTDupdating)
  * dispersion factor eta           Eq. numdis2 (eta = sinc(E dt / hbar))
  * masking absorber                Eqs. expmask, Poshcl-Teller, Gamma
  * TF/SF taper and source          Eqs. PSTD_TF-SF, tildeSchrodinger, zeta_y, xi
  * incident plane wave             Eqs. khat, Oinc (first-contact corner), inc_d
  * leapfrog update                 Eq. PSTDupdating (written in hbar, m units)
  * stability bound                 Eq. PSTDstability
  * running DFT + scaling           Eqs. psiphasor, dpsiphasor, incpsiphasor,
                                    scaledphsiphasor, scaleddpsiphasor

Readings where the paper is silent or garbled (each also listed in the design notes):
  * grid node i sits at x_i = (i - N/2) dx (fixed by the (x + L/2) shift of Eq. AnBottomPsi);
  * the Nyquist index -N/2 is used literally: k^2 = (pi/dx)^2 and i k = -i pi/dx;
  * first-contact corner O = the corner of the TF/SF box minimising khat . r (Eq. Oinc
    as printed swaps two of its cases);
  * "exact" TF/SF form: the state is the scattered field everywhere and the incident
    wave enters only through V psi_inc, so that the injected wave is consistent with
    the grid's own operator; "paper" form: Eq. tildeSchrodinger verbatim;
  * the CW source is a raised-cosine ramp a(t) = (1 - cos(pi t / T_r)) / 2 for t < T_r;
    a wave-packet source is the free Gaussian packet in closed form along d = khat . (r - r_O);
  * initial state psi^{-1} = psi^0 = 0; step n uses psi_inc at t_n = n dt and the DFT
    of step n takes the state psi^n before it is advanced;
  * normal derivatives on the virtual planes are spectral derivatives along the
    plane's normal axis (the paper does not say how grad psi is formed).
"""
from __future__ import annotations

import math

import numpy as np

AXES_NP = {0: 2, 1: 1, 2: 0}   # physical axis (x, y, z) -> numpy axis of a [z, y, x] array


# ----------------------------------------------------------------------------------
# 1-D tables
# ----------------------------------------------------------------------------------

def coords(n: int, d: float) -> np.ndarray:
    """Node coordinates x_i = (i - N/2) d, so that x_i + L/2 = i d (Eq. AnBottomPsi)."""
    return (np.arange(n) - n // 2) * d


def wavenumbers(n: int, d: float) -> np.ndarray:
    """k_m = 2 pi m / (N d) for the FFT index order, m in -N/2..N/2-1 (note after Eq. PSTDupdating)."""
    m = np.rint(np.fft.fftfreq(n) * n)
    return 2.0 * math.pi * m / (n * d)


def eta(E0: float, dt: float, hbar: float = 1.0) -> float:
    """Phase-velocity correction eta = sinc(E0 dt / hbar), sinc(x) = sin(x)/x (Eq. numdis2)."""
    x = E0 * dt / hbar
    return 1.0 if x == 0.0 else math.sin(x) / x


def stability_dt_max(n, d, vmax: float, hbar: float = 1.0, mass: float = 1.0) -> float:
    """Sufficient PSTD stability bound on dt (Eq. PSTDstability)."""
    kin = hbar * hbar * math.pi ** 2 / (2.0 * mass) * sum(1.0 / (di * di) for di in d)
    return hbar / (kin + abs(vmax))


def absorber_gamma(n: int, width: int, profile: str, param, E0: float, hbar: float = 1.0) -> np.ndarray:
    """Absorption rate gamma(i) along one axis (units 1/time).

    "poschl_teller": gamma(d) = U0 / cosh^2(alpha d), d = distance in cells from the
    outermost surface (Eq. Poshcl-Teller), U0 given in units of E0/hbar, alpha per cell,
    zero beyond `width` cells.
    "poly": gamma = gamma_max * depth^p, depth = (cells into the layer) / width in (0, 1],
    gamma_max given in units of E0/hbar (a graded mask profile; the paper allows any
    non-negative absorbing profile).
    """
    g = np.zeros(n)
    if width <= 0:
        return g
    i = np.arange(n)
    if profile == "poly":
        p, gmax = float(param[0]), float(param[1]) * E0 / hbar
        depth = np.maximum(np.maximum(width - i, i - (n - 1 - width)), 0) / width
        g = gmax * depth ** p
    elif profile == "poschl_teller":
        U0, alpha = float(param[0]) * E0 / hbar, float(param[1])
        dist = np.minimum(i, n - 1 - i)
        g = np.where(dist < width, U0 / np.cosh(alpha * dist) ** 2, 0.0)
    else:
        raise ValueError(profile)
    return g


def mask_1d(n, width, profile, param, E0, dt, hbar=1.0) -> np.ndarray:
    """One axis factor exp(-gamma dt) of the mask Gamma (Eqs. expmask, Gamma)."""
    return np.exp(-absorber_gamma(n, width, profile, param, E0, hbar) * dt)


def xi(rho):
    """Taper xi(rho) = rho - 2/(3 pi) sin(2 pi rho) + 1/(12 pi) sin(4 pi rho) (Eq. xi)."""
    return rho - 2.0 / (3.0 * math.pi) * np.sin(2 * math.pi * rho) + 1.0 / (12.0 * math.pi) * np.sin(4 * math.pi * rho)


def dxi(rho):
    return 1.0 - 4.0 / 3.0 * np.cos(2 * math.pi * rho) + 1.0 / 3.0 * np.cos(4 * math.pi * rho)


def d2xi(rho):
    return 8.0 * math.pi / 3.0 * np.sin(2 * math.pi * rho) - 4.0 * math.pi / 3.0 * np.sin(4 * math.pi * rho)


def zeta_1d(n: int, d: float, lo: int, hi: int, taper: int):
    """zeta_a, d zeta_a/dx, d^2 zeta_a/dx^2 along one axis (Eq. zeta_y).

    y0 = x_lo, y1 = x_{lo+taper}, y2 = x_{hi-taper}, y3 = x_hi.
    """
    i = np.arange(n, dtype=float)
    z = np.zeros(n)
    z1 = np.zeros(n)
    z2 = np.zeros(n)
    w = taper * d
    rise = (i > lo) & (i < lo + taper)
    fall = (i > hi - taper) & (i < hi)
    core = (i >= lo + taper) & (i <= hi - taper)
    r = (i - lo) / taper
    z[rise] = xi(r[rise])
    z1[rise] = dxi(r[rise]) / w
    z2[rise] = d2xi(r[rise]) / (w * w)
    z[core] = 1.0
    r = (i - (hi - taper)) / taper
    z[fall] = 1.0 - xi(r[fall])
    z1[fall] = -dxi(r[fall]) / w
    z2[fall] = -d2xi(r[fall]) / (w * w)
    return z, z1, z2


def envelope(t: float, ramp_time: float) -> float:
    """CW raised-cosine switch-on a(t)."""
    if ramp_time <= 0.0 or t >= ramp_time:
        return 1.0
    if t <= 0.0:
        return 0.0
    return 0.5 * (1.0 - math.cos(math.pi * t / ramp_time))


def gaussian_packet(x, t: float, k: float, sigma: float, hbar: float = 1.0, mass: float = 1.0):
    """Free 1-D Gaussian wave packet (one of the incident waves with an analytic form that
    Section 2.2.3 names), psi(x, 0) = exp(-x^2 / (4 sigma^2) + i k x), evolved by
    i hbar d_t psi = -hbar^2/2m d_x^2 psi:
        psi(x, t) = (1 + i tau)^(-1/2) exp(-(x - v t)^2 / (4 sigma^2 (1 + i tau)) + i (k x - w t)),
    tau = hbar t / (2 m sigma^2), v = hbar k / m, w = hbar k^2 / 2m."""
    x = np.asarray(x, dtype=float)
    tau = hbar * t / (2.0 * mass * sigma * sigma)
    v = hbar * k / mass
    w = hbar * k * k / (2.0 * mass)
    q = 1.0 + 1j * tau
    return q ** -0.5 * np.exp(-(x - v * t) ** 2 / (4.0 * sigma * sigma * q) + 1j * (k * x - w * t))


def first_contact_corner(khat, spec) -> np.ndarray:
    """Corner O of the TF/SF box first met by the incident wavefront (Eq. Oinc).

    Taken as the box corner minimising khat . r; for every direction this is the
    corner Eq. Oinc intends (its cases 90 < phi <= 180 and 270 < phi < 360 print
    the y indices the wrong way round).
    """
    kh = np.asarray(khat, dtype=float)
    lo = [coords(spec.n[a], spec.d[a])[spec.tfsf_lo[a]] for a in range(3)]
    hi = [coords(spec.n[a], spec.d[a])[spec.tfsf_hi[a]] for a in range(3)]
    best, best_val = None, None
    for cz in (lo[2], hi[2]):
        for cy in (lo[1], hi[1]):
            for cx in (lo[0], hi[0]):
                c = np.array([cx, cy, cz])
                v = float(kh @ c)
                if best_val is None or v < best_val - 1e-12:
                    best, best_val = c, v
    return best


# ----------------------------------------------------------------------------------
# spectral operators
# ----------------------------------------------------------------------------------

def apply_axis(u: np.ndarray, axis: int, d: float, mult) -> np.ndarray:
    """F_a^-1[ mult(k_a) F_a[u] ] along physical axis `axis` of a [z, y, x] array."""
    ax = AXES_NP[axis]
    k = wavenumbers(u.shape[ax], d)
    shp = [1] * u.ndim
    shp[ax] = -1
    return np.fft.ifft(mult(k).reshape(shp) * np.fft.fft(u, axis=ax), axis=ax)


def kinetic(u: np.ndarray, d) -> np.ndarray:
    """K u = sum over axes of F_a^-1[k_a^2 F_a[u]] = -laplacian u (Eq. spatialFFTeigen)."""
    out = np.zeros_like(u)
    for a in range(3):
        out += apply_axis(u, a, d[a], lambda k: k * k)
    return out


def derivative(u: np.ndarray, axis: int, d: float) -> np.ndarray:
    """Spectral first derivative F_a^-1[i k_a F_a[u]]."""
    return apply_axis(u, axis, d, lambda k: 1j * k)


# ----------------------------------------------------------------------------------
# faces of the virtual box
# ----------------------------------------------------------------------------------

FACES = [(a, s) for a in range(3) for s in range(2)]   # face index = 2*axis + side (0 = lo, 1 = hi)


def plane_slice(u: np.ndarray, axis: int, index: int) -> np.ndarray:
    """The virtual plane normal to `axis` at node `index`; array [slow, fast] in-plane axes."""
    if axis == 0:
        return u[:, :, index]      # [z, y]
    if axis == 1:
        return u[:, index, :]      # [z, x]
    return u[index, :, :]          # [y, x]


def in_plane_axes(axis: int):
    """(fast, slow) in-plane physical axes of the plane normal to `axis`."""
    return {0: (1, 2), 1: (0, 2), 2: (0, 1)}[axis]


# ----------------------------------------------------------------------------------
# the simulation
# ----------------------------------------------------------------------------------

class Simulation:
    """Leapfrog PSTD run of one incident plane wave on a GridSpec (Eq. PSTDupdating)."""

    def __init__(self, spec, V, khat, k, ramp_time, window=None, omegas=None, probes=None, packet=None, aux=None):
        self.spec = spec
        hb, m = spec.hbar, spec.mass
        self.V = np.asarray(V, dtype=np.float64)
        self.k = float(k)
        self.khat = np.asarray(khat, dtype=float) / np.linalg.norm(khat)
        self.kvec = self.k * self.khat
        self.E0 = hb * hb * self.k ** 2 / (2.0 * m)
        self.w0 = self.E0 / hb
        self.ramp_time = float(ramp_time)
        # optional Gaussian wave-packet incidence (sigma, d0): the packet's centre starts at
        # d0 on the axis d = khat . (r - r_O) and moves along +khat (replaces the CW wave)
        self.packet = None if packet is None else (float(packet[0]), float(packet[1]))
        # optional 1-D auxiliary incident wave (aux_oracle.AuxSource1D, Section 2.2.3): read at
        # d = khat . (r - r_O); replaces the CW wave (k sets eta and the default DFT frequency)
        self.aux = aux
        self.eta = eta(self.E0, spec.dt, hb)
        self.kin_coef = hb * hb / (2.0 * m) * self.eta
        # mask Gamma = Gamma_x Gamma_y Gamma_z (Eq. Gamma)
        g = [mask_1d(spec.n[a], spec.abc_cells[a], spec.abc_profile, spec.abc_param, self.E0, spec.dt, hb)
             for a in range(3)]
        self.Gamma = g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :]
        # incident-wave spatial phase exp(i k . (r - r_O)) (Eqs. khat, Oinc, inc_d)
        self.rO = first_contact_corner(self.khat, spec)
        x = [coords(spec.n[a], spec.d[a]) for a in range(3)]
        ph = [np.exp(1j * self.kvec[a] * (x[a] - self.rO[a])) for a in range(3)]
        self.inc_phase = ph[2][:, None, None] * ph[1][None, :, None] * ph[0][None, None, :]
        dd = [self.khat[a] * (x[a] - self.rO[a]) for a in range(3)]
        self.inc_d = dd[2][:, None, None] + dd[1][None, :, None] + dd[0][None, None, :]   # Eq. inc_d
        # taper zeta and the source factor of Eq. tildeSchrodinger
        zt = [zeta_1d(spec.n[a], spec.d[a], spec.tfsf_lo[a], spec.tfsf_hi[a], spec.taper_cells) for a in range(3)]
        Z = [z[0] for z in zt]
        Z1 = [z[1] for z in zt]
        Z2 = [z[2] for z in zt]

        def outer(fx, fy, fz):
            return fz[:, None, None] * fy[None, :, None] * fx[None, None, :]

        self.zeta = outer(Z[0], Z[1], Z[2])
        lap_zeta = outer(Z2[0], Z[1], Z[2]) + outer(Z[0], Z2[1], Z[2]) + outer(Z[0], Z[1], Z2[2])
        k_grad_zeta = (self.kvec[0] * outer(Z1[0], Z[1], Z[2]) + self.kvec[1] * outer(Z[0], Z1[1], Z[2])
                       + self.kvec[2] * outer(Z[0], Z[1], Z1[2]))
        # hbar^2/2m (lap(zeta) psi_inc + 2 grad(zeta) . grad(psi_inc)), grad psi_inc = i k psi_inc
        self.src_factor = hb * hb / (2.0 * m) * (lap_zeta + 2j * k_grad_zeta)
        self.lap_zeta, self.khat_grad_zeta = lap_zeta, k_grad_zeta / self.k
        if spec.tfsf_mode == "paper" and np.any((self.zeta < 1.0) & (self.V != 0.0)):
            raise ValueError("V must vanish where zeta < 1 ((zeta - 1) V = 0)")
        self.prev = np.zeros(spec.shape, dtype=np.complex128)
        self.cur = np.zeros(spec.shape, dtype=np.complex128)
        self.n = 0
        # DFT state (Eqs. psiphasor, dpsiphasor, incpsiphasor)
        self.window = window
        self.omegas = list(omegas) if omegas is not None else ([self.w0] if window is not None else [])
        self.acc_psi = [[np.zeros(plane_slice(self.cur, a, 0).shape, dtype=np.complex128) for (a, s) in FACES]
                        for _ in self.omegas]
        self.acc_dpsi = [[np.zeros_like(p) for p in row] for row in self.acc_psi]
        self.acc_inc = np.zeros(len(self.omegas), dtype=np.complex128)
        # optional running DFT of the full state at probe nodes (i, j, k)
        self.probes = [tuple(p) for p in probes] if probes is not None else []
        self.acc_probe = np.zeros((len(self.omegas), len(self.probes)), dtype=np.complex128)

    # -- incident wave ---------------------------------------------------------------
    def inc_time_factor(self, n: int) -> complex:
        """The incident wave at O at step n: a(t_n) exp(-i w0 t_n), or the packet at d = 0."""
        t = n * self.spec.dt
        if self.aux is not None:
            return complex(self.aux.value(n, 0.0))
        if self.packet is not None:
            sig, d0 = self.packet
            return complex(gaussian_packet(0.0 - d0, t, self.k, sig, self.spec.hbar, self.spec.mass))
        return envelope(t, self.ramp_time) * complex(math.cos(self.w0 * t), -math.sin(self.w0 * t))

    def psi_inc(self, n: int) -> np.ndarray:
        if self.aux is not None:
            return self.aux.value(n, self.inc_d)
        if self.packet is not None:
            sig, d0 = self.packet
            return gaussian_packet(self.inc_d - d0, n * self.spec.dt, self.k, sig, self.spec.hbar, self.spec.mass)
        return self.inc_time_factor(n) * self.inc_phase

    # -- one leapfrog step -----------------------------------------------------------
    def advance(self, prev: np.ndarray, cur: np.ndarray, n: int) -> np.ndarray:
        """psi^{n+1} from psi^{n-1}, psi^n (Eq. PSTDupdating with Eq. expmask)."""
        spec = self.spec
        hb = spec.hbar
        Hu = self.kin_coef * kinetic(cur, spec.d)
        pinc = self.psi_inc(n)
        if spec.tfsf_mode == "exact":
            Hu = Hu + self.V * (cur + pinc)
        elif spec.tfsf_mode == "paper" and self.aux is not None:
            # grad psi_inc = khat d psi_inc / d d (Eq. pstd_dpsiinc)
            dpinc = self.aux.derivative(n, self.inc_d)
            Hu = Hu + self.V * cur + hb * hb / (2.0 * spec.mass) * (self.lap_zeta * pinc + 2.0 * self.khat_grad_zeta * dpinc)
        elif spec.tfsf_mode == "paper":
            Hu = Hu + self.V * cur + self.src_factor * pinc
        else:
            raise ValueError(spec.tfsf_mode)
        return self.Gamma * (prev - (2j * spec.dt / hb) * Hu)

    def accumulate(self):
        """Add the state psi^n and its normal derivatives on the six planes to the DFT sums."""
        spec = self.spec
        t = self.n * spec.dt
        ders = [derivative(self.cur, a, spec.d[a]) for a in range(3)]
        for fi, w in enumerate(self.omegas):
            e = complex(math.cos(w * t), math.sin(w * t))        # exp(+i w t_n) (Eq. psiphasor)
            for face, (a, s) in enumerate(FACES):
                h = spec.huygens_lo[a] if s == 0 else spec.huygens_hi[a]
                self.acc_psi[fi][face] += e * plane_slice(self.cur, a, h)
                self.acc_dpsi[fi][face] += e * plane_slice(ders[a], a, h)
            self.acc_inc[fi] += e * self.inc_time_factor(self.n)
            for pi, (i, j, k) in enumerate(self.probes):
                self.acc_probe[fi, pi] += e * self.cur[k, j, i]

    def in_window(self, n: int) -> bool:
        return self.window is not None and self.window[0] <= n < self.window[0] + self.window[1]

    def step(self, count: int = 1):
        for _ in range(count):
            if self.in_window(self.n):
                self.accumulate()
            nxt = self.advance(self.prev, self.cur, self.n)
            self.prev, self.cur = self.cur, nxt
            self.n += 1

    def scaled_phasors(self, fi: int = 0):
        """Phasors divided by the incident phasor at O (Eqs. scaledphsiphasor, scaleddpsiphasor)."""
        s = self.acc_inc[fi]
        return [(p / s, q / s) for p, q in zip(self.acc_psi[fi], self.acc_dpsi[fi])]

    def scaled_probes(self, fi: int = 0) -> np.ndarray:
        return self.acc_probe[fi] / self.acc_inc[fi]

    def scattered_field(self) -> np.ndarray:
        """psi^n with the incident part removed where the state holds the total field."""
        if self.spec.tfsf_mode == "exact":
            return self.cur.copy()
        return self.cur - self.zeta * self.psi_inc(self.n)
