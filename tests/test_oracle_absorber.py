"""Pin of the oracle's Poschl-Teller absorbing mask (Eqs. Poshcl-Teller, expmask, Gamma).

CPU only.  A Gaussian packet is run by the oracle's leapfrog into the masking layer with
the parameters the paper prints for its validation runs (Section 4: U0 = 5.0, alpha = 0.1
per grid, a 40-grid layer, 20 grids per wavelength, dtau = pi/1000).  The packet's
reflected and transmitted norms are compared with the same profile taken as a continuum
negative imaginary potential (Eq. NIP) and solved as a stationary scattering problem by a
transfer matrix written here, independently of the oracle.

Reading: the mask e^{-gamma dt} of Eq. expmask multiplies psi^{n+1}, which the leapfrog
forms from psi^{n-1}, i.e. once per 2 dt of the three-level recursion.  Each Fourier mode's
amplitude then decays by e^{-gamma dt / 2} per step: the continuum equivalent is the NIP
-i hbar gamma / 2.  The test also checks that the NIP -i hbar gamma would not match.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import pstd_oracle as po
from paper_2403_04053_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
PT = GOLDEN["absorber_example"]
STAB = GOLDEN["stability_example"]

LAM = 1.0
K0 = 2 * math.pi / LAM
E0 = 0.5 * K0 * K0                      # hbar = m = 1
DZ = STAB["dx_bar_over_pi"] * math.pi / K0   # dx_bar = k0 dx = pi/10: 20 grids per wavelength
DT = STAB["dtau_over_pi"] * math.pi / E0     # dtau = E0 dt / hbar = pi/1000
W = int(PT["width_cells"])
N = 320                                 # 240 free cells between the two 40-cell layers
SIGMA, Z0 = 1.0, -2.0                   # packet exp(-(z - z0)^2 / (4 sigma^2) + i k0 z)


def packet_spec(profile_param):
    # a thin periodic box along z: the packet is uniform in x and y, so only the z lines act
    return inputs.GridSpec(n=(2, 2, N), d=(1.0, 1.0, DZ), dt=DT, abc_cells=(0, 0, W), abc_profile="poschl_teller",
                           abc_param=profile_param, tfsf_lo=(0, 0, 100), tfsf_hi=(1, 1, 220), taper_cells=1,
                           huygens_lo=(0, 0, 90), huygens_hi=(1, 1, 230))


def run_packet(t_end=2.9):
    """Oracle run of the packet; returns (reflected, transmitted) norm fractions measured in the
    free region once both parts have left the layers (split by the sign of k)."""
    spec = packet_spec((PT["U0"], PT["alpha_per_cell"]))
    z = po.coords(N, DZ)
    psi0 = np.exp(-(z - Z0) ** 2 / (4 * SIGMA * SIGMA) + 1j * K0 * z)
    # psi^{-1}: each mode stepped back by its own leapfrog root e^{-i theta}, sin theta =
    # dt eta k^2 / 2 (the packet starts in the free region, where the mask is 1)
    k = 2 * math.pi * np.fft.fftfreq(N, DZ)
    eta = math.sin(E0 * DT) / (E0 * DT)
    theta = np.arcsin(DT * eta * k * k / 2)
    psim1 = np.fft.ifft(np.exp(1j * theta) * np.fft.fft(psi0))
    sim = po.Simulation(spec, np.zeros(spec.shape), (0, 0, 1), K0, 0.0)
    sim.prev = np.broadcast_to(psim1[:, None, None], spec.shape).copy()
    sim.cur = np.broadcast_to(psi0[:, None, None], spec.shape).copy()
    sim.step(int(round(t_end / DT)))
    u = sim.cur[:, 0, 0].copy()
    u[:W] = 0
    u[N - W:] = 0
    U = np.fft.fft(u)
    norm0 = np.sum(np.abs(psi0) ** 2)
    return (float(np.sum(np.abs(U[k < 0]) ** 2) / N / norm0), float(np.sum(np.abs(U[k > 0]) ** 2) / N / norm0),
            np.abs(np.fft.fft(psi0)) ** 2, k)


def continuum_R_T(kk, nip_factor, sub=16):
    """|r|^2, |t|^2 of a unit plane wave e^{i k z} on the absorbing region of the periodic box
    (the right layer, the wrap, the left layer) with the potential -i hbar nip_factor gamma(z),
    gamma(d) = U0 E0/hbar / cosh^2(alpha d), d the distance in cells from the outermost node,
    cut off half a cell beyond the layer's last node.  Piecewise-constant transfer matrix."""
    U0, alpha = PT["U0"], PT["alpha_per_cell"]
    s_lo, s_hi = N - W - 0.5, N + W - 0.5               # node coordinate, unwrapped across the edge
    edges = s_lo + np.arange(int(round((s_hi - s_lo) * sub)) + 1) / sub
    s = 0.5 * (edges[1:] + edges[:-1])
    d = np.maximum(np.where(s <= N - 0.5, (N - 1) - s, s - N), 0.0)
    gam = np.where(d < W - 0.5, U0 * E0 / np.cosh(alpha * d) ** 2, 0.0)
    E = 0.5 * kk * kk
    kap = np.sqrt(2 * (E + 1j * nip_factor * gam) + 0j)
    kaps = np.concatenate([[kk + 0j], kap, [kk + 0j]])
    x = (edges - s_lo) * DZ
    M = np.eye(2, dtype=complex)

    def D(q, xj):
        e, f = np.exp(1j * q * xj), np.exp(-1j * q * xj)
        return np.array([[e, f], [1j * q * e, -1j * q * f]])

    for j, xj in enumerate(x):
        M = np.linalg.solve(D(kaps[j + 1], xj), D(kaps[j], xj)) @ M
    r = -M[1, 0] / M[1, 1]
    t = M[0, 0] + M[0, 1] * r
    return abs(r) ** 2, abs(t) ** 2


def continuum_norms(weights, k, nip_factor):
    R = T = 0.0
    for kk, w in zip(k, weights):
        if kk > 0 and w > 1e-14 * weights.max():
            r2, t2 = continuum_R_T(kk, nip_factor)
            R += w * r2
            T += w * t2
    return R / weights.sum(), T / weights.sum()


@pytest.fixture(scope="module")
def measured():
    return run_packet()


def test_poschl_teller_layer_matches_the_continuum_nip(measured):
    R, T, wts, k = measured
    Rc, Tc = continuum_norms(wts, k, 0.5)
    # the continuum model fixes the cut-off step only to within a cell: 3% on R (a 40-cell
    # smooth layer reflects 3.4e-5 of the norm) and 10% on the 1.5e-6 that crosses both layers
    assert abs(R - Rc) < 3e-2 * Rc
    assert abs(T - Tc) < 1e-1 * Tc
    # the mask damps at gamma / 2 per unit time: the full-gamma NIP is far off
    Rf, Tf = continuum_norms(wts, k, 1.0)
    assert abs(R - Rf) > 0.3 * Rf and T > 100 * Tf


def test_poschl_teller_pin_catches_planted_mistakes(measured, monkeypatch):
    """Plausible misreadings of Eq. Poshcl-Teller or Eq. expmask, planted in the oracle, fail the pin."""
    base_gamma = po.absorber_gamma
    base_mask = po.mask_1d
    _, _, wts, k = measured
    Rc, Tc = continuum_norms(wts, k, 0.5)

    def inner_origin(n, width, profile, param, E0_, hbar=1.0):
        # d measured from the inner edge of the layer instead of its outermost surface
        g = base_gamma(n, width, profile, param, E0_, hbar)
        i = np.arange(n)
        dist = np.minimum(i, n - 1 - i)
        return np.where(dist < width, g[np.clip(width - 1 - dist, 0, n - 1)], 0.0)

    def cosh_once(n, width, profile, param, E0_, hbar=1.0):
        # 1/cosh instead of 1/cosh^2
        g = base_gamma(n, width, profile, param, E0_, hbar)
        return np.sqrt(np.maximum(g, 0.0) * float(param[0]) * E0_ / hbar)

    def double_mask(n, width, profile, param, E0_, dt, hbar=1.0):
        # e^{-2 gamma dt} per step
        return base_mask(n, width, profile, param, E0_, dt, hbar) ** 2

    for name, fn in (("absorber_gamma", inner_origin), ("absorber_gamma", cosh_once), ("mask_1d", double_mask)):
        monkeypatch.setattr(po, name, fn)
        R, T, _, _ = run_packet()
        monkeypatch.setattr(po, "absorber_gamma", base_gamma)
        monkeypatch.setattr(po, "mask_1d", base_mask)
        assert abs(R - Rc) > 3e-2 * Rc or abs(T - Tc) > 1e-1 * Tc, name


def test_poschl_teller_profile_values_at_the_paper_parameters():
    """The 40-cell layer at U0 = 5, alpha = 0.1 per cell: gamma is U0 at the outermost node and
    falls monotonically to U0 / cosh^2(3.9) at the innermost, and is 0 in the free region."""
    g = po.absorber_gamma(N, W, "poschl_teller", (PT["U0"], PT["alpha_per_cell"]), E0)
    assert g[0] == pytest.approx(PT["U0"] * E0) and g[N - 1] == pytest.approx(PT["U0"] * E0)
    assert np.all(np.diff(g[:W]) < 0) and np.all(np.diff(g[N - W:]) > 0)
    assert g[W - 1] == pytest.approx(PT["U0"] * E0 / math.cosh(PT["alpha_per_cell"] * (W - 1)) ** 2)
    assert np.all(g[W:N - W] == 0.0)
