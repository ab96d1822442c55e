"""Pins of the 1-D auxiliary incident wave (oracle/aux_oracle.py, Section 2.2.3).

* the read-out series (Eq. pstd_psiinc) interpolates the 1-D samples exactly, and its
  derivative (Eq. pstd_dpsiinc) of one Fourier mode is i q times the mode;
* each Fourier mode of the literal 1-D leapfrog follows the scheme's closed form z+^n,
  z+ = -i a + sqrt(1 - a^2), a = dt eta hbar q^2 / 2m (Eq. Joukowsky's root);
* at the carrier, eta makes z+ = exp(-i E dt / hbar): a carrier-mode profile reproduces the
  CW plane wave, so a 3-D run driven by it equals the CW run with no ramp, in both TF/SF
  forms (this ties the auxiliary source to the pinned CW path; a sign error planted in the
  derivative weights breaks the PAPER-form case);
* a Gaussian profile evolved by the 1-D leapfrog stays close to the free packet in closed
  form (the leapfrog's dispersion error only), and the 3-D run driven by it stays close to
  the closed-form packet run.
"""
import math

import numpy as np
import pytest

from oracle import aux_oracle as ao
from oracle import pstd_oracle as po
from paper_2403_04053_gb300 import inputs

K = 2 * math.pi
E0 = 0.5 * K * K
KHAT = (0.3, -0.5, 0.81)


def spec(mode="exact"):
    return inputs.GridSpec(n=(24, 32, 48), d=(0.25, 0.3, 0.2), dt=0.002, abc_cells=(4, 5, 6), tfsf_lo=(9, 12, 17),
                           tfsf_hi=(15, 20, 31), taper_cells=2, huygens_lo=(7, 9, 14), huygens_hi=(17, 23, 34),
                           tfsf_mode=mode)


def random_core_V(sp, seed, amp=3.0):
    rng = np.random.default_rng(seed)
    V = np.zeros(sp.shape)
    c = sp.core_box()
    V[c[2][0]:c[2][1] + 1, c[1][0]:c[1][1] + 1, c[0][0]:c[0][1] + 1] = rng.uniform(
        -amp, amp, (c[2][1] - c[2][0] + 1, c[1][1] - c[1][0] + 1, c[0][1] - c[0][0] + 1))
    return V


def test_series_interpolates_the_samples_and_differentiates_modes():
    rng = np.random.default_rng(1)
    n1, dd, d_lo = 64, 0.2, -3.3
    psi0 = rng.standard_normal(n1) + 1j * rng.standard_normal(n1)
    aux = ao.AuxSource1D(d_lo, dd, psi0, E0, 0.002)
    d = d_lo + dd * np.arange(n1)
    assert np.max(np.abs(aux.value(0, d) - psi0)) < 1e-12
    # one mode l: exp(i q_l (d - d_lo)) at any d, derivative i q_l times it
    for l in (3, -7, 20):
        q = 2 * math.pi * l / (n1 * dd)
        mode = np.exp(1j * q * (d - d_lo))
        a1 = ao.AuxSource1D(d_lo, dd, mode, E0, 0.002)
        x = np.array([-2.71, 0.0, 1.234, 7.5])
        assert np.max(np.abs(a1.value(0, x) - np.exp(1j * q * (x - d_lo)))) < 1e-12
        assert np.max(np.abs(a1.derivative(0, x) - 1j * q * np.exp(1j * q * (x - d_lo)))) < 1e-11 * abs(q)


def test_leapfrog_modes_follow_the_closed_form_root():
    rng = np.random.default_rng(2)
    n1, dd, dt = 128, 0.25, 0.003
    psi0 = rng.standard_normal(n1) + 1j * rng.standard_normal(n1)
    aux = ao.AuxSource1D(-10.0, dd, psi0, E0, dt)
    q = po.wavenumbers(n1, dd)
    a = dt * po.eta(E0, dt) * q ** 2 / 2
    zp = -1j * a + np.sqrt(1 - a * a)
    F0 = np.fft.fft(psi0)
    for n in (1, 2, 17, 200):
        F = np.fft.fft(aux.level(n))
        assert np.max(np.abs(F - F0 * zp ** n)) < 1e-11 * np.max(np.abs(F0))


def test_unstable_axis_is_rejected():
    with pytest.raises(ValueError):
        ao.AuxSource1D(0.0, 0.05, np.ones(32), E0, 0.004)      # dt pi^2 / (2 dd^2) > 1


def carrier_aux(sp, n1=256):
    # an axis whose grid wavenumbers contain k = 2 pi: n1 dd = integer wavelengths
    dd = 0.125
    d_lo = -8.0
    d = d_lo + dd * np.arange(n1)
    return ao.AuxSource1D(d_lo, dd, np.exp(1j * K * d), E0, sp.dt)


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_carrier_mode_profile_reproduces_the_cw_run(mode):
    sp = spec(mode)
    V = random_core_V(sp, 4)
    win = (10, 20)
    cw = po.Simulation(sp, V, KHAT, K, 0.0, window=win)
    ax = po.Simulation(sp, V, KHAT, K, 0.0, window=win, aux=carrier_aux(sp))
    cw.step(40)
    ax.step(40)
    assert np.linalg.norm(ax.cur - cw.cur) <= 1e-11 * np.linalg.norm(cw.cur)
    for (p1, q1), (p2, q2) in zip(ax.scaled_phasors(0), cw.scaled_phasors(0)):
        assert np.linalg.norm(p1 - p2) <= 1e-10 * np.linalg.norm(p2)
        assert np.linalg.norm(q1 - q2) <= 1e-10 * np.linalg.norm(q2)


def test_planted_derivative_sign_error_is_caught(monkeypatch):
    sp = spec("paper")
    V = random_core_V(sp, 4)
    cw = po.Simulation(sp, V, KHAT, K, 0.0)
    aux = carrier_aux(sp)
    good = aux.derivative
    monkeypatch.setattr(aux, "derivative", lambda n, d: -good(n, d))
    ax = po.Simulation(sp, V, KHAT, K, 0.0, aux=aux)
    cw.step(20)
    ax.step(20)
    assert np.linalg.norm(ax.cur - cw.cur) > 1e-3 * np.linalg.norm(cw.cur)


def test_gaussian_profile_tracks_the_free_packet():
    # sigma = 1, k = 2 pi: the 1-D leapfrog differs from the free evolution only by its
    # dispersion away from the carrier, |asin(a)/dt - hbar q^2/2m| t over the packet's band
    sig, d0 = 1.0, -5.0
    n1, dd, dt = 256, 0.125, 0.002
    d = -16.0 + dd * np.arange(n1)
    aux = ao.AuxSource1D(-16.0, dd, po.gaussian_packet(d - d0, 0.0, K, sig), E0, dt)
    x = np.linspace(-8.0, 6.0, 57)
    # |exp(-i W t) - exp(-i w t)| <= |W - w| t per mode, weighted by the packet's spectrum
    # 2 sigma sqrt(pi) exp(-sigma^2 (q - k)^2) / 2 pi (W = asin(a)/dt, w = q^2/2)
    q = np.linspace(K - 8 / sig, K + 8 / sig, 20001)
    W = np.arcsin(dt * po.eta(E0, dt) * q ** 2 / 2) / dt
    spread = np.trapezoid(2 * sig * math.sqrt(math.pi) * np.exp(-(sig * (q - K)) ** 2) * np.abs(W - q ** 2 / 2), q)
    for n in (0, 100, 400):
        ref = po.gaussian_packet(x - d0, n * dt, K, sig)
        err = np.max(np.abs(aux.value(n, x) - ref))
        assert err < 1e-12 + 1.05 * n * dt * spread / (2 * math.pi)
    # the 3-D run driven by it, against the closed-form packet run
    sp = spec()
    V = random_core_V(sp, 5)
    a3 = po.Simulation(sp, V, KHAT, K, 0.0, aux=ao.AuxSource1D(-16.0, dd, po.gaussian_packet(d - d0, 0.0, K, sig),
                                                              E0, sp.dt))
    p3 = po.Simulation(sp, V, KHAT, K, 0.0, packet=(sig, d0))
    a3.step(60)
    p3.step(60)
    assert np.linalg.norm(a3.cur - p3.cur) < 1e-2 * np.linalg.norm(p3.cur)
