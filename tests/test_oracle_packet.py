"""Pins of the oracle's wave-packet incidence (CPU).

The closed-form Gaussian packet must solve the free 1-D Schrodinger equation (and a planted
sign error must not), conserve its norm and move at the group velocity hbar k / m; and,
since the scattering problem is linear and time-invariant, the scaled phasors of one packet
run at frequency w must reproduce the steady state of a CW run at energy hbar w (exact at
the carrier, to the leapfrog's carrier-tuned dispersion factor eta elsewhere).
"""
import math

import numpy as np
import pytest

from oracle import ntdf_oracle as no
from oracle import pstd_oracle as po
from paper_2403_04053_gb300 import inputs

K = 2 * math.pi


def _free_residual(fn, sig=1.5, t=0.37):
    L, N = 80.0, 4096
    x = (np.arange(N) - N / 2) * (L / N)
    h = 1e-5
    psi = fn(x, t, K, sig)
    dt_psi = (fn(x, t + h, K, sig) - fn(x, t - h, K, sig)) / (2 * h)
    kk = 2 * math.pi * np.fft.fftfreq(N, L / N)
    lap = np.fft.ifft(-(kk ** 2) * np.fft.fft(psi))
    return np.abs(1j * dt_psi + 0.5 * lap).max() / np.abs(0.5 * lap).max()


def test_gaussian_packet_solves_the_free_equation():
    assert _free_residual(po.gaussian_packet) < 1e-6

    def wrong(x, t, k, sigma):   # spreading with the wrong sign of tau
        return po.gaussian_packet(x, -t, k, sigma) * np.exp(-1j * k * k * t)
    assert _free_residual(wrong) > 1e-2


def test_packet_norm_and_group_velocity():
    x = np.linspace(-40, 60, 20001)
    dx = x[1] - x[0]
    for t in (0.0, 1.0, 3.0):
        p = np.abs(po.gaussian_packet(x, t, K, 1.2)) ** 2
        norm = p.sum() * dx
        assert abs(norm - math.sqrt(2 * math.pi) * 1.2) < 1e-9 * norm
        assert abs((x * p).sum() * dx / norm - K * t) < 1e-6


def test_packet_run_reproduces_cw_cross_sections():
    spec = inputs.GridSpec(n=(24, 24, 24), d=(0.25, 0.25, 0.25), dt=0.004, abc_cells=(4, 4, 4), tfsf_lo=(6, 6, 6),
                           tfsf_hi=(17, 17, 17), taper_cells=2, huygens_lo=(5, 5, 5), huygens_hi=(18, 18, 18))
    x = [spec.coords(a) for a in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    V = 6.0 * np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * 0.5 ** 2))
    c = spec.core_box()
    inside = np.zeros(spec.shape, bool)
    inside[c[2][0]:c[2][1] + 1, c[1][0]:c[1][1] + 1, c[0][0]:c[0][1] + 1] = True
    V[~inside] = 0
    w0 = K * K / 2
    oms = [0.9 * w0, w0, 1.1 * w0]
    th, ph = np.deg2rad([10.0, 60.0, 120.0, 170.0]), np.zeros(4)
    sim = po.Simulation(spec, V, (0, 0, 1), K, 0.0, window=(0, 1200), omegas=oms, packet=(1.0, -6.0))
    sim.step(1200)
    for i, (w, tol) in enumerate(zip(oms, (2e-2, 1e-3, 2e-2))):
        kw = math.sqrt(2 * w)
        cw = po.Simulation(spec, V, (0, 0, 1), kw, 0.5, window=inputs.dft_window(w, spec.dt, 900), omegas=[w])
        cw.step(900)
        fc = no.cross_section(spec, kw, cw.scaled_phasors(0), th, ph)[1]
        fp = no.cross_section(spec, kw, sim.scaled_phasors(i), th, ph)[1]
        assert np.linalg.norm(fp - fc) < tol * np.linalg.norm(fc)
