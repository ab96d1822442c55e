"""FP64 CPU oracle: the 1-D auxiliary incident wave of Section 2.2.3.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For an incident packet of arbitrary shape the paper solves the free 1-D Schroedinger equation
along the incidence axis d = khat . (r - r_O) (Eq. inc_d) alongside the 3-D problem, and reads
the wave and its derivative at each node's d from the 1-D grid's Fourier series
(Eqs. pstd_psiinc, pstd_dpsiinc).  Here, step by step:

  * the 1-D axis: d_m = d_lo + m dd, m = 0..n1-1, periodic (the FFT's), free space (V = 0);
  * its update: the leapfrog of Eq. PSTDupdating in one dimension, with the spectral kinetic
    term of Eq. spatialFFTeigen and the 3-D run's eta (Eq. numdis2) and dt;
  * the 1-D start: psi1^0 is the given profile; psi1^{-1} is one exact backward step of that
    same discrete scheme, mode by mode (so that the leapfrog's computational mode is not
    excited; the paper does not say how the 1-D run starts);
  * the read-out: psi_inc(d) = (1/n1) sum_l F_l exp(i q_l (d - d_lo)) and
    d psi_inc / d d = (1/n1) sum_l i q_l F_l exp(i q_l (d - d_lo)), l = -n1/2..n1/2-1, with
    F = FFT(psi1^n) (the paper writes d from the axis origin; here the origin is d_lo).
"""
from __future__ import annotations

import numpy as np

from .pstd_oracle import eta, wavenumbers


class AuxSource1D:
    """The 1-D auxiliary incident wave, evolved by the literal leapfrog and cached per level."""

    def __init__(self, d_lo: float, dd: float, psi0, E0: float, dt: float, hbar: float = 1.0, mass: float = 1.0):
        self.d_lo, self.dd = float(d_lo), float(dd)
        psi0 = np.asarray(psi0, dtype=np.complex128)
        self.n1 = psi0.size
        self.q = wavenumbers(self.n1, self.dd)
        self.hbar, self.mass, self.dt = hbar, mass, dt
        self.eta = eta(E0, dt, hbar)
        a = dt * self.eta * hbar * self.q ** 2 / (2.0 * mass)
        if np.any(a > 1.0):
            raise ValueError("the 1-D leapfrog is unstable on this axis (dt eta hbar q^2 / 2m > 1)")
        zp = -1j * a + np.sqrt(1.0 - a * a)          # the scheme's physical root: F^{n+1} = zp F^n
        self.levels = [np.fft.ifft(np.fft.fft(psi0) / zp), psi0]   # psi1^{-1}, psi1^0

    def _kinetic(self, u):
        return np.fft.ifft(self.q ** 2 * np.fft.fft(u))

    def level(self, n: int) -> np.ndarray:
        """psi1^n (n >= -1), advancing the leapfrog as far as needed."""
        c = 2j * self.dt / self.hbar * self.eta * self.hbar ** 2 / (2.0 * self.mass)
        while len(self.levels) - 2 < n:
            prev, cur = self.levels[-2], self.levels[-1]
            self.levels.append(prev - c * self._kinetic(cur))
        return self.levels[n + 1]

    def _phases(self, d):
        """exp(i q_l (d - d_lo)) for every d (cached for the last large array of d, which the 3-D
        run passes every step)."""
        if d.size > 64 and getattr(self, "_ph_key", None) is d:
            return self._ph
        ph = np.exp(1j * np.multiply.outer(d.ravel() - self.d_lo, self.q))
        if d.size > 64:
            self._ph_key, self._ph = d, ph
        return ph

    def _series(self, n: int, d, weights):
        F = np.fft.fft(self.level(n)) * weights
        arr = np.asarray(d, dtype=float)
        return (self._phases(arr) @ F / self.n1).reshape(arr.shape)

    def value(self, n: int, d):
        """psi_inc^n at axis coordinates d (Eq. pstd_psiinc)."""
        return self._series(n, d, 1.0)

    def derivative(self, n: int, d):
        """d psi_inc^n / d d at axis coordinates d (Eq. pstd_dpsiinc without the khat factor)."""
        return self._series(n, d, 1j * self.q)
